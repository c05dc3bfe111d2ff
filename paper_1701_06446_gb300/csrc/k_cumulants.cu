// Moment-to-cumulant recovery (Algorithms 3-4) and cumulant norms (Eq. me,
// Algorithm 5), FP64.
//
// Algorithm 4 sums, for every element, products of lower-order cumulants over
// all set partitions of its s indices.  Grouping those partitions by the part
// that holds the first index gives the equivalent subset recursion
//     C_s[i] = M_s[i] - sum_{A contains index 1, A != all} C_|A|[i_A] M_{s-|A|}[i_rest]
// (2^{s-1} - 1 terms instead of B(s) - 1), which is what runs here.  With
// M = S/T it is evaluated as C_s = (S_s[i] - sum_A C_|A|[i_A] S_rest[i_rest]) / T:
// one FP64 multiply-add per subset and one scaling per element (FP64 is the
// scarce pipe on this GPU, so the kernel keeps everything else off it).
//
// For a sorted block j every sub-tuple j_A is sorted, so each operand is a
// stored block whose rank comes from a per-block table, and its in-block
// offset follows from the element's own in-block digits because diagonal
// blocks are stored whole.  The code is specialised per order: the subset
// masks are compile-time constants, each thread owns one in-block offset and
// computes its per-subset operand offsets once; the per-block sub-block ranks
// come from a table all threads of a block read together.  The same pass
// accumulates multiplicity * C^2 (Algorithm 5 with k = 2).
//
// Two launch forms share that per-group routine:
//   * k_recover_fused: orders 1..min(d, 4) in one cooperative launch: every
//     sum takes the shift's workspace first, then orders 1-3 run together (a
//     higher order recomputes the C_1 / C_2 factors it needs from the sums
//     instead of waiting for them), a grid barrier, order 4, a grid barrier
//     and the norms; norm partials per work unit.
//   * k_cumulants<S>: one launch per order above 4, one norm partial per CTA,
//     reduced by k_norm_final.
#include <algorithm>

#include "cw_device.cuh"
#include "cw_internal.h"
#include "cw_tc.h"
#include "cw_tc_device.cuh"

namespace cw {

namespace {

constexpr int NT = 256;
constexpr long long kBarrierLimit = 1LL << 32;  // clock cycles (~2 s)

// Subset t (0 <= t < 2^{S-1} - 1) holds position 0 and the positions of the
// set bits of t shifted by one: mask = 2t + 1 (the host tables use this order).
template <int S>
struct Subsets {
    static constexpr int N = (1 << (S - 1)) - 1;
    static constexpr int ND = N > 0 ? N : 1;
};

__host__ __device__ constexpr int popc_c(unsigned x) { return x ? (int)(x & 1u) + popc_c(x >> 1) : 0; }

__host__ __device__ __forceinline__ int ipow_c(int b, int k)
{
    int r = 1;
    for (int i = 0; i < k; ++i) r *= b;
    return r;
}

// Per-thread constants of one in-block offset of order S.  Up to order 4 the
// in-block offsets of both factors of every subset are kept; above, only the
// digits, and each subset's offsets are formed when it is used (integer work
// is cheap next to the FP64 multiply-add it feeds).
constexpr int kKeepOffsets = 4;
template <int S>
struct Elem {
    static constexpr int NO = S <= kKeepOffsets ? Subsets<S>::ND : 1;
    int slot, off;
    bool valid;
    int dig[S];
    int offA[NO], offR[NO];  // in-block offsets of the two factors (S <= kKeepOffsets)
    int offL, offRw;         // workspace: in-block row / column
};

template <int S>
__device__ __forceinline__ void subset_offsets(const Elem<S>& c, int b, int t, int& oa, int& orr)
{
    if constexpr (S <= kKeepOffsets) {
        oa = c.offA[t];
        orr = c.offR[t];
    } else {
        const unsigned mask = 2u * t + 1u;
        oa = 0;
        orr = 0;
#pragma unroll
        for (int k = 0; k < S; ++k) {
            if ((mask >> k) & 1u) oa = oa * b + c.dig[k];
            else orr = orr * b + c.dig[k];
        }
    }
}

// Thread -> (slot, in-block offset): `slots` blocks per CTA when b^S < NT,
// else slice y of NT offsets of one block.
template <int S, bool V = false>
__device__ __forceinline__ Elem<S> make_elem(int b, int bs, int bR, int slots, int y)
{
    Elem<S> c;
    const int tid = vtid<V>();
    if (slots == 1) {
        c.slot = 0;
        c.off = y * NT + tid;
    } else {
        c.slot = tid / bs;
        c.off = tid - c.slot * bs;
    }
    c.valid = c.slot < slots && c.off < bs;
    int rem = c.off;
#pragma unroll
    for (int k = S - 1; k >= 0; --k) {
        const int q = rem / b;
        c.dig[k] = rem - q * b;
        rem = q;
    }
    if constexpr (S <= kKeepOffsets) {
#pragma unroll
        for (int t = 0; t < Subsets<S>::N; ++t) {
            const unsigned mask = 2u * t + 1u;
            int oa = 0, orr = 0;
#pragma unroll
            for (int k = 0; k < S; ++k) {
                if ((mask >> k) & 1u) oa = oa * b + c.dig[k];
                else orr = orr * b + c.dig[k];
            }
            c.offA[t] = oa;
            c.offR[t] = orr;
        }
    }
    c.offL = c.off / bR;
    c.offRw = c.off - c.offL * bR;
    return c;
}

// FIFO slot of the batch that leaves with this shift: head / p.
__device__ __forceinline__ int64_t fifo_slot(const CumArgs& a)
{
    const int64_t hd = *a.head;
    return hd < ((int64_t)1 << 31) ? (int64_t)((unsigned)hd / (unsigned)a.p) : hd / a.p;
}

// Fold the shift's workspace into one element e of S_s (block blk, in-block
// offset off): S += (double)D_in - (double)D_out (CumArgs::accum).  Split in
// a load half and a store half so that callers can keep several elements'
// loads in flight.
struct FoldVal {
    double* sp;    // the sum
    float* fptr;   // FIFO entry (accum 2) or null
    double s;
    float din, dout;
};

// Workspace slot of (block blk, in-block offset off) of an order.
__device__ __forceinline__ int64_t wslot(const CumArgs& a, int64_t blk, int off)
{
    const int offL = off / a.bR, offRw = off - (off / a.bR) * a.bR;
    const int2 wb = *reinterpret_cast<const int2*>(a.wblk + 2 * blk);
    return (int64_t)wb.x + (int64_t)offL * wb.y + offRw;
}

// Workspace slot of a canonical element of block blk whose left / right
// digits have the ranks lr >> 16, lr & 0xffff (compressed update tables).
__device__ __forceinline__ int64_t wslot_lr(const CumArgs& a, int64_t blk, int lr)
{
    const int2 wb = *reinterpret_cast<const int2*>(a.wblk + 2 * blk);
    return (int64_t)wb.x + (int64_t)((unsigned)lr >> 16) * wb.y + (lr & 0xffff);
}

// Load half of the fold of the element at workspace slot w whose sum lives
// at S_s[si] (si = w when the order's sums are in workspace order).
__device__ __forceinline__ FoldVal fold_load_at(const CumArgs& a, int64_t w, int64_t si, int64_t fslot)
{
    FoldVal v;
    v.fptr = nullptr;
    if (a.accum == 1) {
        sum_partials(a.W + a.woff + w, a.wslice, a.ksplit, v.din, v.dout);
    } else {
        v.din = sum_in_partials(a.W + a.woff + w, a.wslice, a.ksplit);
        v.fptr = a.fifo + fslot * a.fstride + w;  // FIFO in workspace order
        v.dout = *v.fptr;
    }
    v.sp = a.S[a.s] + si;
    v.s = *v.sp;
    return v;
}

__device__ __forceinline__ FoldVal fold_load(const CumArgs& a, int64_t blk, int off, int64_t e, int64_t fslot)
{
    const int64_t w = wslot(a, blk, off);
    return fold_load_at(a, w, a.sgemm ? w : e, fslot);
}

__device__ __forceinline__ void fold_store(const FoldVal& v)
{
    *v.sp = v.s + (f32_to_f64(v.din) - f32_to_f64(v.dout));
    if (v.fptr != nullptr) *v.fptr = v.din;
}

__device__ __forceinline__ void fold_elem(const CumArgs& a, int64_t blk, int off, int64_t e, int64_t fslot)
{
    fold_store(fold_load(a, blk, off, e, fslot));
}

// Two-word FP32 arithmetic for the subset sums of the mixed forms (a value
// is hi + lo).  The product of two such values uses Dekker's exact product
// (the rounding error of hi*hi recovered with one fused multiply-add, after
// Dekker 1971) plus the two cross terms; the running sum uses Knuth's
// two-sum for the high words and adds the errors into the low word.  Every
// operation is an explicitly rounded intrinsic, so the compiler cannot
// contract or reorder them.  The relative error of a sum of m products is
// about m * 2^-46 of the sum of the products' magnitudes, far below the
// error of the sums being recovered, at a few FP32 operations per product
// instead of one FP64 multiply-add on this GPU's narrow FP64 pipe.
__device__ __forceinline__ void tw_acc_prod(float& hi, float& lo, float2 a, float2 b)
{
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float s = __fadd_rn(hi, p);
    const float v = __fsub_rn(s, hi);
    const float t = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(p, v));
    lo = __fadd_rn(lo, __fadd_rn(t, e));
    hi = s;
}

// L2 eviction priorities of the canonical recovery.  Its operand gathers
// (two-word copies of the orders below, about 78 MB at n=48 d=6) are re-read
// across the whole launch, while ten times that in sums, tile sums, FIFO
// entries and cumulants pass through L2 once.  The gathers carry an
// evict-last policy and the once-touched accesses an evict-first one (PTX
// createpolicy + L2::cache_hint), so that the streamed lines leave L2 first.
__device__ __forceinline__ uint64_t l2_policy_evict_last()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_evict_first()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// A gather of read-only data (nothing in the launch writes it).
__device__ __forceinline__ float2 ld_keep(const float2* a, uint64_t pol)
{
    float2 v;
    asm("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol));
    return v;
}

// Once-touched loads and stores; volatile, so that each load stays before the
// store that follows it to the same address.
__device__ __forceinline__ float ld_once(const float* a, uint64_t pol)
{
    float v;
    asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
    return v;
}

__device__ __forceinline__ double ld_once(const double* a, uint64_t pol)
{
    double v;
    asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
    return v;
}

__device__ __forceinline__ void st_once(float* a, float v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ void st_once(double* a, double v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(a), "d"(v), "l"(pol) : "memory");
}

// fold_load_at + fold_store for the canonical recovery's regular shifts
// (batch-sum FIFO, one K-slice; sums in workspace order, si = w) with the
// evict-first policy on every access: the same values and additions (the
// tile slice added to 0.0f, as sum_in_partials).  Straight-line, its three
// loads issued before the first addition.  Returns the folded sum.
__device__ __forceinline__ double fold_fifo_once(const CumArgs& a, int64_t w, int64_t fslot, uint64_t pol)
{
    double* sp = a.S[a.s] + w;
    float* fp = a.fifo + fslot * a.fstride + w;  // FIFO in workspace order
    const float i0 = ld_once(a.W + a.woff + w, pol);
    const float dout = ld_once(fp, pol);
    const double s0 = ld_once(sp, pol);
    const float din = 0.0f + i0;
    const double sv = s0 + (f32_to_f64(din) - f32_to_f64(dout));
    st_once(sp, sv, pol);
    st_once(fp, din, pol);
    return sv;
}

// hi = x rounded to FP32, lo = the rest rounded to FP32.
__device__ __forceinline__ float2 tw_split(double x)
{
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - f32_to_f64(h)));
}

// C_2 at storage index x of order 2, from the (folded) sums: what the order-2
// element computes, operation for operation, with C_1 = S_1 / T.
// x / T.  For T = 2^k the exponent of x is lowered by k on the integer pipe
// whenever the result is a normal number (bitwise what the multiply by 1/T
// gives); zeros pass through; subnormal results, infinities and NaNs take the
// multiply.  This keeps one FP64 operation per element off the FP64 pipe.
__device__ __forceinline__ double div_T(const CumArgs& a, double x)
{
    const int k = a.tpow2 - 1;  // -1: T is not a power of two
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned ex = (unsigned)(u >> 52) & 0x7ffu;
    if (k >= 0 && ex > (unsigned)k && ex != 0x7ffu)
        return __longlong_as_double((long long)(u - ((unsigned long long)k << 52)));
    if (k >= 0 && (u << 1) == 0) return x;
    return x * a.invT;
}

__device__ __forceinline__ double c2_from_sums(const CumArgs& a2, int64_t x)
{
    const int b = a2.b, bb = b * b;
    const int64_t blk = x / bb;
    const int off = (int)(x - blk * bb);
    const int2 q = *reinterpret_cast<const int2*>(a2.subrank + 2 * blk);  // ranks of (j0), (j1)
    const double cA = a2.S[1][(int64_t)q.x * b + off / b] * a2.invT;
    const double sR = a2.S[1][(int64_t)q.y * b + off % b];
    return fma(-cA, sR, a2.S[2][x]) * a2.invT;
}

// The element of thread `c` in block `blk`: optionally fold the shift's
// workspace into S_S first (FOLD), recover C_S and add multiplicity * C^2 to
// `local`.  Factors C_k with k <= OTF are recomputed from the sums instead of
// read (k = 1: S_1 / T; k = 2: c2_from_sums with the order-2 tables of `a2`),
// which lets orders 1-3 run without a grid barrier between them.  No shared
// memory and no CTA synchronisation: the per-block sub-block ranks come from a
// table whose rows all threads of a block read together (L1 broadcast).
template <int S, bool FOLD, int OTF>
__device__ __forceinline__ void recover_elem(const CumArgs& a, const CumArgs* a2, const Elem<S>& c, int64_t blk,
                                             int64_t fslot, double& local)
{
    constexpr int NS = Subsets<S>::N;
    const int b = a.b;
    const int64_t e = blk * a.bs + c.off;
    if (FOLD && a.accum && !a.sgemm) fold_elem(a, blk, c.off, e, fslot);
    const double sv = a.S[S][a.sgemm ? wslot(a, blk, c.off) : e];
    // the subsets: sub-block ranks (rank(j_A), rank(j_rest)) of the block, one
    // gather per factor, one multiply-add
    const int32_t* sr = a.subrank + (size_t)blk * NS * 2;
    double cv;
    if (S >= kTwoWordMinOrder && a.twoword) {
        float hi = 0.0f, lo = 0.0f;
#pragma unroll(S <= 4 ? NS : 4)
        for (int t = 0; t < NS; ++t) {
            const int2 q = *reinterpret_cast<const int2*>(sr + 2 * t);
            const int la = __popc(2u * t + 1u), lr = S - la;
            int oa, orr;
            subset_offsets<S>(c, b, t, oa, orr);
            const float2 cA = a.C2[la][(unsigned)q.x * (unsigned)ipow_c(b, la) + (unsigned)oa];
            const float2 sR = a.S2[lr][(unsigned)q.y * (unsigned)ipow_c(b, lr) + (unsigned)orr];
            tw_acc_prod(hi, lo, cA, sR);
        }
        cv = div_T(a, sv - (f32_to_f64(hi) + f32_to_f64(lo)));
    } else {
        double acc = sv;
#pragma unroll(S <= 4 ? NS : 4)
        for (int t = 0; t < NS; ++t) {
            const int2 q = *reinterpret_cast<const int2*>(sr + 2 * t);
            const int la = __popc(2u * t + 1u), lr = S - la;
            int oa, orr;
            subset_offsets<S>(c, b, t, oa, orr);
            const unsigned ia = (unsigned)q.x * (unsigned)ipow_c(b, la) + (unsigned)oa;
            double cA;
            if (OTF >= 1 && la == 1) cA = a.S[1][ia] * a.invT;
            else if (OTF >= 2 && la == 2) cA = c2_from_sums(*a2, ia);
            else cA = a.C[la][ia];
            const double sR = a.S[lr][(unsigned)q.y * (unsigned)ipow_c(b, lr) + (unsigned)orr];
            acc = fma(-cA, sR, acc);
        }
        cv = div_T(a, acc);
    }
    a.Cout[e] = cv;
    if (S >= kTwoWordMinOrder && a.split) {  // the two-word copies the next orders read
        a.C2[S][e] = tw_split(cv);
        a.S2[S][e] = tw_split(sv);
    }
    if (S == 1) {
        const double x = cv + (double)a.shift[e];
        local = fma(x, x, local);
    } else {
        local = fma(a.mult[blk] * cv, cv, local);
    }
}

// Deterministic CTA sum (fixed shuffle tree per warp, warps in order) over a
// (virtual) CTA of NT threads; `red` holds NT / 32 doubles of that CTA.
template <bool V = false>
__device__ __forceinline__ double cta_sum(double v, double* red)
{
    const int tid = vtid<V>();
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    vsync<V>();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    vsync<V>();
    double z = 0.0;
    if (tid == 0)
        for (int w = 0; w < NT / 32; ++w) z += red[w];
    return z;  // valid in thread 0
}

// Orders whose per-thread subset offsets are kept in shared memory (packed
// 16 + 16 bits): 2^{S-1} - 1 of them per thread would not fit in registers,
// and forming them per element costs as much integer work as the FP64 work
// they feed.  Above this order they are formed per element.
constexpr int kSmemOffsetsMax = 6;

// Order S >= 5 with the subset offsets of each thread's in-block offset in
// shared memory (computed once, packed 16 + 16 bits) and, per subset of each
// block of a batch of groups, the addresses of its two sub-blocks (the
// operand arrays of the form: two-word copies, or the FP64 arrays), staged
// once per batch: per subset three shared loads, two gathers and the
// multiply-add.  `ptrs` holds [gb][slots][NS] address pairs.
template <int S>
__device__ __forceinline__ void recover_groups_smem(const CumArgs& a, const Elem<S>& c, int64_t g0, int64_t gstride,
                                                    int gb, int slots, int64_t fslot, const int* offs,
                                                    ulonglong2* ptrs, double& local)
{
    constexpr int NS = Subsets<S>::N;
    const int b = a.b;
    const int64_t nblocks = a.E / a.bs;
    const int64_t ngroups = (nblocks + slots - 1) / slots;
    const bool tw = a.twoword != 0;
    __syncthreads();  // the previous batch's readers are done
    for (int i = threadIdx.x; i < gb * slots * NS; i += NT) {
        const int jg = i / (slots * NS), r = i - jg * (slots * NS);
        const int sl = r / NS, t = r - sl * NS;
        const int64_t grp = g0 + jg * gstride, blk = grp * slots + sl;
        if (grp < ngroups && blk < nblocks) {
            const int2 q = *reinterpret_cast<const int2*>(a.subrank + ((size_t)blk * NS + t) * 2);
            const int la = __popc(2u * t + 1u), lr = S - la;
            const char* ca = tw ? (const char*)a.C2[la] : (const char*)a.C[la];
            const char* sr = tw ? (const char*)a.S2[lr] : (const char*)a.S[lr];
            ptrs[i] = make_ulonglong2((unsigned long long)(ca + (size_t)q.x * ipow_c(b, la) * 8),
                                      (unsigned long long)(sr + (size_t)q.y * ipow_c(b, lr) * 8));
        }
    }
    __syncthreads();
    for (int jg = 0; jg < gb; ++jg) {
        const int64_t grp = g0 + jg * gstride;
        if (grp >= ngroups) break;
        const int64_t blk = grp * slots + c.slot;
        if (!c.valid || blk >= nblocks) continue;
        const int64_t e = blk * a.bs + c.off;
        if (a.accum && !a.sgemm) fold_elem(a, blk, c.off, e, fslot);
        const double sv = a.S[S][a.sgemm ? wslot(a, blk, c.off) : e];
        const ulonglong2* pp = ptrs + (jg * slots + c.slot) * NS;
        double cv;
        if (tw) {
            float hi = 0.0f, lo = 0.0f;
#pragma unroll 4
            for (int t = 0; t < NS; ++t) {
                const ulonglong2 pr = pp[t];
                const int packed = offs[t * NT + threadIdx.x];
                const float2 cA = reinterpret_cast<const float2*>(pr.x)[packed >> 16];
                const float2 sR = reinterpret_cast<const float2*>(pr.y)[packed & 0xffff];
                tw_acc_prod(hi, lo, cA, sR);
            }
            cv = div_T(a, sv - (f32_to_f64(hi) + f32_to_f64(lo)));
        } else {
            double acc = sv;
#pragma unroll 4
            for (int t = 0; t < NS; ++t) {
                const ulonglong2 pr = pp[t];
                const int packed = offs[t * NT + threadIdx.x];
                acc = fma(-reinterpret_cast<const double*>(pr.x)[packed >> 16],
                          reinterpret_cast<const double*>(pr.y)[packed & 0xffff], acc);
            }
            cv = div_T(a, acc);
        }
        a.Cout[e] = cv;
        if (a.split) {
            a.C2[S][e] = tw_split(cv);
            a.S2[S][e] = tw_split(sv);
        }
        local = fma(a.mult[blk] * cv, cv, local);
    }
}

template <int S>
__global__ void __launch_bounds__(NT, 4) k_cumulants(const CumArgs* __restrict__ args, int slots, int gb)
{
    const CumArgs& a = args[blockIdx.z];  // one window per blockIdx.z
    if (a.E == 0) return;                 // this window has no order S
    __shared__ double red[NT / 32];
    const Elem<S> c = make_elem<S>(a.b, a.bs, a.bR, slots, blockIdx.y);
    const int64_t fslot = a.accum == 2 ? fifo_slot(a) : 0;
    const int64_t nblocks = a.E / a.bs;
    double local = 0.0;
    bool smem_path = false;
    if constexpr (S > kKeepOffsets && S <= kSmemOffsetsMax) smem_path = ipow_c(a.b, S - 1) <= 0xffff;
    if (smem_path) {
        constexpr int NS = Subsets<S>::N;
        extern __shared__ ulonglong2 dyn[];  // [gb][slots][NS] address pairs, then [NS][NT] offsets
        ulonglong2* ptrs = dyn;
        int* offs = reinterpret_cast<int*>(dyn + (size_t)gb * slots * NS);
        for (int t = 0; t < NS; ++t) {
            int oa, orr;
            subset_offsets<S>(c, a.b, t, oa, orr);
            offs[t * NT + threadIdx.x] = (oa << 16) | orr;  // both < b^{S-1} <= 2^16
        }
        const int64_t ngroups = (nblocks + slots - 1) / slots;
        for (int64_t g0 = blockIdx.x; g0 < ngroups; g0 += (int64_t)gridDim.x * gb)
            recover_groups_smem<S>(a, c, g0, gridDim.x, gb, slots, fslot, offs, ptrs, local);
    } else {
        if (c.valid)
            for (int64_t blk = (int64_t)blockIdx.x * slots + c.slot; blk < nblocks; blk += (int64_t)gridDim.x * slots)
                recover_elem<S, true, 0>(a, nullptr, c, blk, fslot, local);
    }
    const double z = cta_sum(local, red);
    if (threadIdx.x == 0) a.normpart[blockIdx.y * gridDim.x + blockIdx.x] = z;
}

// Grid barrier of a cooperative launch over one 64-bit arrival counter that
// only grows: every barrier adds gridDim.x, so between launches it is a
// multiple of gridDim.x, and barrier k of a launch completes when it reaches
// base + (k + 1) * gridDim.x, base being the counter at the launch's start
// rounded down to a multiple of gridDim.x (no CTA can pass barrier 0 before
// all have read it).  Arrivals release, waits acquire; a wait that takes too
// long records kStatusTimeout and goes on.
__device__ __forceinline__ unsigned long long atom_add_release(unsigned long long* p, unsigned long long v)
{
    unsigned long long old;
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
    return old;
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

struct GridBarrier {
    unsigned long long* ctr;
    unsigned long long base;
    unsigned k;
};

__device__ __forceinline__ GridBarrier grid_barrier_init(unsigned* state, unsigned long long* s_base)
{
    GridBarrier g;
    g.ctr = reinterpret_cast<unsigned long long*>(state);
    if (threadIdx.x == 0) {
        const unsigned long long v = ld_acquire(g.ctr);
        *s_base = v - v % gridDim.x;
    }
    __syncthreads();
    g.base = *s_base;
    g.k = 0;
    return g;
}

__device__ __forceinline__ void grid_barrier(GridBarrier& g, int* status)
{
    __syncthreads();
    ++g.k;
    if (threadIdx.x == 0) {
        const unsigned long long target = g.base + (unsigned long long)g.k * gridDim.x;
        atom_add_release(g.ctr, 1ull);
        const long long t0 = clock64();
        while (ld_acquire(g.ctr) < target) {
            if (clock64() - t0 > kBarrierLimit) {
                atomicOr(status, kStatusTimeout);
                break;
            }
        }
    }
    __syncthreads();
}

// Window of work unit u of an order: last w with ustart[w] <= u.
__device__ __forceinline__ int unit_window(const int64_t* ustart, int nwin, int64_t u)
{
    int lo = 0, hi = nwin - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ustart[mid] <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// One order of the fused recovery (the sums already folded).  CTAs [0, ncta)
// take part, this one as `cta`; each takes a contiguous chunk of the order's
// work units (chunks rotated by `rot`, so that the small orders land on
// different CTAs).  A CTA's units of one window are consecutive, so it sums
// them per thread and reduces once per window ("run"): the run's sum goes to
// the slot of its first unit and the other units of the run hold zero, so
// that every unit slot is written and the window's norm is the sum of its
// unit slots.
template <int S, int OTF, bool V = false>
__device__ __forceinline__ void fused_order(const FusedRecovery& f, const CumArgs* sargs, double* red, int64_t rot,
                                            int cta, int ncta)
{
    const int tid = vtid<V>();
    const int slots = f.slots[S], gy = f.gy[S];
    const int64_t* us = f.ustart + (int64_t)S * (f.nwin + 1);  // read only with several windows
    const int64_t total = f.utot[S];
    const int64_t per = (total + ncta - 1) / ncta;
    const int64_t chunk = ((int64_t)cta + ncta - rot % ncta) % ncta;
    const int64_t u0 = min(total, chunk * per), u1 = min(total, u0 + per);
    if (u0 >= u1) return;  // uniform over the CTA
    double* part = f.upart + f.upoff[S];
    int w = f.nwin == 1 ? 0 : unit_window(us, f.nwin, u0);
    const CumArgs* ap = sargs != nullptr ? &sargs[S] : &f.args[(int64_t)S * f.nwin + w];
    const CumArgs* a2 = OTF < 2 ? nullptr : sargs != nullptr ? &sargs[2] : &f.args[(int64_t)2 * f.nwin + w];
    int64_t nblocks = ap->E / ap->bs;
    Elem<S> c = make_elem<S, V>(ap->b, ap->bs, ap->bR, slots, 0);
    int64_t first = u0;
    double local = 0.0;
    for (int64_t u = u0; u < u1; ++u) {
        if (f.nwin > 1 && u >= us[w + 1]) {  // the next window with units: close the run
            const double z = cta_sum<V>(local, red);
            if (tid == 0) part[first] = z;
            first = u;
            local = 0.0;
            while (u >= us[w + 1]) ++w;
            ap = &f.args[(int64_t)S * f.nwin + w];  // several windows: no shared copy
            if (OTF >= 2) a2 = &f.args[(int64_t)2 * f.nwin + w];
            nblocks = ap->E / ap->bs;
            if (gy == 1) c = make_elem<S, V>(ap->b, ap->bs, ap->bR, slots, 0);
        } else if (u != first && tid == 0) {
            part[u] = 0.0;
        }
        const int64_t ul = f.nwin == 1 ? u : u - us[w];
        int64_t grp = ul;
        if (gy > 1) {
            grp = ul / gy;
            c = make_elem<S, V>(ap->b, ap->bs, ap->bR, slots, (int)(ul - grp * gy));
        }
        const int64_t blk = grp * slots + c.slot;
        if (c.valid && blk < nblocks) recover_elem<S, false, OTF>(*ap, a2, c, blk, 0, local);
    }
    const double z = cta_sum<V>(local, red);
    if (tid == 0) part[first] = z;
}

// What the fold of one (window, order) segment needs, resolved once per
// launch (pointers with the FIFO slot applied), so that a thread's first
// data load does not wait on a chain of argument loads.
struct FoldSeg {
    const float* W;       // workspace of the order (slice 0)
    float* fifo;          // FIFO of the order at this shift's slot, or null
    double* S;
    const int32_t* wblk;
    int64_t wslice;
    int32_t E, bs, bR, ksplit, accum, sgemm;
};

constexpr int kFoldSegSmem = 32;  // segments resolved into shared memory (single windows)

__device__ __forceinline__ FoldSeg fold_seg(const CumArgs& a)
{
    FoldSeg g;
    g.W = a.W + a.woff;
    g.fifo = a.accum == 2 ? a.fifo + fifo_slot(a) * a.fstride : nullptr;
    g.S = a.S[a.s];
    g.wblk = a.wblk;
    g.wslice = a.wslice;
    g.E = (int32_t)a.E;
    g.bs = a.bs;
    g.bR = a.bR;
    g.ksplit = a.ksplit;
    g.accum = a.accum;
    g.sgemm = a.sgemm;
    return g;
}

// One element's fold in two halves: loads, then stores.
struct FoldPend {
    double* sp;
    float* fp;  // FIFO entry or null
    double s;
    float din, dout;
};

__device__ __forceinline__ FoldPend fold_seg_load(const FoldSeg& g, int e)
{
    int64_t w = e;  // sums in workspace order: element = slot
    if (!g.sgemm) {
        const int blk = e / g.bs, off = e - (e / g.bs) * g.bs;
        const int offL = off / g.bR, offRw = off - (off / g.bR) * g.bR;
        const int2 wb = *reinterpret_cast<const int2*>(g.wblk + 2 * blk);
        w = (int64_t)wb.x + (int64_t)offL * wb.y + offRw;
    }
    FoldPend v;
    v.fp = nullptr;
    if (g.fifo == nullptr) {
        sum_partials(g.W + w, g.wslice, g.ksplit, v.din, v.dout);
    } else {
        v.din = sum_in_partials(g.W + w, g.wslice, g.ksplit);
        v.fp = g.fifo + w;
        v.dout = *v.fp;
    }
    v.sp = g.S + (g.sgemm ? w : (int64_t)e);
    v.s = *v.sp;
    return v;
}

__device__ __forceinline__ void fold_commit(const FoldPend& v)
{
    *v.sp = v.s + (f32_to_f64(v.din) - f32_to_f64(v.dout));
    if (v.fp != nullptr) *v.fp = v.din;
}

// Fold the shift's workspace into the sums of the (window, order) segments
// [seg0, seg1): one thread per stored element.  A segment whose sums are in
// workspace order (the top order) is a linear pass over its slots, every
// access coalesced; the others go through the per-block slot table.  With few
// segments their descriptors come from shared memory (`sg`, resolved at the
// start of the launch), otherwise from the argument array.
template <bool V = false>
__device__ __forceinline__ void fused_fold(const FusedRecovery& f, const FoldSeg* sg, int seg0, int seg1, int cta,
                                           int ncta)
{
    const int64_t g0 = f.abeg[seg0], g1 = f.abeg[seg1];
    const int64_t per = ((g1 - g0 + ncta - 1) / ncta + NT - 1) / NT * NT;  // contiguous chunk per CTA
    const int64_t c0 = min(g1, g0 + cta * per), c1 = min(g1, c0 + per);
    int64_t g = c0 + vtid<V>();
    if (g >= c1) return;
    int seg = seg0, hi = seg1 - 1;  // last segment with abeg <= g
    while (seg < hi) {
        const int mid = (seg + hi + 1) >> 1;
        if (f.abeg[mid] <= g) seg = mid;
        else hi = mid - 1;
    }
    FoldSeg gs = sg != nullptr ? sg[seg] : fold_seg(f.args[f.aarg[seg]]);
    for (; g < c1; g += NT) {
        if (g >= f.abeg[seg + 1]) {  // the thread's next segment (monotone)
            while (g >= f.abeg[seg + 1]) ++seg;
            gs = sg != nullptr ? sg[seg] : fold_seg(f.args[f.aarg[seg]]);
        }
        const int e = (int)(g - f.abeg[seg]);  // E_s < 2^31
        if (e < gs.E) fold_commit(fold_seg_load(gs, e));  // segments may end in padding
    }
}

// Fold of segments whose sums are in workspace order (the order-4 range):
// four consecutive slots per thread with 16-byte loads and stores (workspace
// orders, FIFO slots and sums start on 16-byte boundaries; the segments are
// padded to multiples of four in this index space).  The FP32 partials of a
// slot are added in slice order, as in sum_partials / sum_in_partials.
template <bool V = false>
__device__ __forceinline__ void fused_fold_quads(const FusedRecovery& f, const FoldSeg* sg, int seg0, int seg1,
                                                 int cta, int ncta)
{
    const int64_t q0 = f.abeg[seg0] >> 2, q1 = f.abeg[seg1] >> 2;
    const int64_t per = ((q1 - q0 + ncta - 1) / ncta + NT - 1) / NT * NT;  // contiguous chunk per CTA
    const int64_t c0 = min(q1, q0 + cta * per), c1 = min(q1, c0 + per);
    int64_t q = c0 + vtid<V>();
    if (q >= c1) return;
    int lo = seg0, hi = seg1 - 1;  // last segment with abeg <= 4q
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (f.abeg[mid] <= (q << 2)) lo = mid;
        else hi = mid - 1;
    }
    FoldSeg gs = sg != nullptr ? sg[lo] : fold_seg(f.args[f.aarg[lo]]);
    for (; q < c1; q += NT) {
        const int64_t g = q << 2;
        if (g >= f.abeg[lo + 1]) {  // the thread's next segment (monotone)
            while (g >= f.abeg[lo + 1]) ++lo;
            gs = sg != nullptr ? sg[lo] : fold_seg(f.args[f.aarg[lo]]);
        }
        const int e0 = (int)(g - f.abeg[lo]);
        if (e0 + 4 > gs.E) {  // ragged end of the segment
            for (int e = e0; e < gs.E; ++e) fold_commit(fold_seg_load(gs, e));
            continue;
        }
        float4 din = make_float4(0.f, 0.f, 0.f, 0.f), dout = make_float4(0.f, 0.f, 0.f, 0.f);
        const float* w = gs.W + e0;
        if (gs.fifo == nullptr) {
            for (int k = 0; k < gs.ksplit; ++k) {
                const float4 a = *reinterpret_cast<const float4*>(w + (int64_t)(2 * k) * gs.wslice);
                const float4 b = *reinterpret_cast<const float4*>(w + (int64_t)(2 * k + 1) * gs.wslice);
                din.x += a.x; din.y += a.y; din.z += a.z; din.w += a.w;
                dout.x += b.x; dout.y += b.y; dout.z += b.z; dout.w += b.w;
            }
        } else {
            for (int k = 0; k < gs.ksplit; ++k) {
                const float4 a = *reinterpret_cast<const float4*>(w + (int64_t)(2 * k) * gs.wslice);
                din.x += a.x; din.y += a.y; din.z += a.z; din.w += a.w;
            }
            dout = *reinterpret_cast<const float4*>(gs.fifo + e0);
        }
        double2* sp = reinterpret_cast<double2*>(gs.S + e0);
        double2 s01 = sp[0], s23 = sp[1];
        s01.x += f32_to_f64(din.x) - f32_to_f64(dout.x);
        s01.y += f32_to_f64(din.y) - f32_to_f64(dout.y);
        s23.x += f32_to_f64(din.z) - f32_to_f64(dout.z);
        s23.y += f32_to_f64(din.w) - f32_to_f64(dout.w);
        sp[0] = s01;
        sp[1] = s23;
        if (gs.fifo != nullptr) *reinterpret_cast<float4*>(gs.fifo + e0) = din;
    }
}

// Orders 1..DF of every window, as a cooperative grid of (virtual) CTAs: this
// one is `cta` of G, all resident.  The grid barriers synchronise the real CTAs
// (every virtual CTA of a real one reaches them together).  `red` is this
// virtual CTA's reduction buffer; s_seg, s_args and s_base are shared by the
// real CTA.
template <int DF, bool V>
__device__ __forceinline__ void recover_fused_body(const FusedRecovery& f, const int cta, const int G, double* red,
                                                   FoldSeg* s_seg, CumArgs* s_args, unsigned long long* s_base)
{
    const int tid = vtid<V>();
    const bool seg_smem = f.fold && f.nseg <= kFoldSegSmem;
    if (seg_smem && (int)threadIdx.x < f.nseg) s_seg[threadIdx.x] = fold_seg(f.args[f.aarg[threadIdx.x]]);
    if (f.nwin == 1) {  // one window: its arguments of orders 1..DF, copied once
        constexpr int words = (int)(sizeof(CumArgs) / sizeof(int));
        static_assert(sizeof(CumArgs) % sizeof(int) == 0, "CumArgs copied as words");
        for (int i = threadIdx.x; i < DF * words; i += blockDim.x) {
            const int o = i / words + 1, k = i - (i / words) * words;
            reinterpret_cast<int*>(&s_args[o])[k] = reinterpret_cast<const int*>(&f.args[o])[k];
        }
    }
    GridBarrier gb = grid_barrier_init(f.bar, s_base);  // synchronises the CTA
    const FoldSeg* sg = seg_smem ? s_seg : nullptr;
    const CumArgs* sargs = f.nwin == 1 ? s_args : nullptr;
    // 1. the sums of orders 1..min(DF, 3) take the shift's workspace
    if (f.fold) {
        fused_fold<V>(f, sg, 0, f.nseg_lo, cta, G);
        grid_barrier(gb, f.status);
    }
    // 2. orders 1..min(DF, 3): C_1, C_2 recomputed from the sums where a higher
    //    order needs them, so no barrier between these orders.  When the
    //    order-4 sums still take their workspace (nothing reads them before
    //    step 3), the first n13 CTAs take the small orders and the others that
    //    fold, so the latency-bound small orders overlap the memory-bound fold.
    int64_t u13 = 0;
    for (int k = 1; k <= (DF < 3 ? DF : 3); ++k) u13 += f.utot[k];
    const bool split = f.fold && f.nseg > f.nseg_lo && G > 1;
    const int n13 = split ? (int)(u13 < G / 2 ? (u13 > 0 ? u13 : 1) : G / 2) : G;
    if (cta >= n13) {
        fused_fold_quads<V>(f, sg, f.nseg_lo, f.nseg, cta - n13, G - n13);
    } else {
        int64_t rot = 0;
        fused_order<1, 0, V>(f, sargs, red, rot, cta, n13);
        rot += f.utot[1];
        if (DF >= 2) {
            fused_order<(DF >= 2 ? 2 : 1), 1, V>(f, sargs, red, rot, cta, n13);
            rot += f.utot[2];
        }
        if (DF >= 3) fused_order<(DF >= 3 ? 3 : 1), 2, V>(f, sargs, red, rot, cta, n13);
    }
    // 3. order 4 reads the stored C_1..C_3
    if (DF >= 4) {
        grid_barrier(gb, f.status);
        fused_order<(DF >= 4 ? 4 : 1), 0, V>(f, sargs, red, 0, cta, G);
    }
    grid_barrier(gb, f.status);
    // norms: one CTA per (window, order), the partials of the order's units of
    // the window added thread-strided, then the fixed CTA tree
    for (int64_t it = cta; it < (int64_t)f.nwin * DF; it += G) {
        const int w = (int)(it / DF), s = (int)(it - (it / DF) * DF) + 1;
        const NormArgs& na = f.norm[w];
        double z = 0.0;
        if (s <= na.d) {
            const int64_t* us = f.ustart + (int64_t)s * (f.nwin + 1);
            const double* part = f.upart + f.upoff[s];
            const int64_t q1 = f.nwin == 1 ? f.utot[s] : us[w + 1];
            int64_t q = (f.nwin == 1 ? 0 : us[w]) + tid;
            for (; q + 3 * NT < q1; q += 4 * NT) {  // four loads in flight, added in index order
                const double v0 = part[q], v1 = part[q + NT], v2 = part[q + 2 * NT], v3 = part[q + 3 * NT];
                z += v0;
                z += v1;
                z += v2;
                z += v3;
            }
            for (; q < q1; q += NT) z += part[q];
        }
        z = cta_sum<V>(z, red);
        if (tid == 0 && s <= na.d) na.fro2[s - 1] = z;
    }
    // the drift of the mean from the shift (single windows with a drift flag):
    // C_1 and C_2 are complete after the barriers above; the last CTA measures it
    if (f.nwin == 1 && DF >= 2 && cta == G - 1 && f.norm[0].drift_flag != nullptr) {
        const NormArgs& na = f.norm[0];
        double r = 0.0;
        vsync<V>();  // red may still be read by a norm reduction of this CTA
        for (int i = tid; i < na.n; i += NT) {
            const int j = i / na.b, a = i - j * na.b;
            // diagonal block (j, j): rank j * nbar - j (j - 1) / 2, in-block offset a * b + a
            const int64_t rk = (int64_t)j * na.nbar - (int64_t)j * (j - 1) / 2;
            const double v = na.C2[rk * na.b * na.b + a * (na.b + 1)];
            const double m = fabs(na.C1[i]);
            if (v > 0.0) r = fmax(r, m / sqrt(v));
        }
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
        if ((tid & 31) == 0) red[tid >> 5] = r;
        vsync<V>();
        if (tid == 0) {
            for (int w = 1; w < NT / 32; ++w) r = fmax(r, red[w]);
            *na.drift = r;
            if (r > na.drift_limit) *na.drift_flag = 1;
        }
    }
    // every CTA read the ring heads (FIFO slots) before the last barrier
    if (f.advance_heads)
        for (int w = cta * NT + tid; w < f.nwin; w += G * NT) {
            const NormArgs& na = f.norm[w];
            *na.head = (*na.head + f.advance) % na.T;
            if (na.head_stage != nullptr) *na.head_stage = (*na.head_stage + f.advance) % na.T;
        }
}

template <int DF>
__global__ void __launch_bounds__(NT, 4) k_recover_fused(const __grid_constant__ FusedRecovery f)
{
    __shared__ double red[NT / 32];
    __shared__ unsigned long long s_base;
    __shared__ FoldSeg s_seg[kFoldSegSmem];
    __shared__ CumArgs s_args[DF + 1];
    recover_fused_body<DF, false>(f, blockIdx.x, gridDim.x, red, s_seg, s_args, &s_base);
}

// One shift of a batch of windows whose orders are all recovered by the fused
// recovery (d <= kFusedMax), as a single cooperative launch: one CTA of 1024
// threads per SM, its phases separated by the grid barrier.
//   0. FP16 form: the per-variable maxima start from zero;
//   1. staging of X_(+) (and X_(-)), four virtual CTAs of 256 threads per CTA;
//   2. the Khatri-Rao operand build (every thread), after which the staging
//      ring heads advance; the operands are then fenced for the async proxy,
//      because the GEMM reads them with TMA;
//   3. the tcgen05 GEMM on warps 0-5 of every CTA (the other warps wait at the
//      grid barrier);
//   4. the fused recovery of orders 1..DF and the norms, the four quarters of a
//      CTA as virtual CTAs.
// Every wait is bounded as in the kernels these phases come from.
constexpr int kShiftThreads = 1024;
// GEMM stages of the single-launch shift: one fewer than the GEMM kernel's, so
// that the recovery phase keeps more of the SM's memory as L1 for its gathers
constexpr int kShiftStages = 2;
constexpr size_t kShiftStageSmem = 4 * 2 * 32 * 33 * sizeof(float);  // staging tiles of four virtual CTAs

template <bool BF16, int DF>
__global__ void __launch_bounds__(kShiftThreads, 1)
k_batch_shift(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB32,
              const __grid_constant__ CUtensorMap mapB64, const __grid_constant__ CUtensorMap mapB128,
              const __grid_constant__ BatchShiftArgs a, const __grid_constant__ FusedRecovery f)
{
    extern __shared__ unsigned char shift_smem[];  // the GEMM's stages; the staging tiles before them
    __shared__ double red[4][NT / 32];
    __shared__ unsigned long long s_base;
    __shared__ FoldSeg s_seg[kFoldSegSmem];
    __shared__ CumArgs s_args[DF + 1];
    const int vid = (int)(threadIdx.x >> 8);
    const int vcta = (int)blockIdx.x * 4 + vid, nv = (int)gridDim.x * 4;
    const int gtid = (int)(blockIdx.x * blockDim.x + threadIdx.x), gstride = (int)(gridDim.x * blockDim.x);
    GridBarrier gb = grid_barrier_init(f.bar, &s_base);
    // 0. the per-variable maxima of the FP16 form
    if (a.scaled) {
        for (int64_t i = gtid; i < a.nvmax; i += gstride) a.vmax[i] = 0.0f;
        grid_barrier(gb, f.status);
    }
    // 1. staging
    {
        float(*tin)[33] = reinterpret_cast<float(*)[33]>(shift_smem + (size_t)vid * 2 * 32 * 33 * sizeof(float));
        float(*tout)[33] = tin + 32;
        const int per_stream = a.tiles_x * a.tiles_y;
        for (int t = vcta; t < per_stream * a.nstreams; t += nv) {
            const int z = t / per_stream, r = t - z * per_stream, y = r / a.tiles_x, x = r - y * a.tiles_x;
            tcdev::stage_push_tile<true>(a.sdesc, a.xin, nullptr, -1, a.p, a.P, a.Kcap, a.leaving, a.scaled, x, y,
                                         z, tin, tout);
        }
    }
    grid_barrier(gb, f.status);
    // 2. operand build; the staging heads advance (every staging read is done)
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < a.nstreams; i += blockDim.x) {
            int64_t* hp = a.sdesc[i].head;
            *hp = (*hp + a.p) % a.sdesc[i].T;
        }
    tcdev::kr_build_range_lean<BF16>(a.sdesc, a.Kcap, a.opvars, a.oprows, a.nkb, a.ops, a.P, a.opexp, gtid,
                                      gstride);
    ptx::fence_proxy_async_global();
    grid_barrier(gb, f.status);
    // 3. the GEMM
    if (threadIdx.x < tcdev::GEMM_THREADS)
        tcdev::kr_gemm_body<BF16, true, kShiftStages>(&mapA, &mapB32, &mapB64, &mapB128, a.gemm, shift_smem);
    grid_barrier(gb, f.status);
    // 4. the recovery of orders 1..DF and the norms
    recover_fused_body<DF, true>(f, vcta, nv, red[vid], s_seg, s_args, &s_base);
}

// Fold of the orders that take the shift's workspace before their recovery
// runs: sums in workspace order (the top order of windows whose recovery is
// not fused) in one linear coalesced pass, and canonical orders whose sums are
// in the block layout element by element through the slot table.
__global__ void __launch_bounds__(NT) k_fold_linear(const CumArgs* __restrict__ args)
{
    const CumArgs& a = args[blockIdx.y];
    // (a canonical top order takes its batch sums inside k_canon, at its canonical elements)
    if (a.E == 0 || !a.accum || !(a.sgemm || a.canon) || (a.sgemm && a.canon)) return;
    const int64_t fslot = a.accum == 2 ? fifo_slot(a) : 0;
    for (int64_t w = (int64_t)blockIdx.x * NT + threadIdx.x; w < a.E; w += (int64_t)gridDim.x * NT) {
        if (a.sgemm) {
            fold_store(fold_load_at(a, w, w, fslot));
        } else {
            const int64_t blk = w / a.bs;
            fold_elem(a, blk, (int)(w - blk * a.bs), w, fslot);
        }
    }
}

// Canonical recovery, pass 1.  A unit is (pattern, slice, up to kCanonGroup
// blocks of that pattern): thread k of the unit owns canonical element
// slice * NT + k of the pattern, i.e. one in-block offset whose digits are
// non-decreasing inside every run of equal block indices; its per-subset
// operand offsets (packed 16 + 16 bits) are formed when the (pattern, slice)
// changes, the blocks' operand addresses are staged per unit, and each owned
// element of each block is recovered (the subset recursion, two-word products
// in the mixed forms) and written at its own, canonical, position.  The top
// order (sums in workspace order) first takes the shift's batch sums there:
// its sums and FIFO are only ever read at canonical elements.  The norm
// partial weights each element by its block's multiplicity and by the number
// of offsets of its block that hold the same entry, so it is the sum over all
// stored elements.  Each CTA takes a contiguous run of units, so the
// (pattern, slice) changes rarely.
template <int S>
__global__ void __launch_bounds__(NT, kCanonCtasPerSm) k_canon(const CumArgs* __restrict__ args)
{
    constexpr int NS = Subsets<S>::N;
    constexpr int GB = kCanonGroup;
    __shared__ double red[NT / 32];
    const CumArgs& a = *args;
    extern __shared__ ulonglong2 dyn[];  // [GB][NS] operand address pairs, then [NS][NT] offsets
    ulonglong2* ptrs = dyn;
    int* offs = reinterpret_cast<int*>(dyn + GB * NS);
    const int b = a.b;
    const bool tw = a.twoword != 0;
    const bool fold = a.accum != 0 && a.sgemm;
    const int64_t fslot = a.accum == 2 ? fifo_slot(a) : 0;
    const uint64_t keep = l2_policy_evict_last(), once = l2_policy_evict_first();
    const int per = (a.nunits + (int)gridDim.x - 1) / (int)gridDim.x;
    const int u0 = min(a.nunits, (int)blockIdx.x * per), u1 = min(a.nunits, u0 + per);
    int cur_q = -1, cur_sl = -1, off = 0, lr = 0;
    double copies = 0.0;
    bool valid = false;
    double local = 0.0;
    for (int u = u0; u < u1; ++u) {
        const int4 U = a.units[u];  // {pattern, slice, first index into pblocks, blocks}
        __syncthreads();            // the previous unit's readers of ptrs / offs are done
        if (U.x != cur_q || U.y != cur_sl) {
            cur_q = U.x;
            cur_sl = U.y;
            const int c = cur_sl * NT + (int)threadIdx.x;
            const int c0 = a.can_start[cur_q], c1 = a.can_start[cur_q + 1];
            valid = c0 + c < c1;
            off = valid ? a.can_off[c0 + c] : 0;
            lr = valid && a.sgemm ? a.can_lr[c0 + c] : 0;
            copies = valid ? (double)a.can_copies[c0 + c] : 0.0;
            int dig[S];
            int rem = off;
#pragma unroll
            for (int k = S - 1; k >= 0; --k) {
                const int q = rem / b;
                dig[k] = rem - q * b;
                rem = q;
            }
            for (int t = 0; t < NS; ++t) {
                const unsigned mask = 2u * t + 1u;
                int oa = 0, orr = 0;
#pragma unroll
                for (int k = 0; k < S; ++k) {
                    if ((mask >> k) & 1u) oa = oa * b + dig[k];
                    else orr = orr * b + dig[k];
                }
                offs[t * NT + threadIdx.x] = (oa << 16) | orr;  // both < b^{S-1} <= 2^16
            }
        }
        for (int i = threadIdx.x; i < U.w * NS; i += NT) {
            const int jg = i / NS, t = i - jg * NS;
            const int64_t blk = a.pblocks[U.z + jg];
            const int2 q = *reinterpret_cast<const int2*>(a.subrank + ((size_t)blk * NS + t) * 2);
            const int la = __popc(2u * t + 1u), lr = S - la;
            const char* ca = tw ? (const char*)a.C2[la] : (const char*)a.C[la];
            const char* sr = tw ? (const char*)a.S2[lr] : (const char*)a.S[lr];
            ptrs[i] = make_ulonglong2((unsigned long long)(ca + (size_t)q.x * ipow_c(b, la) * 8),
                                      (unsigned long long)(sr + (size_t)q.y * ipow_c(b, lr) * 8));
        }
        __syncthreads();
        if (!valid) continue;
        for (int jg = 0; jg < U.w; ++jg) {
            const int64_t blk = a.pblocks[U.z + jg];
            const int64_t e = blk * a.bs + off;
            double sv;
            if (a.sgemm) {
                const int64_t w = wslot_lr(a, blk, lr);
                if (fold && a.accum == 2 && a.ksplit == 1) {
                    sv = fold_fifo_once(a, w, fslot, once);
                } else if (fold) {
                    FoldVal fv = fold_load_at(a, w, w, fslot);
                    fold_store(fv);
                    sv = fv.s + (f32_to_f64(fv.din) - f32_to_f64(fv.dout));
                } else {
                    sv = a.S[S][w];
                }
            } else {
                sv = a.S[S][e];  // folded before (k_fold_linear), every element
            }
            const ulonglong2* pp = ptrs + jg * NS;
            double cv;
            if (tw) {
                float hi = 0.0f, lo = 0.0f;
#pragma unroll 4
                for (int t = 0; t < NS; ++t) {
                    const ulonglong2 pr = pp[t];
                    const int packed = offs[t * NT + threadIdx.x];
                    const float2 cA = ld_keep(reinterpret_cast<const float2*>(pr.x) + (packed >> 16), keep);
                    const float2 sR = ld_keep(reinterpret_cast<const float2*>(pr.y) + (packed & 0xffff), keep);
                    tw_acc_prod(hi, lo, cA, sR);
                }
                cv = div_T(a, sv - (f32_to_f64(hi) + f32_to_f64(lo)));
            } else {
                double acc = sv;
#pragma unroll 4
                for (int t = 0; t < NS; ++t) {
                    const ulonglong2 pr = pp[t];
                    const int packed = offs[t * NT + threadIdx.x];
                    acc = fma(-reinterpret_cast<const double*>(pr.x)[packed >> 16],
                              reinterpret_cast<const double*>(pr.y)[packed & 0xffff], acc);
                }
                cv = div_T(a, acc);
            }
            st_once(a.Cout + e, cv, once);
            if (a.split) {
                a.C2[S][e] = tw_split(cv);
                a.S2[S][e] = tw_split(sv);
            }
            local = fma(a.mult[blk] * copies * cv, cv, local);
        }
    }
    const double z = cta_sum(local, red);
    if (threadIdx.x == 0) a.normpart[blockIdx.x] = z;
}

// Canonical recovery, pass 2: in every recovered block whose pattern has
// repeated block indices, each non-canonical offset takes the value of its
// canonical offset (the same tensor entry), and orders below d copy their
// two-word C_s and S_s there too when an order above without the canonical
// recovery reads them (the sums, kept at canonical elements only, reach the
// other offsets this way).  One block per CTA at a time, threads over the
// pattern's list of non-canonical offsets.
__global__ void __launch_bounds__(NT) k_canon_expand(const CumArgs* __restrict__ args)
{
    const CumArgs& a = *args;
    for (int i = blockIdx.x; i < a.npblocks; i += gridDim.x) {
        const int64_t blk = a.pblocks[i];
        const int q = a.blkpat[blk];
        const int d0 = a.dup_start[q], d1 = a.dup_start[q + 1];
        double* C = a.Cout + blk * a.bs;
        float2* S2 = a.split && a.split_copies ? a.S2[a.s] + blk * a.bs : nullptr;
        // four copies per thread and round, their loads issued before their stores
        constexpr int U = 4;
        for (int i0 = d0 + (int)threadIdx.x; i0 < d1; i0 += U * NT) {
            int2 oc[U];  // {offset, canonical offset}
            double v[U];
            float2 sv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) oc[u] = i0 + u * NT < d1 ? a.dup[i0 + u * NT] : make_int2(-1, 0);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                v[u] = oc[u].x >= 0 ? C[oc[u].y] : 0.0;
                sv[u] = oc[u].x >= 0 && S2 != nullptr ? S2[oc[u].y] : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (oc[u].x < 0) continue;
                C[oc[u].x] = v[u];
                if (S2 != nullptr) {
                    a.C2[a.s][blk * a.bs + oc[u].x] = tw_split(v[u]);
                    S2[oc[u].x] = sv[u];
                }
            }
        }
    }
}

// Two-word copies of C_k and S_k for the orders k <= s_hi recovered below
// kTwoWordMinOrder (the higher orders write theirs as they go); blockIdx.y =
// k - 1, blockIdx.z = window.
__global__ void __launch_bounds__(NT) k_split(const CumArgs* __restrict__ args)
{
    const CumArgs& a = args[(int64_t)(blockIdx.y + 1) * gridDim.z + blockIdx.z];
    if (!a.split) return;
    for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < a.E; e += (int64_t)gridDim.x * NT) {
        a.C2[a.s][e] = tw_split(a.Cout[e]);
        a.S2[a.s][e] = tw_split(a.S[a.s][e]);
    }
}

// out[e] = S_s[slot(e)] * scale: the sums of an order kept in workspace order,
// or at canonical elements only, back in storage order (every element reads its
// canonical element's sum).
__global__ void __launch_bounds__(NT) k_gather_sums(const CumArgs* __restrict__ args, double scale, double* out)
{
    const CumArgs& a = *args;
    for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < a.E; e += (int64_t)gridDim.x * NT) {
        const int64_t blk = e / a.bs;
        const int off = (int)(e - blk * a.bs);
        int64_t w;
        if (!a.canon) {
            w = wslot(a, blk, off);
        } else {
            const int64_t q = (int64_t)a.blkpat[blk] * a.bs + off;
            w = a.sgemm ? wslot_lr(a, blk, a.map_lr[q]) : blk * a.bs + a.map_off[q];
        }
        out[e] = a.S[a.s][w] * scale;
    }
}

// Entry-wise k-norm partials of C_s (Algorithm 5 with a general k): each
// CTA adds multiplicity * |c|^k over a strided share of the stored elements
// (order 1: |C_1 + shift|^k) and reduces it in a fixed order.
__global__ void __launch_bounds__(NT) k_knorm(const CumArgs* __restrict__ args, double k, double* partials)
{
    __shared__ double red[NT / 32];
    const CumArgs& a = *args;
    double local = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < a.E; e += (int64_t)gridDim.x * NT) {
        double c = a.Cout[e];
        if (a.s == 1) c += (double)a.shift[e];
        local += (a.s == 1 ? 1.0 : a.mult[e / a.bs]) * pow(fabs(c), k);
    }
    const double z = cta_sum(local, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = z;
}

__global__ void k_gather_idx(const double* __restrict__ src, const int64_t* __restrict__ idx, int n, double* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = src[idx[i]];
}

// One CTA per window, one warp per order s >= s_from: lanes add strided
// partials, then a fixed shuffle tree.  Also advances the window's ring head.
__global__ void k_norm_final(const NormArgs* __restrict__ args, int64_t advance, int s_from)
{
    const NormArgs& a = args[blockIdx.x];
    const int lane = threadIdx.x & 31, s = threadIdx.x >> 5;
    if (threadIdx.x == 0 && advance != 0) {
        *a.head = (*a.head + advance) % a.T;
        if (a.head_stage != nullptr) *a.head_stage = (*a.head_stage + advance) % a.T;
    }
    if (s >= a.d || s + 1 < s_from) return;
    double z = 0.0;
    const double* part = a.normpart + (int64_t)s * a.parts;
    int q = lane;
    for (; q + 96 < a.parts; q += 128) {  // four loads in flight, added in index order
        const double v0 = part[q], v1 = part[q + 32], v2 = part[q + 64], v3 = part[q + 96];
        z += v0;
        z += v1;
        z += v2;
        z += v3;
    }
    for (; q < a.parts; q += 32) z += part[q];
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    if (lane == 0) a.fro2[s] = z;
}

// The estimators of Eqs. me / mef from the squared norms: ||C_s|| = sqrt of
// the squared norm, nu_s = ||C_s|| / ||C_2||^{s/2} for s >= 3 (NaN below, and
// NaN when ||C_2|| = 0 by 0/0), and L = sum_s w_s ||C_s||^2.  One warp.
__global__ void k_estimators(const double* __restrict__ fro2, EstArgs a)
{
    const int s = threadIdx.x + 1;
    const bool on = s <= a.d;
    const double z = on ? fro2[s - 1] : 0.0;
    const double f = sqrt(z);
    if (on && a.fro != nullptr) a.fro[s - 1] = f;
    if (on && a.nu != nullptr) {
        const double c2 = a.d >= 2 ? sqrt(fro2[1]) : 0.0;
        a.nu[s - 1] = (s < 3 || a.d < 2) ? __longlong_as_double(0x7ff8000000000000LL) : f / pow(c2, 0.5 * s);
    }
    if (a.loss != nullptr) {  // fixed order: lane s-1 contributes w_s z_s, reduced by a fixed tree
        double v = on ? a.w[s] * z : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) *a.loss = v;
    }
}

template <int S>
cudaError_t launch_order(const CumArgs* args, int nwin, const CumLaunch& L, cudaStream_t st)
{
    size_t smem = 0;
    int gb = 1;
    if (S > kKeepOffsets && S <= kSmemOffsetsMax && L.bpow1 <= 0xffff) {  // the kernel takes the same branch
        constexpr int NS = Subsets<S>::N;
        // groups whose operand addresses are staged together: up to 8, within 16 KB
        const size_t per = sizeof(ulonglong2) * (size_t)L.slots * NS;
        gb = (int)std::max<size_t>(1, std::min<size_t>(8, (16 * 1024) / per));
        smem = per * gb + sizeof(int) * (size_t)NS * NT;
        if (smem > 48 * 1024) {  // above 48 KB needs the opt-in
            cudaError_t e = smem_opt_in((const void*)k_cumulants<S>, smem);
            if (e != cudaSuccess) return e;
        }
    }
    k_cumulants<S><<<dim3(L.gx, L.gy, nwin), NT, smem, st>>>(args, L.slots, gb);
    return cudaGetLastError();
}

template <int DF>
cudaError_t launch_fused_df(const FusedRecovery& f, int grid, size_t smem, cudaStream_t st)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_recover_fused<DF>, f);
}

}  // namespace

// Launch shape of order s: `slots` blocks per group when b^s < 256 (one thread
// per element of each), else one block per group spread over gy CTAs of 256
// offsets; gx groups in flight.  Partials: gx * gy per order.
CumLaunch plan_cumulants(int s, int bs, int64_t nblocks, int sm_count)
{
    CumLaunch L{};
    int b = 1;
    while (ipow_c(b, s) < bs) ++b;  // bs = b^s
    L.bpow1 = ipow_c(b, s - 1);
    const int ns = (1 << (s - 1)) - 1;
    if (bs >= NT) {
        L.slots = 1;
        L.gy = (bs + NT - 1) / NT;
    } else {
        int slots = NT / bs;
        const int cap = ns > 0 ? (40 * 1024) / (ns * 2 * (int)sizeof(int)) : NT;
        if (slots > cap) slots = cap;
        L.slots = slots < 1 ? 1 : slots;
        L.gy = 1;
    }
    const int64_t groups = (nblocks + L.slots - 1) / L.slots;
    int64_t gx = (4LL * sm_count + L.gy - 1) / L.gy;
    if (gx > groups) gx = groups;
    L.gx = (int)(gx < 1 ? 1 : gx);
    return L;
}

cudaError_t launch_cumulants(int s, const CumArgs* args_dev, int nwin, const CumLaunch& L, cudaStream_t st)
{
    switch (s) {
    case 1: return launch_order<1>(args_dev, nwin, L, st);
    case 2: return launch_order<2>(args_dev, nwin, L, st);
    case 3: return launch_order<3>(args_dev, nwin, L, st);
    case 4: return launch_order<4>(args_dev, nwin, L, st);
    case 5: return launch_order<5>(args_dev, nwin, L, st);
    case 6: return launch_order<6>(args_dev, nwin, L, st);
    case 7: return launch_order<7>(args_dev, nwin, L, st);
    case 8: return launch_order<8>(args_dev, nwin, L, st);
    default: return cudaErrorInvalidValue;
    }
}

size_t fused_smem_bytes(const FusedRecovery&, int) { return 0; }

int fused_grid(int dfused, size_t smem, int sm_count, int per_sm_max)
{
    int per_sm = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (dfused) {
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_recover_fused<1>, NT, smem); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_recover_fused<2>, NT, smem); break;
    case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_recover_fused<3>, NT, smem); break;
    case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_recover_fused<4>, NT, smem); break;
    default: break;
    }
    if (e != cudaSuccess || per_sm < 1) return 0;
    return std::min(per_sm, per_sm_max) * sm_count;
}

template <bool BF16, int DF>
cudaError_t launch_batch_shift_t(const TcPlan& plan, const BatchShiftArgs& a, const FusedRecovery& f, int grid,
                                 cudaStream_t st)
{
    const size_t smem = std::max(tcdev::gemm_smem(kShiftStages), kShiftStageSmem);
    cudaError_t e = smem_opt_in((const void*)k_batch_shift<BF16, DF>, smem);
    if (e != cudaSuccess) return e;
    // the smallest shared-memory split that holds it: the rest of the SM's memory is L1
    e = cudaFuncSetAttribute((const void*)k_batch_shift<BF16, DF>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)std::min<size_t>(100, ((smem + 16 * 1024) * 100 + 228 * 1024 - 1) / (228 * 1024)));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kShiftThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_shift<BF16, DF>, plan.mapA, plan.mapB[0], plan.mapB[1], plan.mapB[2], a, f);
}

template <bool BF16, int DF>
int batch_shift_blocks_t()
{
    const size_t smem = std::max(tcdev::gemm_smem(kShiftStages), kShiftStageSmem);
    if (smem_opt_in((const void*)k_batch_shift<BF16, DF>, smem) != cudaSuccess) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_shift<BF16, DF>, kShiftThreads, smem) !=
        cudaSuccess)
        return 0;
    return per_sm;
}

int batch_shift_blocks_per_sm(int precision, int dfused)
{
    const bool bf = precision == 1;
    switch (dfused) {
    case 1: return bf ? batch_shift_blocks_t<true, 1>() : batch_shift_blocks_t<false, 1>();
    case 2: return bf ? batch_shift_blocks_t<true, 2>() : batch_shift_blocks_t<false, 2>();
    case 3: return bf ? batch_shift_blocks_t<true, 3>() : batch_shift_blocks_t<false, 3>();
    case 4: return bf ? batch_shift_blocks_t<true, 4>() : batch_shift_blocks_t<false, 4>();
    default: return 0;
    }
}

cudaError_t launch_batch_shift(const TcPlan& plan, const BatchShiftArgs& a, const FusedRecovery& f, int dfused,
                               int grid, cudaStream_t st)
{
    const bool bf = plan.precision == 1;
    switch (dfused) {
    case 1: return bf ? launch_batch_shift_t<true, 1>(plan, a, f, grid, st) : launch_batch_shift_t<false, 1>(plan, a, f, grid, st);
    case 2: return bf ? launch_batch_shift_t<true, 2>(plan, a, f, grid, st) : launch_batch_shift_t<false, 2>(plan, a, f, grid, st);
    case 3: return bf ? launch_batch_shift_t<true, 3>(plan, a, f, grid, st) : launch_batch_shift_t<false, 3>(plan, a, f, grid, st);
    case 4: return bf ? launch_batch_shift_t<true, 4>(plan, a, f, grid, st) : launch_batch_shift_t<false, 4>(plan, a, f, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_recover_fused(const FusedRecovery& f, int dfused, int grid, size_t smem, cudaStream_t st)
{
    switch (dfused) {
    case 1: return launch_fused_df<1>(f, grid, smem, st);
    case 2: return launch_fused_df<2>(f, grid, smem, st);
    case 3: return launch_fused_df<3>(f, grid, smem, st);
    case 4: return launch_fused_df<4>(f, grid, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_split(const CumArgs* args_dev, int nwin, int s_hi, int64_t maxE, int sm_count, cudaStream_t st)
{
    const int64_t need = (maxE + NT - 1) / NT;
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(need, 4LL * sm_count));
    k_split<<<dim3(gx, s_hi, nwin), NT, 0, st>>>(args_dev);
    return cudaGetLastError();
}

cudaError_t launch_knorm(const CumArgs* args_dev, int64_t E, double k, double* partials, int nparts, cudaStream_t st)
{
    k_knorm<<<nparts, NT, 0, st>>>(args_dev, k, partials);
    return cudaGetLastError();
}

cudaError_t launch_gather_idx(const double* src, const int64_t* idx, int n, double* out, cudaStream_t st)
{
    k_gather_idx<<<(n + NT - 1) / NT, NT, 0, st>>>(src, idx, n, out);
    return cudaGetLastError();
}

cudaError_t launch_fold_linear(const CumArgs* args_dev, int nwin, int64_t maxE, int sm_count, cudaStream_t st)
{
    const int64_t need = (maxE + NT - 1) / NT;
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(need, 8LL * sm_count));
    k_fold_linear<<<dim3(gx, nwin), NT, 0, st>>>(args_dev);
    return cudaGetLastError();
}

cudaError_t launch_gather_sums(const CumArgs* args_dev, int64_t E, double scale, double* out, cudaStream_t st)
{
    const int64_t need = (E + NT - 1) / NT;
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(need, 16384));
    k_gather_sums<<<gx, NT, 0, st>>>(args_dev, scale, out);
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_canon_s(const CumArgs* args_dev, int grid, cudaStream_t st)
{
    constexpr int NS = Subsets<S>::N;
    const size_t smem = sizeof(ulonglong2) * kCanonGroup * NS + sizeof(int) * (size_t)NS * NT;
    if (smem > 48 * 1024) {
        const cudaError_t e = smem_opt_in((const void*)k_canon<S>, smem);
        if (e != cudaSuccess) return e;
    }
    k_canon<S><<<grid, NT, smem, st>>>(args_dev);
    return cudaGetLastError();
}

cudaError_t launch_canon(int s, const CumArgs* args_dev, int grid, cudaStream_t st)
{
    static_assert(kCanonSlice == NT, "a unit is one CTA");
    switch (s) {
    case 5: return launch_canon_s<5>(args_dev, grid, st);
    case 6: return launch_canon_s<6>(args_dev, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_canon_expand(const CumArgs* args_dev, int grid, cudaStream_t st)
{
    k_canon_expand<<<grid, NT, 0, st>>>(args_dev);
    return cudaGetLastError();
}

cudaError_t launch_estimators(const double* fro2, const EstArgs& a, cudaStream_t st)
{
    k_estimators<<<1, 32, 0, st>>>(fro2, a);
    return cudaGetLastError();
}

cudaError_t launch_norm_final(const NormArgs* args_dev, int nwin, int64_t advance, int s_from, cudaStream_t st)
{
    k_norm_final<<<nwin, 32 * kMaxOrder, 0, st>>>(args_dev, advance, s_from);
    return cudaGetLastError();
}

}  // namespace cw
