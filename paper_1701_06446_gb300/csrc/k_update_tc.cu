// Moment-sum update on the 5th-generation tensor cores (Eqs. 6-7, Algorithm 2).
//
// Per item: 128 columns (right factor, MMA M) x up to 256 rows (left factor,
// MMA N) of one order's GEMM.  For every K-chunk of 32 samples:
//   1. one thread TMA-loads the chunk of the transposed, shifted sample buffer
//      (npad variables x 36 samples, FP32) into shared memory (2 stages);
//   2. all 256 threads form the Khatri-Rao products of the item's columns and
//      rows for the chunk's samples on the CUDA cores, split each FP32 product
//      into 16-bit hi + lo parts and store them in the canonical K-major
//      no-swizzle layout (8-row x 16-byte core matrices);
//   3. one thread issues hi*hi + hi*lo + lo*hi tcgen05 MMAs per 16-sample step
//      into an FP32 accumulator in tensor memory: samples entering the window
//      into D_in (columns 0..255), samples leaving it into D_out (256..511).
// After the last chunk of a pass, every thread reads its TMEM lane and adds
// (double)D_in - (double)D_out to the FP64 running sums.  Because a batch is
// reduced by the same instruction sequence when it enters and when it leaves,
// its FP32 sum is bitwise the same both times.
//
// Every wait on an mbarrier is bounded; on a timeout the CTA records
// kStatusTimeout, drains its own copies and MMAs (bounded), frees its tensor
// memory and returns.
#include <climits>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "cw_tc.h"
#include "tc_ptx.cuh"

namespace cw {

namespace {

using namespace ptx;

constexpr int KC = kTcKC, XS = kTcXS, TM = kTcM, NMAX = kTcNmax;
constexpr int NT = 256;
constexpr long long kWaitLimit = 1LL << 32;  // clock cycles (~2 s)

constexpr int A_BYTES = TM * KC * 2;    // one 16-bit part of the A tile
constexpr int B_BYTES = NMAX * KC * 2;  // one 16-bit part of the B tile (max rows)
constexpr int OFF_A = 0;                // A[stage][hi/lo]
constexpr int OFF_B = OFF_A + 4 * A_BYTES;
constexpr int OFF_X = OFF_B + 4 * B_BYTES;

// Byte stride of the two staged-sample buffers (TMA destinations, 1024-aligned).
__host__ __device__ constexpr uint32_t tc_xstride(int npad)
{
    return ((uint32_t)npad * XS * 4 + 1023u) & ~1023u;
}

__host__ __device__ constexpr size_t tc_smem_bytes(int npad)
{
    return (size_t)OFF_X + 2ull * tc_xstride(npad) + 1024;  // + alignment slack
}

template <bool BF16>
__device__ __forceinline__ void split_store(const float (&p)[8], unsigned char* hi, unsigned char* lo)
{
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if constexpr (BF16) {
            const __nv_bfloat162 hv = __floats2bfloat162_rn(p[2 * q], p[2 * q + 1]);
            const float2 hf = __bfloat1622float2(hv);
            const __nv_bfloat162 lv = __floats2bfloat162_rn(p[2 * q] - hf.x, p[2 * q + 1] - hf.y);
            h[q] = *reinterpret_cast<const uint32_t*>(&hv);
            l[q] = *reinterpret_cast<const uint32_t*>(&lv);
        } else {
            const __half2 hv = __floats2half2_rn(p[2 * q], p[2 * q + 1]);
            const float2 hf = __half22float2(hv);
            const __half2 lv = __floats2half2_rn(p[2 * q] - hf.x, p[2 * q + 1] - hf.y);
            h[q] = *reinterpret_cast<const uint32_t*>(&hv);
            l[q] = *reinterpret_cast<const uint32_t*>(&lv);
        }
    }
    *reinterpret_cast<uint4*>(hi) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Products over `nf` variables (packed one byte each) of 8 consecutive samples.
__device__ __forceinline__ void kr8(const float* __restrict__ xs, uint32_t vars, int nf, int grp,
                                    float (&p)[8])
{
#pragma unroll
    for (int e = 0; e < 8; ++e) p[e] = 1.0f;
    for (int f = 0; f < nf; ++f) {
        const float* xr = xs + ((vars >> (8 * f)) & 0xffu) * XS + 8 * grp;
        const float4 a = *reinterpret_cast<const float4*>(xr);
        const float4 b = *reinterpret_cast<const float4*>(xr + 4);
        p[0] *= a.x; p[1] *= a.y; p[2] *= a.z; p[3] *= a.w;
        p[4] *= b.x; p[5] *= b.y; p[6] *= b.z; p[7] *= b.w;
    }
}

template <bool BF16>
__global__ void __launch_bounds__(NT, 1)
k_update_tc(const __grid_constant__ CUtensorMap xmap, const TcArgs args)
{
    extern __shared__ unsigned char dsm_raw[];
    unsigned char* dsm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t bar_x[2], bar_mma[2], bar_acc;
    __shared__ uint32_t s_tbase;
    __shared__ uint32_t s_rowvar[NMAX], s_colvar[TM];
    __shared__ int32_t s_rowcolmin[NMAX];
    __shared__ int64_t s_rowoff[NMAX], s_coloff[TM];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int npad = args.npad;
    const uint32_t xbytes = (uint32_t)npad * XS * 4;   // bytes of one TMA box
    const uint32_t xstride = tc_xstride(npad);

    if (tid == 0) {
        mbar_init(&bar_x[0], 1);
        mbar_init(&bar_x[1], 1);
        mbar_init(&bar_mma[0], 1);
        mbar_init(&bar_mma[1], 1);
        mbar_init(&bar_acc, 1);
        fence_mbar_init();
        prefetch_tensormap(&xmap);
    }
    if (warp == 0) {
        tmem_alloc(&s_tbase, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = s_tbase;

    uint32_t g = 0;                  // K-chunks consumed by this CTA
    uint32_t npairs_done = 0;        // completed passes (bar_acc phases)
    uint32_t tma_issued[2] = {0, 0}; // thread 0 only
    uint32_t tma_waited[2] = {0, 0}; // thread 0 only
    bool bad = false;

    for (int it = blockIdx.x; it < args.nitems && !bad; it += gridDim.x) {
        const TcItem item = args.items[it];
        const TcOrder& od = args.ord[item.s];
        const int NB = (item.nrows + 31) & ~31;
        for (int r = tid; r < NMAX; r += NT) {
            const bool v = r < item.nrows;
            s_rowvar[r] = v ? od.rowvar[item.row0 + r] : 0u;
            s_rowoff[r] = v ? od.rowoff[item.row0 + r] : 0;
            s_rowcolmin[r] = v ? od.rowcolmin[item.row0 + r] : INT_MAX;
        }
        if (tid < TM) {
            const bool v = tid < item.ncols;
            s_colvar[tid] = v ? od.colvar[item.col0 + tid] : 0u;
            s_coloff[tid] = v ? od.coloff[item.col0 + tid] : 0;
        }
        __syncthreads();
        const uint32_t idesc = idesc_f16(TM, NB, BF16);
        const int h = od.h, sh = od.sh;

        for (int j = 0; j < args.npairs && !bad; ++j) {
            const int nplus = args.seglen / KC;
            const int nminus = (j == 0) ? args.minus_len / KC : 0;
            const int nch = nplus + nminus;
            const int plus0 = j * args.seg_stride;
            if (tid == 0) {
                for (int q = 0; q < 2 && q < nch; ++q) {
                    const uint32_t st = (g + q) & 1;
                    const int k = q < nplus ? plus0 + q * KC : args.minus_off + (q - nplus) * KC;
                    mbar_arrive_expect_tx(&bar_x[st], xbytes);
                    tma_load_2d(dsm + OFF_X + st * xstride, &xmap, &bar_x[st], k, 0);
                    tma_issued[st]++;
                }
            }
            for (int q = 0; q < nch; ++q) {
                const uint32_t gc = g + q, st = gc & 1, use = gc >> 1;
                bool ok = mbar_wait(&bar_x[st], use & 1, kWaitLimit);
                if (tid == 0 && ok) tma_waited[st]++;
                if (ok && gc >= 2) ok = mbar_wait(&bar_mma[st], (use - 1) & 1, kWaitLimit);
                unsigned char* Ahi = dsm + OFF_A + (st * 2 + 0) * A_BYTES;
                unsigned char* Alo = dsm + OFF_A + (st * 2 + 1) * A_BYTES;
                unsigned char* Bhi = dsm + OFF_B + (st * 2 + 0) * B_BYTES;
                unsigned char* Blo = dsm + OFF_B + (st * 2 + 1) * B_BYTES;
                if (ok) {
                    const float* xs = reinterpret_cast<const float*>(dsm + OFF_X + st * xstride);
                    // A: 128 columns x 4 groups of 8 samples
                    for (int task = tid; task < TM * (KC / 8); task += NT) {
                        const int r = task % TM, grp = task / TM;
                        float p[8];
                        if (r < item.ncols) {
                            kr8(xs, s_colvar[r], sh, grp, p);
                        } else {
#pragma unroll
                            for (int e = 0; e < 8; ++e) p[e] = 0.0f;
                        }
                        const int off = grp * (TM * 16) + (r >> 3) * 128 + (r & 7) * 16;
                        split_store<BF16>(p, Ahi + off, Alo + off);
                    }
                    // B: NB rows x 4 groups of 8 samples
                    for (int task = tid; task < NB * (KC / 8); task += NT) {
                        const int r = task % NB, grp = task / NB;
                        float p[8];
                        if (r < item.nrows) {
                            kr8(xs, s_rowvar[r], h, grp, p);
                        } else {
#pragma unroll
                            for (int e = 0; e < 8; ++e) p[e] = 0.0f;
                        }
                        const int off = grp * (NB * 16) + (r >> 3) * 128 + (r & 7) * 16;
                        split_store<BF16>(p, Bhi + off, Blo + off);
                    }
                }
                fence_proxy_async_smem();
                if (__syncthreads_or(!ok)) {
                    bad = true;
                    break;
                }
                if (tid == 0) {
                    tc_fence_after();
                    const bool plus = q < nplus;
                    const bool first = (q == 0) || (q == nplus);
                    const uint32_t d = tbase + (plus ? 0u : 256u);
#pragma unroll
                    for (int ks = 0; ks < KC / 16; ++ks) {
                        const uint64_t ah = smem_desc_kmajor(smem_u32(Ahi) + ks * 2 * (TM * 16), TM * 16, 128);
                        const uint64_t al = smem_desc_kmajor(smem_u32(Alo) + ks * 2 * (TM * 16), TM * 16, 128);
                        const uint64_t bh = smem_desc_kmajor(smem_u32(Bhi) + ks * 2 * (NB * 16), NB * 16, 128);
                        const uint64_t bl = smem_desc_kmajor(smem_u32(Blo) + ks * 2 * (NB * 16), NB * 16, 128);
                        tc_mma_f16(d, ah, bh, idesc, (first && ks == 0) ? 0u : 1u);
                        tc_mma_f16(d, ah, bl, idesc, 1u);
                        tc_mma_f16(d, al, bh, idesc, 1u);
                    }
                    tc_commit(&bar_mma[st]);
                    if (q == nch - 1) tc_commit(&bar_acc);
                    if (q + 2 < nch) {
                        const int k = (q + 2) < nplus ? plus0 + (q + 2) * KC
                                                      : args.minus_off + (q + 2 - nplus) * KC;
                        mbar_arrive_expect_tx(&bar_x[st], xbytes);
                        tma_load_2d(dsm + OFF_X + st * xstride, &xmap, &bar_x[st], k, 0);
                        tma_issued[st]++;
                    }
                }
            }
            if (bad) break;
            g += nch;

            // epilogue: S += D_in - D_out
            const bool ok = mbar_wait(&bar_acc, npairs_done & 1, kWaitLimit);
            npairs_done++;
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            tc_fence_after();
            {
                const int quarter = warp & 3, half = warp >> 2;
                const int i = 32 * quarter + lane;
                const bool ivalid = i < item.ncols;
                const int cglob = item.col0 + i;
                const int64_t co = s_coloff[i];
                const bool has_minus = nminus > 0;
                double* __restrict__ S = od.S;
                const int jb0 = half * (NB / 2), jb1 = jb0 + NB / 2;
                for (int jb = jb0; jb < jb1; jb += 16) {
                    uint32_t d0[16], d1[16];
                    const uint32_t ta = tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)jb;
                    tmem_ld16(ta, d0);
                    if (has_minus) tmem_ld16(ta + 256u, d1);
                    tmem_ld_wait();
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        const int r = jb + t;
                        if (ivalid && r < item.nrows && cglob >= s_rowcolmin[r]) {
                            double v = (double)__uint_as_float(d0[t]);
                            if (has_minus) v -= (double)__uint_as_float(d1[t]);
                            S[s_rowoff[r] + co] += v;
                        }
                    }
                }
            }
            tc_fence_before();
            __syncthreads();
        }
    }

    if (bad) {
        if (tid == 0) {
            atomicOr(args.status, kStatusTimeout);
            // drain this CTA's own copies and MMAs before the memory goes away
            for (int st = 0; st < 2; ++st)
                while (tma_waited[st] < tma_issued[st]) {
                    if (!mbar_wait(&bar_x[st], tma_waited[st] & 1, kWaitLimit)) break;
                    tma_waited[st]++;
                }
            tc_commit(&bar_acc);
            mbar_wait(&bar_acc, npairs_done & 1, kWaitLimit);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tbase, 512);
}

// ---------------------------------------------------------------------------
// staging: shifted samples, transposed to [variable][sample]
// ---------------------------------------------------------------------------
// Rows [0, P) of the K axis hold X_(+), rows [P, 2P) hold X_(-), zero beyond p.
// The thread of (r, v) also moves X_(+) into the ring slot it reads X_(-) from.
__global__ void __launch_bounds__(256)
k_tc_stage_push(const float* __restrict__ x_in, int64_t ld_in, const float* __restrict__ x_out,
                int64_t ld_out, float* __restrict__ ring, int64_t T, const int64_t* __restrict__ head_p,
                int p, int P, int n, int npad, const float* __restrict__ shift, float* __restrict__ XT,
                int64_t Kcap, int* __restrict__ status)
{
    const int64_t total = (int64_t)npad * P;
    const int64_t head = *head_p;
    bool badv = false;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(e / P);
        const int r = (int)(e - (int64_t)v * P);
        float xin = 0.0f, xo = 0.0f;
        if (r < p) {
            int64_t slot = head + r;
            if (slot >= T) slot -= T;
            const float raw_in = v < n ? x_in[(int64_t)r * ld_in + v] : 0.0f;
            float raw_out;
            if (x_out != nullptr) raw_out = v < n ? x_out[(int64_t)r * ld_out + v] : 0.0f;
            else raw_out = ring[slot * npad + v];
            ring[slot * npad + v] = raw_in;
            badv |= !isfinite(raw_in);
            if (v < n) {
                xin = raw_in - shift[v];
                xo = raw_out - shift[v];
            }
        }
        XT[(int64_t)v * Kcap + r] = xin;
        XT[(int64_t)v * Kcap + P + r] = xo;
    }
    if (badv) atomicOr(status, kStatusNonFinite);
}

// Window rows in batches of p (window order, oldest first): batch q at K
// offset q*P, zero-padded to P.
__global__ void __launch_bounds__(256)
k_tc_stage_window(const float* __restrict__ ring, int64_t T, const int64_t* __restrict__ head_p,
                  int p, int P, int nbatch, int n, int npad, const float* __restrict__ shift,
                  float* __restrict__ XT, int64_t Kcap)
{
    const int64_t total = (int64_t)npad * nbatch * P;
    const int64_t head = *head_p;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(e / ((int64_t)nbatch * P));
        const int64_t k = e - (int64_t)v * nbatch * P;
        const int64_t q = k / P;
        const int r = (int)(k - q * P);
        const int64_t w = q * p + r;
        float x = 0.0f;
        if (r < p && w < T && v < n) {
            int64_t slot = head + w;
            if (slot >= T) slot -= T;
            x = ring[slot * npad + v] - shift[v];
        }
        XT[(int64_t)v * Kcap + k] = x;
    }
}

inline int grid_for(int64_t work)
{
    int64_t g = (work + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 8192));
}

cudaError_t launch_tc_kernel(const TcPlan& plan, int npairs, int seglen, int seg_stride,
                             int minus_off, int minus_len, cudaStream_t st)
{
    TcArgs a{};
    for (int s = 0; s <= kMaxOrder; ++s) a.ord[s] = plan.ord[s];
    a.items = plan.items;
    a.nitems = plan.nitems;
    a.npad = plan.npad;
    a.npairs = npairs;
    a.seglen = seglen;
    a.seg_stride = seg_stride;
    a.minus_off = minus_off;
    a.minus_len = minus_len;
    a.status = plan.status;
    const size_t smem = tc_smem_bytes(plan.npad);
    if (plan.precision == 1)
        k_update_tc<true><<<plan.grid, NT, smem, st>>>(plan.xmap, a);
    else
        k_update_tc<false><<<plan.grid, NT, smem, st>>>(plan.xmap, a);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// planning (host)
// --------------------------------------------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (fn == nullptr) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Per-K-chunk cost model of one item (cycles): the larger of the tensor time
// (3 MMAs of 128 x N x 32) and the operand build time, plus a fixed overhead.
double item_cost(int nrows)
{
    const int NB = (nrows + 31) & ~31;
    const double mma = 3.0 * TM * NB * KC / 4096.0;
    const double build = (TM + NB) * KC / 20.0;
    return std::max(mma, build) + 120.0;
}

}  // namespace

int tc_plan_create(TcPlan& plan, const std::vector<UpdateTables>& tables, const UpdateArgs& upd,
                   int d, int n, int b, int npad, int64_t T, int p, int sm_count, int precision,
                   int* status, const DevAlloc& alloc)
{
    (void)n;
    (void)b;
    plan.precision = precision;
    plan.npad = npad;
    plan.T = T;
    plan.p = p;
    plan.P = (p + KC - 1) / KC * KC;
    plan.nbatch = (int)((T + p - 1) / p);
    const int64_t Pmax = (T + KC - 1) / KC * KC;
    plan.Kcap = std::max<int64_t>((int64_t)plan.nbatch * plan.P, 2 * Pmax);
    plan.Kcap = (plan.Kcap + 3) / 4 * 4;
    plan.status = status;

    cudaError_t e = alloc(sizeof(float) * (size_t)npad * plan.Kcap, (void**)&plan.XT);
    if (e != cudaSuccess) return (int)e;
    e = cudaMemset(plan.XT, 0, sizeof(float) * (size_t)npad * plan.Kcap);
    if (e != cudaSuccess) return (int)e;

    EncodeTiledFn enc = get_encode_fn();
    if (enc == nullptr) return (int)cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)plan.Kcap, (cuuint64_t)npad};
    const cuuint64_t strides[1] = {(cuuint64_t)plan.Kcap * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)XS, (cuuint32_t)npad};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&plan.xmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, plan.XT, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return (int)cudaErrorInvalidValue;

    // per-order device tables (row/column tables are shared with the FP64 form)
    std::vector<TcItem> items;
    double useful = 0, issued = 0;
    for (int s = 1; s <= d; ++s) {
        const UpdateTables& t = tables[s];
        const OrderTables& ot = upd.ord[s];
        TcOrder& o = plan.ord[s];
        o.rowvar = ot.rowvar;
        o.rowoff = ot.rowoff;
        o.colvar = ot.colvar;
        o.coloff = ot.coloff;
        o.S = ot.S;
        o.h = t.h;
        o.sh = t.sh;
        const int nbar = (int)t.colstart.size();
        const int ncols = (int)t.colvar.size();
        std::vector<int32_t> colmin(t.rowvar.size());
        for (int m = 0; m < nbar; ++m)
            for (int r = t.rowstart[m]; r < t.rowstart[m + 1]; ++r) colmin[r] = t.colstart[m];
        int32_t* dcm = nullptr;
        e = alloc(sizeof(int32_t) * std::max<size_t>(colmin.size(), 1), (void**)&dcm);
        if (e != cudaSuccess) return (int)e;
        e = cudaMemcpy(dcm, colmin.data(), sizeof(int32_t) * colmin.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return (int)e;
        o.rowcolmin = dcm;

        // row ranges: groups larger than NMAX rows are split; consecutive small
        // groups are merged while that lowers the modelled cost
        struct Range { int r0, r1, c0; };
        std::vector<Range> ranges;
        for (int m = 0; m < nbar; ++m) {
            const int r0 = t.rowstart[m], r1 = t.rowstart[m + 1];
            if (r1 <= r0 || t.colstart[m] >= ncols) continue;
            for (int r = r0; r < r1; r += NMAX) ranges.push_back({r, std::min(r1, r + NMAX), t.colstart[m]});
        }
        auto cost = [&](const Range& R) {
            const int span = ncols - R.c0;
            return ((span + TM - 1) / TM) * item_cost(R.r1 - R.r0);
        };
        std::vector<Range> merged;
        for (const Range& R : ranges) {
            if (!merged.empty()) {
                Range& L = merged.back();
                if (L.r1 == R.r0 && R.r1 - L.r0 <= NMAX) {
                    Range M{L.r0, R.r1, L.c0};
                    if (cost(M) <= cost(L) + cost(R)) {
                        L = M;
                        continue;
                    }
                }
            }
            merged.push_back(R);
        }
        for (const Range& R : merged) {
            for (int c = R.c0; c < ncols; c += TM) {
                TcItem it{};
                it.s = s;
                it.row0 = R.r0;
                it.nrows = R.r1 - R.r0;
                it.col0 = c;
                it.ncols = std::min(TM, ncols - c);
                items.push_back(it);
                issued += 3.0 * TM * ((it.nrows + 31) & ~31);
            }
            for (int r = R.r0; r < R.r1; ++r) useful += 3.0 * std::max(0, ncols - colmin[r]);
        }
    }
    // larger items first, then round-robin over the persistent CTAs
    std::stable_sort(items.begin(), items.end(),
                     [](const TcItem& x, const TcItem& y) { return x.nrows > y.nrows; });
    plan.useful_macs_per_sample = useful;
    plan.issued_macs_per_sample = issued;
    plan.nitems = (int)items.size();
    plan.grid = std::max(1, std::min(plan.nitems, sm_count));
    e = alloc(sizeof(TcItem) * std::max<size_t>(items.size(), 1), (void**)&plan.items);
    if (e != cudaSuccess) return (int)e;
    e = cudaMemcpy(plan.items, items.data(), sizeof(TcItem) * items.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return (int)e;

    const size_t smem = tc_smem_bytes(npad);
    e = cudaFuncSetAttribute(k_update_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(k_update_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    plan.ready = 1;
    return 0;
}

int tc_launch_count(const TcPlan&) { return 2; }

cudaError_t tc_update_push(const TcPlan& plan, const float* x_in, int64_t ld_in, const float* x_out,
                           int64_t ld_out, float* ring, const int64_t* head, int p, int n,
                           const float* shift, cudaStream_t st)
{
    const int P = (p + KC - 1) / KC * KC;
    if (2 * (int64_t)P > plan.Kcap) return cudaErrorInvalidValue;
    k_tc_stage_push<<<grid_for((int64_t)plan.npad * P), 256, 0, st>>>(
        x_in, ld_in, x_out, ld_out, ring, plan.T, head, p, P, n, plan.npad, shift, plan.XT,
        plan.Kcap, plan.status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_tc_kernel(plan, 1, P, 0, P, P, st);
}

cudaError_t tc_update_window(const TcPlan& plan, const float* ring, const int64_t* head, int n,
                             const float* shift, cudaStream_t st)
{
    k_tc_stage_window<<<grid_for((int64_t)plan.npad * plan.nbatch * plan.P), 256, 0, st>>>(
        ring, plan.T, head, plan.p, plan.P, plan.nbatch, n, plan.npad, shift, plan.XT, plan.Kcap);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_tc_kernel(plan, plan.nbatch, plan.P, plan.P, 0, 0, st);
}

}  // namespace cw
