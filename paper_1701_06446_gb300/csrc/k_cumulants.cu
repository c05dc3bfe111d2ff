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
// blocks are stored whole.  The kernel is specialised per order: the subset
// masks are compile-time constants, each thread owns one in-block offset and
// computes its per-subset operand offsets once, and the per-block operand
// bases (rank * b^|A|) are staged in shared memory for a group of blocks.
// The same pass accumulates multiplicity * C^2 (Algorithm 5 with k = 2) into
// one partial per CTA; a second kernel adds the partials of each order in a
// fixed order.
#include "cw_device.cuh"
#include "cw_internal.h"

namespace cw {

namespace {

constexpr int NT = 256;

// Subset t (0 <= t < 2^{S-1} - 1) holds position 0 and the positions of the
// set bits of t shifted by one: mask = 2t + 1 (the host tables use this order).
template <int S>
struct Subsets {
    static constexpr int N = (1 << (S - 1)) - 1;
};

__host__ __device__ constexpr int popc_c(unsigned x) { return x ? (int)(x & 1u) + popc_c(x >> 1) : 0; }

template <int S>
__global__ void __launch_bounds__(NT) k_cumulants(const CumArgs* __restrict__ args, int slots)
{
    constexpr int NS = Subsets<S>::N;
    const CumArgs& a = args[blockIdx.z];  // one window per blockIdx.z
    if (a.E == 0) return;                 // this window has no order S
    extern __shared__ int sbase[];  // [slots][NS][2]: rank(j_A) * b^|A|, rank(j_rest) * b^|rest|
    const int b = a.b, bs = a.bs;
    int bp[kMaxOrder + 1];
    bp[0] = 1;
#pragma unroll
    for (int k = 1; k <= kMaxOrder; ++k) bp[k] = bp[k - 1] * b;

    // this thread's slot and in-block offset
    int slot, off;
    if (slots == 1) {
        slot = 0;
        off = blockIdx.y * NT + threadIdx.x;
    } else {
        slot = threadIdx.x / bs;
        off = threadIdx.x - slot * bs;
    }
    const bool tvalid = slot < slots && off < bs;
    int dig[S];
    {
        int rem = off;
#pragma unroll
        for (int k = S - 1; k >= 0; --k) {
            const int q = rem / b;
            dig[k] = rem - q * b;
            rem = q;
        }
    }
    int offA[NS > 0 ? NS : 1], offR[NS > 0 ? NS : 1];
#pragma unroll
    for (int t = 0; t < NS; ++t) {
        const unsigned mask = 2u * t + 1u;
        int oa = 0, orr = 0;
#pragma unroll
        for (int k = 0; k < S; ++k) {
            if ((mask >> k) & 1u) oa = oa * b + dig[k];
            else orr = orr * b + dig[k];
        }
        offA[t] = oa;
        offR[t] = orr;
    }

    double* __restrict__ Ss = a.S[S];
    double local = 0.0;
    const int64_t nblocks = a.E / bs;
    const int64_t ngroups = (nblocks + slots - 1) / slots;
    for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int64_t blk0 = grp * slots;
        if (NS > 0) {
            __syncthreads();
            constexpr int NSD = NS > 0 ? NS : 1;
            for (int i = threadIdx.x; i < slots * NS; i += NT) {
                const int64_t blk = blk0 + i / NSD;
                const int t = i - (i / NSD) * NSD;
                if (blk < nblocks) {
                    const int32_t* sr = a.subrank + ((size_t)blk * NS + t) * 2;
                    const int la = __popc(2u * t + 1u), lr = S - la;
                    sbase[2 * i] = sr[0] * bp[la];
                    sbase[2 * i + 1] = sr[1] * bp[lr];
                }
            }
            __syncthreads();
        }
        const int64_t blk = blk0 + slot;
        if (!tvalid || blk >= nblocks) continue;
        const int64_t e = blk * bs + off;
        double acc = Ss[e];
        if (a.accum) {
            float din, dout;
            sum_partials(a.W + a.woff + e, a.wslice, a.ksplit, din, dout);
            acc += f32_to_f64(din) - f32_to_f64(dout);
            Ss[e] = acc;
        }
        const int* sb = sbase + 2 * slot * NS;
#pragma unroll
        for (int t = 0; t < NS; ++t) {
            const int la = popc_c(2u * t + 1u), lr = S - la;
            const double cA = a.C[la][sb[2 * t] + offA[t]];
            const double sR = a.S[lr][sb[2 * t + 1] + offR[t]];
            acc = fma(-cA, sR, acc);
        }
        const double c = acc * a.invT;
        a.Cout[e] = c;
        if (S == 1) {
            const double x = c + (double)a.shift[e];
            local = fma(x, x, local);
        } else {
            local = fma(a.mult[blk] * c, c, local);
        }
    }
    // deterministic CTA reduction
    __shared__ double red[NT];
    __syncthreads();
    red[threadIdx.x] = local;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.normpart[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// One CTA per window, one warp per order: lanes add strided partials, then a
// fixed shuffle tree.  Also advances the window's ring head.
__global__ void k_norm_final(const NormArgs* __restrict__ args, int64_t advance)
{
    const NormArgs& a = args[blockIdx.x];
    const int lane = threadIdx.x & 31, s = threadIdx.x >> 5;
    if (threadIdx.x == 0 && advance != 0) *a.head = (*a.head + advance) % a.T;
    if (s >= a.d) return;
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

template <int S>
cudaError_t launch_order(const CumArgs* args, int nwin, const CumLaunch& L, cudaStream_t st)
{
    constexpr int NS = Subsets<S>::N;
    const size_t smem = (size_t)L.slots * (NS > 0 ? NS : 1) * 2 * sizeof(int);
    k_cumulants<S><<<dim3(L.gx, L.gy, nwin), NT, smem, st>>>(args, L.slots);
    return cudaGetLastError();
}

}  // namespace

// Launch shape of order s: `slots` blocks per group when b^s < 256 (one thread
// per element of each), else one block per group spread over gy CTAs of 256
// offsets; gx groups in flight.  Partials: gx * gy per order.
CumLaunch plan_cumulants(int s, int bs, int64_t nblocks, int sm_count)
{
    CumLaunch L{};
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

cudaError_t launch_norm_final(const NormArgs* args_dev, int nwin, int64_t advance, cudaStream_t st)
{
    k_norm_final<<<nwin, 32 * kMaxOrder, 0, st>>>(args_dev, advance);
    return cudaGetLastError();
}

}  // namespace cw
