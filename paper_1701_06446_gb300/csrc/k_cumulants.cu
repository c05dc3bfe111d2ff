// Moment-to-cumulant recovery (Algorithms 3-4) and cumulant norms (Eq. me,
// Algorithm 5), FP64.
//
// Algorithm 4 sums, for every element, products of lower-order cumulants over
// all set partitions of its s indices.  Grouping those partitions by the part
// that holds the first index gives the equivalent subset recursion
//     C_s[i] = M_s[i] - sum_{A contains index 1, A != all} C_|A|[i_A] M_{s-|A|}[i_rest]
// (2^{s-1} - 1 terms instead of B(s) - 1), which is what runs here.  With
// M = S/T it is evaluated as C_s = (S_s[i] - sum_A C_|A|[i_A] S_rest[i_rest]) / T,
// one FP64 multiply-add per subset and one scaling per element (FP64 is the
// scarce pipe on this GPU).
//
// For a sorted block j every sub-tuple j_A is sorted, so the operands are
// stored blocks whose ranks come from a per-block table; the in-block offsets
// follow from the element's own in-block digits because diagonal blocks are
// stored whole.  One warp handles one block at a time, its lanes striding
// over the block's b^s elements.  The same pass accumulates
// multiplicity * C^2 (Algorithm 5 with k = 2) into one partial per CTA; a
// second kernel adds the partials of each order in a fixed order.
#include "cw_device.cuh"
#include "cw_internal.h"

namespace cw {

namespace {

constexpr int NT = 256;

constexpr int WARPS = NT / 32;

__global__ void __launch_bounds__(NT) k_cumulants(const CumArgs a)
{
    const int s = a.s, b = a.b, bs = a.bs, nsub = a.nsub;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // per-subset digit weights: offA = sum_k dig[k] * wA[u][k], offR likewise
    __shared__ int wA[128][kMaxOrder], wR[128][kMaxOrder];
    __shared__ int la_s[128], lr_s[128];
    __shared__ int bpow[kMaxOrder + 1];
    if (threadIdx.x <= kMaxOrder) {
        int p = 1;
        for (int k = 0; k < (int)threadIdx.x; ++k) p *= b;
        bpow[threadIdx.x] = p;
    }
    for (int u = threadIdx.x; u < nsub; u += NT) {
        const unsigned mask = a.mask[u];
        int na = 0, nr = 0;
        for (int k = 0; k < s; ++k) na += (mask >> k) & 1u;
        nr = s - na;
        int ka = 0, kr = 0, pa = 1, pr = 1;
        for (int k = 0; k < na; ++k) pa *= b;
        for (int k = 0; k < nr; ++k) pr *= b;
        for (int k = 0; k < s; ++k) {
            if ((mask >> k) & 1u) {
                pa /= b;
                wA[u][k] = pa;
                wR[u][k] = 0;
                ++ka;
            } else {
                pr /= b;
                wR[u][k] = pr;
                wA[u][k] = 0;
                ++kr;
            }
        }
        la_s[u] = na;
        lr_s[u] = nr;
    }
    __syncthreads();

    double* __restrict__ Ss = a.S[s];
    double local = 0.0;
    const int64_t nblocks = a.E / bs;
    for (int64_t blk = (int64_t)blockIdx.x * WARPS + warp; blk < nblocks;
         blk += (int64_t)gridDim.x * WARPS) {
        const int32_t* __restrict__ sr = a.subrank + (size_t)blk * nsub * 2;
        const double mult = s > 1 ? a.mult[blk] : 1.0;
        for (int off = lane; off < bs; off += 32) {
            const int64_t e = blk * bs + off;
            double acc = Ss[e];
            if (a.accum) {
                float din = 0.0f, dout = 0.0f;
                const float* w = a.W + a.woff + e;
                for (int k = 0; k < a.ksplit; ++k) {
                    din += w[(int64_t)(2 * k) * a.wslice];
                    dout += w[(int64_t)(2 * k + 1) * a.wslice];
                }
                acc += f32_to_f64(din) - f32_to_f64(dout);
                Ss[e] = acc;
            }
            if (s == 1) {
                const double c = acc * a.invT;
                a.Cout[e] = c;
                const double x = c + (double)a.shift[e];
                local = fma(x, x, local);
                continue;
            }
            int dig[kMaxOrder];
            int rem = off;
            for (int k = s - 1; k >= 0; --k) {
                const int q = rem / b;
                dig[k] = rem - q * b;
                rem = q;
            }
            for (int u = 0; u < nsub; ++u) {
                int offA = 0, offR = 0;
#pragma unroll
                for (int k = 0; k < kMaxOrder; ++k) {
                    if (k < s) {
                        offA += dig[k] * wA[u][k];
                        offR += dig[k] * wR[u][k];
                    }
                }
                const int la = la_s[u], lr = lr_s[u];
                const double cA = a.C[la][(int64_t)sr[2 * u] * bpow[la] + offA];
                const double sR = a.S[lr][(int64_t)sr[2 * u + 1] * bpow[lr] + offR];
                acc = fma(-cA, sR, acc);
            }
            const double c = acc * a.invT;
            a.Cout[e] = c;
            local = fma(mult * c, c, local);
        }
    }
    // deterministic CTA reduction
    __shared__ double red[NT];
    red[threadIdx.x] = local;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.normpart[blockIdx.x] = red[0];
}

// One warp per order: lanes add strided partials, then a fixed shuffle tree.
__global__ void k_norm_final(const double* __restrict__ normpart, const int32_t* __restrict__ part_off,
                             int d, double* __restrict__ fro2, int64_t* __restrict__ head,
                             int64_t advance, int64_t T)
{
    const int lane = threadIdx.x & 31, s = threadIdx.x >> 5;
    if (threadIdx.x == 0 && advance != 0) *head = (*head + advance) % T;
    if (s >= d) return;
    double z = 0.0;
    for (int q = part_off[s] + lane; q < part_off[s + 1]; q += 32) z += normpart[q];
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    if (lane == 0) fro2[s] = z;
}

}  // namespace

cudaError_t launch_cumulants(const CumArgs& a, int grid, cudaStream_t st)
{
    k_cumulants<<<grid, NT, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_norm_final(const double* normpart, const int32_t* part_off, int d, double* fro2,
                              int64_t* head, int64_t advance, int64_t T, cudaStream_t st)
{
    k_norm_final<<<1, 32 * kMaxOrder, 0, st>>>(normpart, part_off, d, fro2, head, advance, T);
    return cudaGetLastError();
}

}  // namespace cw
