// Moment-to-cumulant recovery (Algorithms 3-4) and cumulant norms (Eq. me,
// Algorithm 5), FP64.
//
// Algorithm 4 sums, for every element, products of lower-order cumulants over
// all set partitions of its s indices.  Grouping those partitions by the part
// that holds the first index gives the equivalent subset recursion
//     C_s[i] = M_s[i] - sum_{A contains index 1, A != all} C_|A|[i_A] M_{s-|A|}[i_rest]
// (2^{s-1} - 1 terms instead of B(s) - 1), which is what runs here.  For a
// sorted block j every sub-tuple j_A is sorted, so the operands are stored
// blocks whose ranks come from a per-block table; the in-block offsets follow
// from the element's own in-block digits because diagonal blocks are stored
// whole.  The same pass accumulates multiplicity * C^2 for the norm
// (Algorithm 5 with k = 2) into one partial per CTA; a second kernel adds the
// partials of each order in a fixed order.
#include "cw_internal.h"

namespace cw {

namespace {

constexpr int NT = 256;

__global__ void __launch_bounds__(NT) k_cumulants(const CumArgs a)
{
    const int s = a.s, b = a.b;
    int bpow[kMaxOrder + 1];
    bpow[0] = 1;
    for (int k = 1; k <= kMaxOrder; ++k) bpow[k] = bpow[k - 1] * b;
    const double* __restrict__ Ss = a.S[s];
    double local = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * NT + threadIdx.x; e < a.E;
         e += (int64_t)gridDim.x * NT) {
        const int64_t blk = e / a.bs;
        const int off = (int)(e - blk * a.bs);
        double c = Ss[e] * a.invT;
        if (s == 1) {
            a.Cout[e] = c;
            const double x = c + (double)a.shift[e];
            local += x * x;
            continue;
        }
        int dig[kMaxOrder];
        int rem = off;
        for (int k = s - 1; k >= 0; --k) {
            dig[k] = rem % b;
            rem /= b;
        }
        const int32_t* sr = a.subrank + (size_t)blk * a.nsub * 2;
        for (int u = 0; u < a.nsub; ++u) {
            const unsigned mask = a.mask[u];
            int offA = 0, offR = 0, la = 0, lr = 0;
            for (int k = 0; k < s; ++k) {
                if ((mask >> k) & 1u) {
                    offA = offA * b + dig[k];
                    ++la;
                } else {
                    offR = offR * b + dig[k];
                    ++lr;
                }
            }
            const double cA = a.C[la][(int64_t)sr[2 * u] * bpow[la] + offA];
            const double mR = a.S[lr][(int64_t)sr[2 * u + 1] * bpow[lr] + offR] * a.invT;
            c = fma(-cA, mR, c);
        }
        a.Cout[e] = c;
        local += a.mult[blk] * c * c;
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

__global__ void k_norm_final(const double* __restrict__ normpart, const int32_t* __restrict__ part_off,
                             int d, double* __restrict__ fro2, int64_t* __restrict__ head,
                             int64_t advance, int64_t T)
{
    const int s = threadIdx.x;
    if (s == 0 && advance != 0) *head = (*head + advance) % T;
    if (s >= d) return;
    double z = 0.0;
    for (int q = part_off[s]; q < part_off[s + 1]; ++q) z += normpart[q];
    fro2[s] = z;
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
    k_norm_final<<<1, 32, 0, st>>>(normpart, part_off, d, fro2, head, advance, T);
    return cudaGetLastError();
}

}  // namespace cw
