// Moment-sum update, FP64 form (Eqs. 6-7, Algorithm 2).
//
// Every tile is a 64 x 64 block of one order-s GEMM (see UpdateArgs):
//     S[rowoff[r] + coloff[c]] += sum_k sign_k * L[k][r] * R[k][c]
// with L[k][r] = prod of h entries of sample k (the row's variables) and
// R[k][c] = prod of s-h entries (the column's variables), i.e. an on-the-fly
// Khatri-Rao product of the staged samples.  The samples are staged in shared
// memory as FP64 (x - shift), the Khatri-Rao operands are built per K-chunk in
// shared memory, and each thread accumulates a 4 x 4 register tile in FP64.
// Every stored element belongs to exactly one tile, so the read-modify-write of
// the running sums needs no atomics and the result is deterministic.  With the
// batch-sum FIFO (UpdFifoMode) the epilogue also stores the tile's sums in the
// batch's slot and, for a regular shift, subtracts the leaving batch's stored
// sums instead of multiplying its samples again.
#include "cw_internal.h"

namespace cw {

namespace {

constexpr int TM = 64, TN = 64, KC = 16, NT = 256;

__device__ __forceinline__ double kr_product(const double* __restrict__ y, uint32_t vars, int cnt)
{
    double p = 1.0;
    for (int f = 0; f < cnt; ++f) p *= y[(vars >> (8 * f)) & 0xffu];
    return p;
}

__global__ void __launch_bounds__(NT)
k_update_f64(const UpdateArgs args, const UpdTile* __restrict__ tiles,
             const float* __restrict__ rows, int64_t K, int64_t npos,
             const float* __restrict__ shift, int fmode, int fq)
{
    extern __shared__ double smem[];
    const int npad = args.npad;
    double* ys = smem;                 // [KC][npad]
    double* As = ys + KC * npad;       // [KC][TM]
    double* Bs = As + KC * TM;         // [KC][TN]
    __shared__ uint32_t rv[TM], cv[TN];
    __shared__ int64_t ro[TM], co[TN];

    const UpdTile tile = tiles[blockIdx.x];
    const OrderTables& ot = args.ord[tile.s];
    const int tid = threadIdx.x;
    if (tid < TM) {
        const bool ok = tid < tile.nrows;
        rv[tid] = ok ? ot.rowvar[tile.row0 + tid] : 0u;
        ro[tid] = ok ? ot.rowoff[tile.row0 + tid] : 0;
    } else if (tid < TM + TN) {
        const int c = tid - TM;
        const bool ok = c < tile.ncols;
        cv[c] = ok ? ot.colvar[tile.col0 + c] : 0u;
        co[c] = ok ? ot.coloff[tile.col0 + c] : 0;
    }
    const int h = ot.h, sh = ot.sh;
    const int ty = tid / 16, tx = tid % 16;

    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    for (int64_t k0 = 0; k0 < K; k0 += KC) {
        __syncthreads();
        for (int e = tid; e < KC * npad; e += NT) {
            const int k = e / npad, v = e - k * npad;
            const int64_t t = k0 + k;
            ys[e] = t < K ? (double)rows[t * npad + v] - (double)shift[v] : 0.0;
        }
        __syncthreads();
        for (int e = tid; e < KC * TM; e += NT) {
            const int k = e / TM, r = e - k * TM;
            double a = r < tile.nrows ? kr_product(ys + k * npad, rv[r], h) : 0.0;
            As[e] = (k0 + k < npos) ? a : -a;
        }
        for (int e = tid; e < KC * TN; e += NT) {
            const int k = e / TN, c = e - k * TN;
            Bs[e] = c < tile.ncols ? kr_product(ys + k * npad, cv[c], sh) : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < KC; ++k) {
            double a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[k * TM + ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bb[j] = Bs[k * TN + tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
        }
    }

    double* F = nullptr;  // this launch's FIFO slot of order s
    if (fmode != kUpdNoFifo) {
        const int64_t hd = *args.head;
        F = ot.F + (hd / args.p + fq) % args.nslots * args.fstride;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = ty + 16 * i;
        if (r >= tile.nrows) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = tx + 16 * j;
            if (c >= tile.ncols) continue;
            const int64_t e = ro[r] + co[c];
            if (fmode == kUpdNoFifo) {
                ot.S[e] += acc[i][j];
            } else {
                const double leaving = fmode == kUpdFifoShift ? F[e] : 0.0;
                ot.S[e] += acc[i][j] - leaving;
                F[e] = acc[i][j];
            }
        }
    }
}

}  // namespace

cudaError_t launch_update_f64(const UpdateArgs& a, const UpdTile* tiles, int ntiles,
                              const float* rows, int64_t K, int64_t npos, const float* shift,
                              int fmode, int fq, cudaStream_t st)
{
    if (fmode != kUpdNoFifo && (a.nslots < 1 || a.p < 1 || a.head == nullptr)) return cudaErrorInvalidValue;
    if (ntiles <= 0 || K <= 0) return cudaSuccess;
    const size_t smem = sizeof(double) * ((size_t)KC * a.npad + KC * TM + KC * TN);
    cudaError_t e = smem_opt_in((const void*)k_update_f64, sizeof(double) * ((size_t)KC * kMaxN + KC * TM + KC * TN));
    if (e != cudaSuccess) return e;
    k_update_f64<<<ntiles, NT, smem, st>>>(a, tiles, rows, K, npos, shift, fmode, fq);
    return cudaGetLastError();
}

}  // namespace cw
