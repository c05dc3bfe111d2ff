// Internal definitions shared by the host library and the CUDA kernels.
#pragma once

#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include <cuda_runtime.h>

namespace cw {

// Raise a kernel's dynamic shared memory limit to `bytes` on the current
// device; done once per (kernel, device) and size, under a lock, so that
// launches on several devices or threads each get the opt-in.
inline cudaError_t smem_opt_in(const void* func, size_t bytes)
{
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = done[{func, dev}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

constexpr int kMaxOrder = 8;
constexpr int kMaxN = 256;

// ---------------------------------------------------------------------------
// Moment-sum update (Eqs. 6-7, Algorithm 2) as a set of dense GEMMs.
//
// For order s the stored elements are split between a left factor of h = ceil(s/2)
// indices and a right factor of sh = s - h indices.  Left rows are (sorted
// block h-tuple jL, in-block aL) grouped by the last block index m of jL;
// right columns are (sorted block sh-tuple jR, aR) in lexicographic order.
// Group m pairs its rows with every column whose first block index is >= m,
// so that jL ++ jR is a sorted block s-tuple, and every stored element is
// produced exactly once:
//     dS[rowoff[r] + coloff[c]] = sum_t sign_t * prod_{k<h} y[t, rowvar_k(r)]
//                                              * prod_{k<sh} y[t, colvar_k(c)]
// rowvar/colvar pack the variable indices one byte each (lowest byte first).
// ---------------------------------------------------------------------------
struct OrderTables {
    const uint32_t* rowvar;
    const int64_t* rowoff;
    const uint32_t* colvar;
    const int64_t* coloff;
    double* S;      // running FP64 sums of order s (block layout)
    double* F;      // FP64 form: batch-sum FIFO slot 0 of order s (same indexing as S), or null
    int32_t h, sh;  // factors on the row side / column side
    int32_t nrows, ncols;
};

// FIFO of batch sums, FP64 form (Section 2.4's alternative to recomputing
// X_(-)): for a window of T = nslots * p samples, slot f holds the FP64 sums of
// the batch of p ring rows starting at f * p + (head mod p).  A regular shift
// forms only the entering batch's sums D and applies S += D - F[slot],
// F[slot] = D, with slot = head / p (head before the shift advances it).
enum UpdFifoMode { kUpdNoFifo = 0, kUpdFifoStore = 1, kUpdFifoShift = 2 };

struct UpdateArgs {
    OrderTables ord[kMaxOrder + 1];  // index = order
    int32_t npad;                    // row stride of the sample buffers
    int32_t p, nslots;               // FIFO: batch length and slots (nslots = 0: no FIFO)
    int64_t fstride;                 // FIFO: doubles per slot
    const int64_t* head;             // FIFO: ring head of the window (device)
};

// One output tile of the update: rows [row0, row0+nrows) and columns
// [col0, col0+ncols) of the order-s GEMM of one group.
struct UpdTile {
    int32_t s, row0, nrows, col0, ncols, pad0, pad1, pad2;
};

// ---------------------------------------------------------------------------
// Moment-to-cumulant recovery (Algorithms 3-4) through the subset recursion
//     C_s[i] = M_s[i] - sum_{A contains position 0, A != all} C_|A|[i_A] M_{s-|A|}[i_rest]
// For a sorted block j every sub-tuple j_A is sorted, hence a stored block;
// subrank holds (rank(j_A), rank(j_rest)) for each block and each subset.
// ---------------------------------------------------------------------------
constexpr int kAccModes = 3;  // CumArgs::accum values

struct CumArgs {
    double* S[kMaxOrder + 1];        // running sums per order (moments = S * invT)
    const double* C[kMaxOrder + 1];  // cumulants per order (order 1 about the shift)
    double* Cout;                    // = C[s]
    const int32_t* subrank;          // [nblocks][nsub][2]
    const double* mult;              // [nblocks] block multiplicity s!/prod r_l!
    double* normpart;                // [gridDim.x] partial sums of mult * C^2
    const float* shift;              // order-1 norm uses C_1 + shift
    double invT;
    int32_t tpow2;  // k + 1 when T = 2^k, 0 otherwise
    int64_t E;                       // stored elements of order s
    int32_t s, b, bs, nsub;
    uint8_t mask[128];               // subset bitmasks over the s positions
    // tensor-core form: before recovering C_s, fold the FP32 tile sums of the
    // shift into S_s: S += (double)D_in - (double)D_out with D_in = sum_k W[k][0],
    // read at the element's workspace slot wblk[2 blk] + aL * wblk[2 blk + 1] + aR
    // (in-block offset a = aL * bR + aR).  accum 1: D_out = sum_k W[k][1];
    // accum 2: D_out = the element's entry in slot head / p of the batch-sum
    // FIFO (workspace order), which then takes D_in.
    const float* W;                  // [ksplit][2][wslice]
    const int32_t* wblk;             // [nblocks][2] (build_w_blocks)
    float* fifo;                     // this order's FIFO in slot 0 (accum 2)
    const int64_t* head;             // ring head (accum 2)
    int64_t wslice, woff, fstride;
    int32_t ksplit, accum;           // accum: 0 = no workspace, 1 = stacked in/out, 2 = FIFO
    int32_t bR, p;                   // b^(s - h); shift size (accum 2)
    int32_t sgemm;                   // S_s kept in workspace order (the top order and the canonical
                                     // orders of the mixed forms)
    // Mixed forms with d >= kTwoWordMinOrder: the orders below d also keep
    // C_k and S_k as two-word FP32 values (hi + lo, written by their own
    // recovery: `split`), and orders >= kTwoWordMinOrder form the products of
    // their subset sum in that two-word arithmetic (`twoword`), leaving only
    // the final subtraction from S_s, the scaling and the norm on the FP64 pipe.
    float2* C2[kMaxOrder + 1];
    float2* S2[kMaxOrder + 1];
    int32_t split, twoword;
    // Canonical recovery (CanonTables, cw_layout.h): C_s is computed once per
    // class of entries that super-symmetry makes equal, at the canonical
    // in-block offset, then copied to the other offsets of its block; canon = 0
    // when the order uses the per-element path.  Its update tables are
    // compressed (cw_layout.h): the workspace slot of a canonical element is
    // wblk[2 blk] + rL * wblk[2 blk + 1] + rR, (rL, rR) = can_lr / map_lr, and
    // its sums (workspace order) exist only at those slots.
    const int32_t* blkpat;
    const int32_t* can_start;
    const int32_t* can_off;
    const int32_t* map_off;
    const int32_t* can_copies;
    const int32_t* can_lr;     // per canonical offset: rL << 16 | rR
    const int32_t* map_lr;     // [npat][bs]: can_lr of each offset's canonical offset
    const int32_t* dup_start;
    const int2* dup;
    const int32_t* pblocks;    // the blocks recovered (all, or a shard's range), grouped by pattern
    const int4* units;
    int32_t nunits, canon, npblocks;
    // k_canon_expand also copies the two-word C_s and S_s to the non-canonical
    // offsets (only an order above without the canonical recovery reads them:
    // a canonical element's sub-tuples are canonical in their own blocks)
    int32_t split_copies;
};
constexpr int kTwoWordMinOrder = 5;
// Orders with the canonical recovery (when b^s >= kCanonMinBlock, single windows).
constexpr int kCanonMinOrder = 5;
constexpr int kCanonMaxOrder = 6;
constexpr int kCanonMinBlock = 256;
constexpr int kCanonSlice = 256;  // threads of a unit (one canonical element each)
constexpr int kCanonGroup = 8;    // blocks of a unit
constexpr int kCanonCtasPerSm = 4;  // resident k_canon CTAs per SM (64 registers a thread)

// Adjoint kernels (k_adjoint.cu): full-tensor expansion, contraction over the
// trailing indices, seeding, compaction over sorted tuples, and dL/dX.
cudaError_t launch_expand(const double* blk, int64_t nfull, int s, int n, int b, const int64_t* nst,
                          double scale, const float* add1, double* full, cudaStream_t st);
cudaError_t launch_contract(const double* G, const double* V, int64_t nx, int64_t ny, double alpha,
                            double* out, cudaStream_t st);
cudaError_t launch_seed(const double* C, double two_w, int64_t nfull, double* G, double* GM,
                        cudaStream_t st);
cudaError_t launch_compact(const double* GM, int s, int n, const uint64_t* uvars, const float* umult,
                           int nu, double coef, float* Gc, cudaStream_t st);
cudaError_t launch_grad_x(const float* ring, int64_t T, const int64_t* head, int n, int npad,
                          const float* shift, const uint64_t* uvars, const uint8_t* unf, int nu,
                          const float* Gc, float* dX, cudaStream_t st);

// Message returned by cumwin_last_error() on the calling thread.
void set_last_error(const std::string& msg);

// Device-side status bits (sticky).
constexpr int kStatusNonFinite = 1;
constexpr int kStatusTimeout = 2;

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files).
// ---------------------------------------------------------------------------
cudaError_t launch_stage(const float* x_in, int64_t ld_in, const float* x_out, int64_t ld_out,
                         float* ring, int64_t T, const int64_t* head, int p, int n, int npad,
                         float* stage, int* status, cudaStream_t st);
cudaError_t launch_fill_ring(const float* X, int64_t ldx, float* ring, int64_t T, int n, int npad,
                             int* status, cudaStream_t st);
cudaError_t launch_column_mean(const float* ring, int64_t T, int n, int npad, float* shift,
                               cudaStream_t st);
cudaError_t launch_window_copy(const float* ring, int64_t T, const int64_t* head, int n, int npad,
                               float* out, cudaStream_t st);
// fmode (UpdFifoMode): kUpdFifoStore stores the sums in FIFO slot (head / p + fq)
// mod nslots and adds them; kUpdFifoShift replaces slot head / p (all K rows enter).
cudaError_t launch_update_f64(const UpdateArgs& a, const UpdTile* tiles, int ntiles,
                              const float* rows, int64_t K, int64_t npos, const float* shift,
                              int fmode, int fq, cudaStream_t st);
// rows [r0, r0 + p) of the window (oldest first, from the ring's head) -> out [p][npad]
cudaError_t launch_window_rows(const float* ring, int64_t T, const int64_t* head, int64_t r0, int p,
                               int npad, float* out, cudaStream_t st);
// Launch shape of the recovery kernel of one order (see plan_cumulants).
struct CumLaunch {
    int slots, gx, gy;
    int bpow1;  // b^(s-1)
};
CumLaunch plan_cumulants(int s, int bs, int64_t nblocks, int sm_count);
// Recovery of order s for nwin windows at once (args_dev[w] for window w;
// windows without order s have E = 0).
cudaError_t launch_cumulants(int s, const CumArgs* args_dev, int nwin, const CumLaunch& L, cudaStream_t st);
// Canonical recovery of order s (kCanonMinOrder..kCanonMaxOrder): the
// canonical elements with their norm partials (grid CTAs over the order's
// units, one partial each; grid <= the order's norm partial slots) and, for
// the top order, the fold of the shift's batch sums at those elements; then
// the copies to the other offsets of every block (and their two-word copies
// for orders below d).
cudaError_t launch_canon(int s, const CumArgs* args_dev, int grid, cudaStream_t st);
cudaError_t launch_canon_expand(const CumArgs* args_dev, int grid, cudaStream_t st);
// Fold of the workspace into the sums of orders that are folded before their
// recovery runs (sums kept in workspace order, and canonical orders), one
// linear pass per window; others are skipped.
cudaError_t launch_fold_linear(const CumArgs* args_dev, int nwin, int64_t maxE, int sm_count, cudaStream_t st);
// Per-CTA partials of sum multiplicity * |C_s|^k (nparts CTAs).
cudaError_t launch_knorm(const CumArgs* args_dev, int64_t E, double k, double* partials, int nparts, cudaStream_t st);
// Two-word copies (CumArgs::C2 / S2) of orders 1..s_hi of the windows whose
// arguments are args_dev[order * nwin + window] (those with `split` set);
// maxE = the largest of their E.
cudaError_t launch_split(const CumArgs* args_dev, int nwin, int s_hi, int64_t maxE, int sm_count, cudaStream_t st);
// out[i] = src[idx[i]], i < n.
cudaError_t launch_gather_idx(const double* src, const int64_t* idx, int n, double* out, cudaStream_t st);
// out = S_s * scale in storage order for sums kept in workspace order.
cudaError_t launch_gather_sums(const CumArgs* args_dev, int64_t E, double scale, double* out, cudaStream_t st);

// Norm reduction of one window: partials of order s at normpart[(s-1)*parts ..].
struct NormArgs {
    const double* normpart;
    double* fro2;         // [d]
    int64_t* head;        // ring head of the recovery (FIFO slots), advanced by `advance` rows (mod T)
    int64_t* head_stage;  // ring head of the staging, advanced too when not null (FP64 form)
    int64_t T;
    int32_t parts, d;
    // Drift of the stream's mean from the shift vector (mixed forms; the fused
    // recovery measures it when drift_flag is not null): max_i |C_1[i]| /
    // sqrt(C_2[i,i]) with C_1 about the shift, into *drift; when it exceeds
    // drift_limit, *drift_flag (mapped host memory) is set to 1.
    const double* C1;
    const double* C2;
    double* drift;
    volatile int* drift_flag;
    double drift_limit;
    int32_t n, b, nbar;
};
// Orders s >= s_from only.  Also advances each ring head by `advance` rows
// (mod T): the head lives in device memory so that a captured shift can be
// replayed.
cudaError_t launch_norm_final(const NormArgs* args_dev, int nwin, int64_t advance, int s_from,
                              cudaStream_t st);

// Orders 1..dfused (dfused <= kFusedMax) of every window in one cooperative
// launch (grid barriers between its phases); one norm partial per work unit
// (a group of blocks of one window, or a 256-offset slice of one block), the
// norms of those orders reduced at the end, and the ring heads advanced when
// no higher order follows.
constexpr int kFusedMax = 4;
constexpr int kBarrierWords = 2;  // one 64-bit arrival counter
struct FusedRecovery {
    const CumArgs* args;     // args[s * nwin + w], one accumulate mode
    const int64_t* ustart;   // [(kFusedMax + 1)][nwin + 1] first work unit of each window, per order
    double* upart;           // norm partial of each work unit; order s from upoff[s]
    const NormArgs* norm;    // [nwin]
    unsigned* bar;           // grid barrier state [kBarrierWords], zero at creation
    int* status;
    const int64_t* abeg;     // [nseg + 1] first stored element of each (window, order) segment:
    const int32_t* aarg;     // [nseg] its index into args; orders <= 3 first (nseg_lo), then order 4
    int64_t upoff[kFusedMax + 1];
    int64_t utot[kFusedMax + 1];  // work units of each order (all windows): ustart[s][nwin]
    int64_t advance;
    int32_t nwin, advance_heads, nseg, nseg_lo, fold;
    int32_t slots[kFusedMax + 1], gy[kFusedMax + 1];
};
size_t fused_smem_bytes(const FusedRecovery& f, int dfused);
// Resident CTAs for the cooperative launch, at most per_sm_max per SM (0: not possible).
int fused_grid(int dfused, size_t smem, int sm_count, int per_sm_max);
cudaError_t launch_recover_fused(const FusedRecovery& f, int dfused, int grid, size_t smem, cudaStream_t st);
// ||C_s||, nu_s and L = sum_s w_s ||C_s||^2 from the squared norms (any
// output may be null).
struct EstArgs {
    double* fro;   // [d]
    double* nu;    // [d]
    double* loss;  // [1]
    double w[kMaxOrder + 1];
    int32_t d;
};
cudaError_t launch_estimators(const double* fro2, const EstArgs& a, cudaStream_t st);
cudaError_t launch_zero(double* p, int64_t count, cudaStream_t st);
cudaError_t launch_add_shift(const double* C1, const float* shift, int n, int npad, double* out,
                             cudaStream_t st);
cudaError_t launch_scale(const double* S, double invT, int64_t count, double* out, cudaStream_t st);

}  // namespace cw
