// Tensor-core (tcgen05) form of the moment-sum update: plan and launchers.
//
// One plan serves one or many independent windows ("streams", each with its
// own n, d, T, ring buffer and sums; b and p are shared).  The order-s update
// of a stream is the set of GEMMs described in cw_internal.h: the right factor
// (s - h indices, "columns") is the MMA M side (128 per item), the left factor
// (h indices, "rows") the MMA N side (up to kTcNmax rows).
//
// Per shift, for all streams at once (one launch per phase):
//   1. k_tc_stage_push: X_(+) (and X_(-) when the leaving samples are
//      recomputed), minus the shift vector, transposed to [variable][sample]
//      (FP32), zero-padded to P samples each.
//   2. k_kr_build: every distinct Khatri-Rao operand row (the products of its
//      variables over the staged samples) is formed once in FP32, split into
//      bf16 hi + lo and written with the samples contiguous, so that a TMA box
//      of 64 samples (128 bytes) x rows lands in shared memory in the
//      128-byte-swizzled K-major layout the MMA descriptors read.
//   3. k_kr_gemm (persistent): per unit (item x K-split) a TMA warp streams the
//      item's A (128 columns) and B (rows) tiles through a 3-stage mbarrier
//      ring, an MMA warp issues hi*hi + hi*lo + lo*hi per 16-sample step into
//      one of two TMEM accumulator sets (entering samples into D_in, leaving
//      samples into D_out), and four epilogue warps store the FP32 tiles into
//      a workspace W[split][in/out] while the next unit's MMAs run.  The
//      workspace is in GEMM order (each row's outputs contiguous, see
//      build_w_rows), so the stores are whole 128-byte lines.
//   4. the recovery kernel of each order folds the workspace into the FP64
//      sums: S += (double)(sum_k D_in,k) - (double)(D_out), the FP32 sums over
//      splits taken in a fixed order.  D_out is either recomputed from the
//      leaving samples (stacked form) or, when T is a multiple of p, read from
//      a FIFO that keeps each batch's FP32 sum from when it entered (the
//      batch-moment variant of Section 2.4; the leaving half of the GEMM is
//      then skipped).  Either way a batch's sum is bitwise the same when it
//      enters and when it leaves the window.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <functional>
#include <vector>

#include "cw_internal.h"
#include "cw_layout.h"

namespace cw {

constexpr int kTcKC = 64;      // samples per K-chunk (one 128-byte swizzle row)
constexpr int kTcM = 128;      // columns per item (MMA M)
constexpr int kTcNmax = 128;   // rows per item (MMA N, multiple of 16)
constexpr int kTcStages = 3;   // TMA / MMA pipeline depth (64 KB per stage)

// Per-stream state the staging / build kernels read (device array).
struct TcStreamDesc {
    float* ring;
    int64_t* head;      // ring head of the staging (advanced by the operand build of a shift)
    const float* shift;
    float* XT;          // [npad][Kcap]
    float* vmax;        // [2][npad] largest |staged sample| per variable, entering / leaving half
                        // (FP16 form: the power-of-two scale of the variable's factors)
    int* status;
    int64_t T;
    int64_t xoff;       // offset of this stream's X_(+) rows in a packed push buffer
    int32_t n, npad;
};

struct TcItem {
    int32_t s;      // order
    int32_t row0;   // first row in the order's left table
    int32_t nrows;  // rows (<= kTcNmax)
    int32_t col0;   // first column in the order's right table
    int32_t ncols;  // columns (<= kTcM)
    int32_t brow;   // TMA row coordinate of row0 in the operand array
    int32_t acol;   // TMA row coordinate of col0 in the operand array
    int32_t bbox;   // rows of the B tile box (32, 64 or 128)
    int32_t stream; // index of the stream
    int32_t fast;   // all rows in one group: slot(row0 + k, c) = wrow0 + k * wwidth + c
    int32_t wwidth; // row stride of the group in the workspace (fast items)
    int32_t wrow0;  // workspace slot of (row0, column 0) (fast items)
};

// Per (stream, order) tables of the epilogue (device array [stream][kMaxOrder + 1]).
struct TcOrder {
    const int64_t* roww;       // workspace slot of (row r, column 0): slot(r, c) = roww[r] + c
    const int32_t* rowcolmin;  // first valid column of each row (its group's start)
    int64_t woff;              // offset of this (stream, order) in one workspace slice
};

struct TcGemmArgs {
    const TcOrder* ord;
    const TcItem* items;
    const int32_t* opexp;  // FP16 form: [2][oprows] power-of-two exponent of each operand row
    int64_t oprows;
    float* W;            // [ksplit][2][wslice] FP32 tile sums
    int64_t wslice;
    int32_t nitems, ksplit;
    int32_t nplus, nminus;  // K-chunks of the entering / leaving segment
    int32_t minus_k;        // first sample of the leaving segment
    int* status;
};

// One shift of a batch as a single cooperative launch (k_batch_shift): the
// staging, the operand build, the GEMM and the fused recovery of orders 1..4
// as phases separated by grid barriers.
struct BatchShiftArgs {
    const TcStreamDesc* sdesc;
    const float* xin;         // packed X_(+) of all streams
    int32_t p, P, nstreams, tiles_x, tiles_y, leaving, scaled;
    int64_t Kcap;
    float* vmax;              // FP16 form: per-variable maxima, zeroed first
    int64_t nvmax;
    const uint64_t* opvars;   // operand build
    int64_t oprows;
    uint16_t* ops;
    int32_t* opexp;
    int32_t nkb;
    TcGemmArgs gemm;
};

// Host description of one stream for the planner.
struct TcPlanStream {
    const std::vector<UpdateTables>* tables;  // [order]
    const UpdateArgs* upd;                    // device tables of the update
    const int64_t* Eoff;                      // [order] element offsets inside the stream
    int d, n, npad;
    int64_t T;
    float* ring;
    int64_t* head;
    const float* shift;
    int* status;
    int64_t xoff;
    // block shard of the top order d (lexicographic block ranks [top0, top1)):
    // only the rows whose blocks meet it are updated; top1 < 0 = all blocks
    int64_t top0 = 0, top1 = -1;
};

// The GEMM of one (stream, order) before it is cut into items: its row ranges
// (groups split or merged, each pairing with the columns from c0 on), and
// what an item needs to address its operands and workspace slots.
struct TcRangeSet {
    int s = 0, stream = 0, ncols = 0;
    int64_t loff = 0, roff = 0;           // first row of the left / right operand set in the operand array
    std::vector<int32_t> rowstart, colstart;
    std::vector<int64_t> roww;            // workspace slot of (row, column 0)
    std::vector<int32_t> colmin;          // first valid column of each row
    struct Range { int r0, r1, c0; };
    std::vector<Range> ranges;
};

struct TcPlan {
    int ready = 0;
    int precision = 0;
    int nstreams = 0, p = 0, P = 0, nbatch = 0, sm_count = 1;
    int64_t Kcap = 0;
    TcStreamDesc* sdesc = nullptr;  // device [nstreams]
    int npad_max = 0;
    // operand array: rows of all Khatri-Rao sets of all streams, [part][row][Kcap] bf16
    uint16_t* ops = nullptr;
    int64_t oprows = 0;
    uint64_t* opvars = nullptr;    // per row: packed variables | factors << 32 | stream << 40
    // FP16 form: the operand rows are scaled by powers of two so that every
    // factor lies in [-1, 1] (FP16 has 5 exponent bits); vmax holds the largest
    // |staged sample| per (stream, half, variable), zeroed before each staging,
    // and opexp the exponent of each row's scale, undone exactly in the epilogue
    float* vmax = nullptr;         // [nstreams][2][npad_max]
    int32_t* opexp = nullptr;      // [2][oprows]
    CUtensorMap mapA{}, mapB[3]{};  // A boxes of 128 rows; B boxes of 32, 64, 128 rows
    TcItem* items = nullptr;
    int nitems = 0, ksplit = 1, ksplit_max = 1;
    // tile shape (tc_plan_items): rows per item at most `nmax` (64 or 128), and
    // items issued in super-blocks of `group` row tiles x all their column tiles,
    // column-major inside a block, so that the CTAs running at the same time
    // share a few left-factor tiles and a run of right-factor tiles in L2
    int nmax = kTcNmax, group = 8, items_cap = 0;
    std::vector<TcRangeSet> rsets;
    TcOrder* ord = nullptr;        // device [nstreams][kMaxOrder + 1]
    float* W = nullptr;
    float* W2 = nullptr;           // second workspace (shifts alternate) or null
    int64_t wslice = 0;
    std::vector<int64_t> wbase;    // per stream: offset of the stream in a workspace slice
    std::vector<int> nbatch_stream;
    // batch-sum FIFO (null when some T is not a multiple of p, or it does not
    // fit): stream i keeps T_i / p slots of its E_i = sum_s E_s FP32 sums in
    // workspace order at fifo + fbase[i] + slot * E_i
    float* fifo = nullptr;
    std::vector<int64_t> fbase;
    int* status = nullptr;
    double useful_macs_per_sample = 0, issued_macs_per_sample = 0;
};

// The single-launch batch shift (k_cumulants.cu): resident CTAs per SM of its
// 1024-thread CTA (0: it cannot run), and its launch with `grid` CTAs.
int batch_shift_blocks_per_sm(int precision, int dfused);
cudaError_t launch_batch_shift(const TcPlan& plan, const BatchShiftArgs& a, const FusedRecovery& f, int dfused,
                               int grid, cudaStream_t st);
// The GEMM arguments of one shift (nplus / nminus K-chunks of the entering and
// leaving samples; parity 1 = the second workspace when there is one).
TcGemmArgs tc_gemm_args(const TcPlan& plan, bool leaving, int parity);

using DevAlloc = std::function<cudaError_t(size_t, void**)>;

// Returns 0 or a cudaError_t code.
// `fifo`: allocate the batch-sum FIFO when every T is a multiple of p and it
// takes at most a quarter of the free device memory.  `double_w`: a second
// workspace, so that the GEMM of a shift can run while the recovery of the
// previous shift still reads the first.
int tc_plan_create(TcPlan& plan, const std::vector<TcPlanStream>& streams, int b, int p, int sm_count,
                   int precision, int* status, bool fifo, bool double_w, const DevAlloc& alloc);

// Staging + operand build for all streams (2 launches).  Stream i reads its
// X_(+) at xin + xoff_i (row stride ld, or n_i when ld < 0).  With `leaving`,
// X_(-) is staged too: from xout + xoff_i when xout is not null, else from the
// ring buffer.
cudaError_t tc_stage_push(const TcPlan& plan, const float* xin, const float* xout, int64_t ld, int p,
                          bool leaving, cudaStream_t st);
// The GEMM units of a shift (1 launch); `leaving` adds the X_(-) half;
// `parity` 1 writes the second workspace when there is one.
cudaError_t tc_gemm_push(const TcPlan& plan, bool leaving, int parity, cudaStream_t st);

// Batch q (window order, p samples) of every stream's ring buffer: stage, build
// and GEMM with no leaving segment (3 launches); streams with fewer batches
// contribute zeros.  Then fold the workspace into the sums with
// launch_tc_accumulate.
cudaError_t tc_update_window_batch(const TcPlan& plan, int q, cudaStream_t st);

// Batch q of a window's sums, one (stream, order) segment: S += (double)D_in
// with D_in = sum_k W[k][0] at the element's workspace slot, and, with a FIFO,
// D_in is kept in slot (head / p + q) mod nslots of the stream's FIFO.
struct TcAccSeg {
    double* S;
    const int32_t* wblk;   // build_w_blocks of the order
    float* fifo;           // FIFO of the order in slot 0, or null
    const int64_t* head;   // ring head of the stream
    int64_t begin;         // first element of the segment in a workspace slice
    int64_t E;             // elements of the segment
    int64_t fstride;       // FIFO slot stride (floats)
    int32_t bs, bR;        // b^s, b^(s - h)
    int32_t p, nslots;
    int32_t sgemm, pad;    // S in workspace order
};
cudaError_t launch_tc_accumulate(const TcPlan& plan, const TcAccSeg* segs_dev, int nsegs, int q,
                                 cudaStream_t st);

// Cut the GEMMs into items of at most nmax rows (a multiple of 16, <= kTcNmax)
// issued in super-blocks of `group` row tiles, and upload them (0 or a
// cudaError_t code).
int tc_plan_items(TcPlan& plan, int nmax, int group);

// Time the GEMM for candidate tile shapes (rows per item 128 or 64, super-block
// heights 1, 4, 8, 16) and then K-splits on the data currently staged, and keep
// the fastest; returns the chosen K-split (or a negative cudaError_t).
// `leaving`: time the shape with the X_(-) half.
int tc_autotune(TcPlan& plan, int reps, bool leaving, cudaStream_t st, double* best_ms);

}  // namespace cw
