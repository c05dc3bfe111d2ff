// Tensor-core (tcgen05) form of the moment-sum update: plan and launchers.
//
// The order-s update is the set of GEMMs described in cw_internal.h: the
// right factor (s - h indices, "columns") is the MMA M side (128 per item),
// the left factor (h indices, "rows") the MMA N side (up to kTcNmax rows).
//
// Per shift:
//   1. k_tc_stage_push: X_(+) and X_(-), minus the shift vector, transposed to
//      [variable][sample] (FP32), zero-padded to P samples each.
//   2. k_kr_build: every distinct Khatri-Rao operand row (the products of its
//      variables over the staged samples) is formed once in FP32, split into
//      bf16 hi + lo and written with the samples contiguous, so that a TMA box
//      of 64 samples (128 bytes) x rows lands in shared memory in the
//      128-byte-swizzled K-major layout the MMA descriptors read.
//   3. k_kr_gemm: per unit (item x K-split) a TMA warp streams the item's
//      A (128 columns) and B (rows) tiles through a 3-stage mbarrier ring, an
//      MMA warp issues hi*hi + hi*lo + lo*hi per 16-sample step into TMEM
//      (entering samples into D_in, leaving samples into D_out), and four
//      epilogue warps store the FP32 tiles into a workspace W[split][in/out].
//   4. the recovery kernel of each order first folds the workspace into the
//      FP64 sums: S += (double)(sum_k D_in,k) - (double)(sum_k D_out,k), the
//      FP32 sums over splits taken in a fixed order, so that a batch's sum is
//      bitwise the same when it enters and when it leaves the window.
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

struct TcItem {
    int32_t s;      // order
    int32_t row0;   // first row in the order's left table
    int32_t nrows;  // rows (<= kTcNmax)
    int32_t col0;   // first column in the order's right table
    int32_t ncols;  // columns (<= kTcM)
    int32_t brow;   // TMA row coordinate of row0 in the operand array
    int32_t acol;   // TMA row coordinate of col0 in the operand array
    int32_t bbox;   // rows of the B tile box (32, 64 or 128)
};

struct TcOrder {
    const int64_t* rowoff;
    const int32_t* rowcolmin;  // first valid column of each row (its group's start)
    const int64_t* coloff;
    int64_t woff;              // offset of this order in one workspace slice
};

struct TcGemmArgs {
    TcOrder ord[kMaxOrder + 1];
    const TcItem* items;
    float* W;            // [ksplit][2][Etot] FP32 tile sums
    int64_t wslice;      // Etot
    int32_t nitems, ksplit;
    int32_t nplus, nminus;  // K-chunks of the entering / leaving segment
    int32_t minus_k;        // first sample of the leaving segment
    int* status;
};

struct TcPlan {
    int ready = 0;
    int precision = 0;
    int npad = 0, p = 0, P = 0, nbatch = 0;
    int64_t T = 0, Kcap = 0;
    float* XT = nullptr;           // [npad][Kcap] shifted samples, variable-major
    // operand array: rows of all Khatri-Rao sets, [part][row][Kcap] bf16
    uint16_t* ops = nullptr;
    int64_t oprows = 0;
    uint64_t* opvars = nullptr;    // per operand row: packed variables | factors << 32
    CUtensorMap mapA{}, mapB[3]{};  // A boxes of 128 rows; B boxes of 32, 64, 128 rows
    TcItem* items = nullptr;
    int nitems = 0, ksplit = 1, sm_count = 1;
    TcOrder ord[kMaxOrder + 1]{};
    float* W = nullptr;
    int64_t wslice = 0;
    int* status = nullptr;
    // planning statistics (host)
    double useful_macs_per_sample = 0, issued_macs_per_sample = 0;
};

using DevAlloc = std::function<cudaError_t(size_t, void**)>;

// Returns 0 or a cudaError_t code.
int tc_plan_create(TcPlan& plan, const std::vector<UpdateTables>& tables, const UpdateArgs& upd,
                   const int64_t* Eoff, int d, int n, int b, int npad, int64_t T, int p,
                   int sm_count, int precision, int* status, const DevAlloc& alloc);

// One window shift, first half: stage X_(+) / X_(-) (moving X_(+) into the
// ring) and build the Khatri-Rao operands (2 launches).
cudaError_t tc_stage_push(const TcPlan& plan, const float* x_in, int64_t ld_in, const float* x_out,
                          int64_t ld_out, float* ring, const int64_t* head, int p, int n,
                          const float* shift, cudaStream_t st);
// Second half: the GEMM units (1 launch).  The FP64 sums are then updated by
// the recovery kernels in accumulate mode.
cudaError_t tc_gemm_push(const TcPlan& plan, cudaStream_t st);

// Batch q of the window held in the ring (window order, p_nominal samples):
// stage, build and GEMM with no leaving segment; the caller then folds the
// workspace into the sums (launch_tc_accumulate).
cudaError_t tc_update_window_batch(const TcPlan& plan, const float* ring, const int64_t* head,
                                   int q, int n, const float* shift, cudaStream_t st);

// S_s += (double)sum_k W[k][0] (entering only), all orders.
struct TcAccArgs {
    double* S[kMaxOrder + 1];
    int64_t Eoff[kMaxOrder + 2];
    int32_t d;
};
cudaError_t launch_tc_accumulate(const TcPlan& plan, const TcAccArgs& a, cudaStream_t st);

// Kernels one window batch launches (with the accumulation).
constexpr int kTcBatchLaunches = 4;

}  // namespace cw
