// Tensor-core (tcgen05) form of the moment-sum update: plan and launchers.
//
// The order-s update is the set of GEMMs described in cw_internal.h.  Here the
// right factor (s - h indices, "columns") is the MMA M side (128 per item) and
// the left factor (h indices, "rows") the MMA N side (up to 256 per item).
// Each K-chunk of samples is staged in shared memory by TMA (FP32, already
// shifted), the Khatri-Rao products are formed on the CUDA cores and split
// into 16-bit hi + lo parts, and hi*hi + hi*lo + lo*hi are accumulated in
// FP32 in tensor memory: samples entering the window into one accumulator,
// samples leaving it into another.  The epilogue adds (double)D_in -
// (double)D_out to the FP64 running sums.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <functional>
#include <vector>

#include "cw_internal.h"
#include "cw_layout.h"

namespace cw {

constexpr int kTcKC = 32;      // samples per K-chunk
constexpr int kTcXS = 36;      // shared-memory row stride of the staged samples (floats)
constexpr int kTcM = 128;      // columns per item (MMA M)
constexpr int kTcNmax = 256;   // rows per item (MMA N)

struct TcItem {
    int32_t s, row0, nrows, col0, ncols, pad0, pad1, pad2;
};

struct TcOrder {
    const uint32_t* rowvar;
    const int64_t* rowoff;
    const int32_t* rowcolmin;  // first valid column of each row (its group's start)
    const uint32_t* colvar;
    const int64_t* coloff;
    double* S;
    int32_t h, sh;
};

struct TcArgs {
    TcOrder ord[kMaxOrder + 1];
    const TcItem* items;
    int32_t nitems;
    int32_t npad;
    // pass structure (sample counts, multiples of kTcKC): pair j adds the
    // plus segment [j*seg_stride, j*seg_stride + seglen) and, for j == 0, the
    // minus segment [minus_off, minus_off + minus_len); one epilogue per pair.
    int32_t npairs, seglen, seg_stride, minus_off, minus_len;
    int* status;
};

struct TcPlan {
    int ready = 0;
    int precision = 0;
    int npad = 0, p = 0, nbatch = 0, P = 0;
    int64_t T = 0, Kcap = 0;
    float* XT = nullptr;  // [npad][Kcap] shifted samples, var-major
    CUtensorMap xmap{};
    TcItem* items = nullptr;
    int nitems = 0, grid = 0;
    TcOrder ord[kMaxOrder + 1]{};
    int* status = nullptr;
    // planning statistics (host)
    double useful_macs_per_sample = 0, issued_macs_per_sample = 0;
};

using DevAlloc = std::function<cudaError_t(size_t, void**)>;

// Returns 0 or a cudaError_t code.
int tc_plan_create(TcPlan& plan, const std::vector<UpdateTables>& tables, const UpdateArgs& upd,
                   int d, int n, int b, int npad, int64_t T, int p, int sm_count, int precision,
                   int* status, const DevAlloc& alloc);

// Number of kernels one tc_update_* call issues.
int tc_launch_count(const TcPlan& plan);

// One window shift: stage X_(+) / X_(-) (shifted, transposed) and update the sums.
cudaError_t tc_update_push(const TcPlan& plan, const float* x_in, int64_t ld_in, const float* x_out,
                           int64_t ld_out, float* ring, const int64_t* head, int p, int n,
                           const float* shift, cudaStream_t st);

// Sums of the whole window held in the ring buffer, in batches of the nominal
// shift size taken in window order (fill and recompute).
cudaError_t tc_update_window(const TcPlan& plan, const float* ring, const int64_t* head, int n,
                             const float* shift, cudaStream_t st);

}  // namespace cw
