// Tensor-core (tcgen05) form of the moment-sum update: plan and launcher.
#pragma once

#include <cstdint>
#include <functional>
#include <vector>

#include "cw_internal.h"
#include "cw_layout.h"

namespace cw {

struct TcPlan {
    int ready = 0;
};

using DevAlloc = std::function<cudaError_t(size_t, void**)>;

// Returns 0 or a cudaError_t code.
int tc_plan_create(TcPlan& plan, const std::vector<UpdateTables>& tables, int d, int n, int b,
                   int npad, int T, int sm_count, int precision, const DevAlloc& alloc);

// Number of kernels one launch_update_tc call issues.
int tc_launch_count(const TcPlan& plan, int64_t K, int64_t npos, int64_t batch);

cudaError_t launch_update_tc(const TcPlan& plan, const UpdateArgs& a, const float* rows, int64_t K,
                             int64_t npos, int64_t batch, const float* shift, cudaStream_t st);

}  // namespace cw
