// Squared Frobenius norm of a block-layout super-symmetric tensor for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool or under a memory budget that forbids new device
// allocations, or a host thread that must not risk the implicit
// synchronisation an allocation can cause.  They still need the norm of a
// tensor they hold.  This entry point computes it with no allocation: its
// scratch (one partial per stored block) is a file-scope __device__ array of
// fixed size that every GPU loading the library keeps until exit.
//
// The host code below never hands the array's host-side name to a kernel:
// the device address is looked up with cudaGetSymbolAddress with the device
// current.  Outside stream capture it is looked up on every call (the lookup
// allocates nothing), so a device reset that tears the context down cannot
// leave a stale address behind; under capture the address cached by the last
// uncaptured call on that device is used.
#include <climits>
#include <mutex>
#include <string>

#include "../../include/cumwin.h"
#include "cw_internal.h"
#include "cw_layout.h"

namespace cw {

namespace {

constexpr int kMaxDevices = 64;

// One partial per stored block; every call overwrites the slots it reads.
static __device__ __align__(256) double g_block_norm_scratch[CUMWIN_NOALLOC_MAX_BLOCKS];

__device__ __forceinline__ int64_t d_binom(int64_t a, int k)
{
    if (k < 0 || a < k) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (a - k + i) / i;
    return r;
}

// Pass 1: one warp per block; lane 0 recovers the sorted block tuple from its
// lexicographic rank to get the multiplicity s!/prod r_l! (r_l the run
// lengths of equal block indices).
__global__ void __launch_bounds__(256)
k_block_sumsq(const double* __restrict__ A, int64_t nblocks, int64_t bs, int s, int nbar,
              double* __restrict__ part)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t blk = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); blk < nblocks;
         blk += warps) {
        double acc = 0.0;
        for (int64_t e = lane; e < bs; e += 32) {
            const double v = A[blk * bs + e];
            acc = fma(v, v, acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            int64_t r = blk;
            int prev = 0, run = 0, last = -1;
            double mult = 1.0;
            for (int i = 2; i <= s; ++i) mult *= i;
            for (int k = 0; k < s; ++k) {
                int v = prev;
                for (; v < nbar; ++v) {
                    const int64_t cnt = d_binom((int64_t)(nbar - v) + (s - k - 1) - 1, s - k - 1);
                    if (r < cnt) break;
                    r -= cnt;
                }
                if (v == last) {
                    ++run;
                } else {
                    for (int i = 2; i <= run; ++i) mult /= i;
                    run = 1;
                    last = v;
                }
                prev = v;
            }
            for (int i = 2; i <= run; ++i) mult /= i;
            part[blk] = mult * acc;
        }
    }
}

// Pass 2: one CTA adds the partials in a fixed order.
__global__ void __launch_bounds__(256)
k_sum_parts(const double* __restrict__ part, int64_t nblocks, double* __restrict__ out)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < nblocks; i += blockDim.x) acc += part[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

}  // namespace

}  // namespace cw

extern "C" int cumwin_block_norm2_noalloc(int n, int b, int order, const double* A_dev,
                                          double* out_dev, void* cuda_stream)
{
    using namespace cw;
    if (n < 1 || n > kMaxN || b < 1 || order < 1 || order > kMaxOrder || A_dev == nullptr ||
        out_dev == nullptr) {
        set_last_error("invalid argument");
        return CUMWIN_EINVAL;
    }
    const int nbar = (n + b - 1) / b;
    // the padded variable count is bounded as for cumwin_create (so b <= 256),
    // and a block must hold fewer than 2^31 elements; b^order is formed with a
    // check after every factor, so it cannot overflow
    int64_t bs = 1;
    bool big = (int64_t)nbar * b > kMaxN;
    for (int k = 0; k < order && !big; ++k) {
        bs *= b;
        big = bs > INT_MAX;
    }
    if (big) {
        set_last_error("block size too large: nbar * b must be at most " + std::to_string(kMaxN) +
                       " and b^order below 2^31");
        return CUMWIN_EINVAL;
    }
    const int64_t nblocks = n_sorted(nbar, order);
    if (nblocks > CUMWIN_NOALLOC_MAX_BLOCKS) {
        set_last_error("tensor has " + std::to_string(nblocks) +
                       " stored blocks, more than the fixed scratch of " +
                       std::to_string(CUMWIN_NOALLOC_MAX_BLOCKS) + " blocks");
        return CUMWIN_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_last_error("no usable current device");
        return CUMWIN_ECUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // Look the scratch address up on every call made outside stream capture
    // (cheap, no allocation; survives a device reset), and fall back to the
    // address of the last uncaptured call on this device while capturing.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capture = cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!capture) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_block_norm_scratch);
            if (e != cudaSuccess || p == nullptr) {
                set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return CUMWIN_ECUDA;
            }
            g_scratch_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    if (scratch == nullptr) {
        set_last_error("the first call on a device must come before any stream capture");
        return CUMWIN_ESTATE;
    }
    int64_t grid = (nblocks + 7) / 8;
    if (grid > 1024) grid = 1024;
    k_block_sumsq<<<(int)grid, 256, 0, st>>>(A_dev, nblocks, bs, order, nbar, scratch);
    k_sum_parts<<<1, 256, 0, st>>>(scratch, nblocks, out_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("launch: ") + cudaGetErrorString(e));
        return CUMWIN_ECUDA;
    }
    return CUMWIN_OK;
}
