// Window buffer kernels: ring append / X_(-) extraction (Algorithm 1, "acquire
// X_(+)", "calculate X_(-) from the first t_up rows", "update the data
// buffer"), first-window load, shift vector, window read-out and small helpers.
#include "cw_internal.h"

namespace cw {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t work, int cap = 4096)
{
    int64_t g = (work + kThreads - 1) / kThreads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// stage rows [0, p) = X_(+), rows [p, 2p) = X_(-); the ring slots of X_(-)
// receive X_(+).  Each (row, variable) is read and written by one thread.
__global__ void __launch_bounds__(kThreads)
k_stage(const float* __restrict__ x_in, int64_t ld_in, const float* __restrict__ x_out,
        int64_t ld_out, float* __restrict__ ring, int64_t T, const int64_t* __restrict__ head_p,
        int p, int n, int npad, float* __restrict__ stage, int* __restrict__ status)
{
    const int64_t total = (int64_t)p * npad;
    const int64_t head = *head_p;
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / npad;
        const int v = (int)(e - r * npad);
        int64_t slot = head + r;
        if (slot >= T) slot -= T;
        const float xin = v < n ? x_in[r * ld_in + v] : 0.0f;
        float xo;
        if (x_out != nullptr) xo = v < n ? x_out[r * ld_out + v] : 0.0f;
        else xo = ring[slot * npad + v];
        stage[r * npad + v] = xin;
        stage[((int64_t)p + r) * npad + v] = xo;
        ring[slot * npad + v] = xin;
        bad |= !isfinite(xin);
    }
    if (bad) atomicOr(status, kStatusNonFinite);
}

__global__ void __launch_bounds__(kThreads)
k_fill_ring(const float* __restrict__ X, int64_t ldx, float* __restrict__ ring, int64_t T, int n,
            int npad, int* __restrict__ status)
{
    const int64_t total = T * npad;
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / npad;
        const int v = (int)(e - r * npad);
        const float x = v < n ? X[r * ldx + v] : 0.0f;
        ring[e] = x;
        bad |= !isfinite(x);
    }
    if (bad) atomicOr(status, kStatusNonFinite);
}

// One block per variable: FP64 column mean, rounded to FP32 (fixed order).
__global__ void __launch_bounds__(kThreads)
k_column_mean(const float* __restrict__ ring, int64_t T, int n, int npad, float* __restrict__ shift)
{
    const int v = blockIdx.x;
    __shared__ double red[kThreads];
    double acc = 0.0;
    if (v < n)
        for (int64_t r = threadIdx.x; r < T; r += blockDim.x) acc += (double)ring[r * npad + v];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) shift[v] = v < n ? (float)(red[0] / (double)T) : 0.0f;
}

__global__ void __launch_bounds__(kThreads)
k_window_copy(const float* __restrict__ ring, int64_t T, const int64_t* __restrict__ head_p, int n,
              int npad, float* __restrict__ out)
{
    const int64_t total = T * n;
    const int64_t head = *head_p;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / n;
        const int v = (int)(e - r * n);
        int64_t slot = head + r;
        if (slot >= T) slot -= T;
        out[e] = ring[slot * npad + v];
    }
}

// out[r][v] = window row r0 + r (ring slot head + r0 + r, wrapped), every padded column.
__global__ void __launch_bounds__(kThreads)
k_window_rows(const float* __restrict__ ring, int64_t T, const int64_t* __restrict__ head_p, int64_t r0, int p,
              int npad, float* __restrict__ out)
{
    const int64_t total = (int64_t)p * npad;
    const int64_t head = *head_p;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / npad;
        const int v = (int)(e - r * npad);
        const int64_t slot = (head + r0 + r) % T;
        out[e] = ring[slot * npad + v];
    }
}

__global__ void k_zero(double* __restrict__ p, int64_t count)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        p[e] = 0.0;
}

__global__ void k_add_shift(const double* __restrict__ C1, const float* __restrict__ shift, int n,
                            int npad, double* __restrict__ out)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < npad) out[v] = v < n ? C1[v] + (double)shift[v] : 0.0;
}

__global__ void k_scale(const double* __restrict__ S, double invT, int64_t count,
                        double* __restrict__ out)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = S[e] * invT;
}

}  // namespace

cudaError_t launch_stage(const float* x_in, int64_t ld_in, const float* x_out, int64_t ld_out,
                         float* ring, int64_t T, const int64_t* head, int p, int n, int npad,
                         float* stage, int* status, cudaStream_t st)
{
    k_stage<<<grid_for((int64_t)p * npad), kThreads, 0, st>>>(x_in, ld_in, x_out, ld_out, ring, T,
                                                               head, p, n, npad, stage, status);
    return cudaGetLastError();
}

cudaError_t launch_fill_ring(const float* X, int64_t ldx, float* ring, int64_t T, int n, int npad,
                             int* status, cudaStream_t st)
{
    k_fill_ring<<<grid_for(T * npad), kThreads, 0, st>>>(X, ldx, ring, T, n, npad, status);
    return cudaGetLastError();
}

cudaError_t launch_column_mean(const float* ring, int64_t T, int n, int npad, float* shift,
                               cudaStream_t st)
{
    k_column_mean<<<npad, kThreads, 0, st>>>(ring, T, n, npad, shift);
    return cudaGetLastError();
}

cudaError_t launch_window_copy(const float* ring, int64_t T, const int64_t* head, int n, int npad,
                               float* out, cudaStream_t st)
{
    k_window_copy<<<grid_for(T * n), kThreads, 0, st>>>(ring, T, head, n, npad, out);
    return cudaGetLastError();
}

cudaError_t launch_window_rows(const float* ring, int64_t T, const int64_t* head, int64_t r0, int p,
                               int npad, float* out, cudaStream_t st)
{
    k_window_rows<<<grid_for((int64_t)p * npad), kThreads, 0, st>>>(ring, T, head, r0, p, npad, out);
    return cudaGetLastError();
}

cudaError_t launch_zero(double* p, int64_t count, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    k_zero<<<grid_for(count), kThreads, 0, st>>>(p, count);
    return cudaGetLastError();
}

cudaError_t launch_add_shift(const double* C1, const float* shift, int n, int npad, double* out,
                             cudaStream_t st)
{
    k_add_shift<<<(npad + kThreads - 1) / kThreads, kThreads, 0, st>>>(C1, shift, n, npad, out);
    return cudaGetLastError();
}

cudaError_t launch_scale(const double* S, double invT, int64_t count, double* out, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    k_scale<<<grid_for(count), kThreads, 0, st>>>(S, invT, count, out);
    return cudaGetLastError();
}

}  // namespace cw
