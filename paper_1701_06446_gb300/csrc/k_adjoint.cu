// Adjoint of L = sum_s w_s ||C_s||_F^2 with respect to the window (not in the
// paper; it differentiates Algorithms 2-4 and Eq. me).
//
// The cumulants are evaluated by the subset recursion
//     C_s[i] = M_s[i] - sum_{A contains 1, A != all} C_|A|[i_A] M_{s-|A|}[i_rest].
// Reverse mode over full (n^s) symmetric tensors: with G_s the adjoint of C_s,
//     G_s    = 2 w_s C_s + (contributions of higher orders)
//     GM_s  += G_s
// and every subset A of size k of an order-s term contributes, by symmetry,
// the same contraction, C(s-1, k-1) times:
//     G_k  -= C(s-1,k-1) * sum_y G_s[x, y] M_{s-k}[y]
//     GM_r -= C(s-1,k-1) * sum_y G_s[x, y] C_{s-r}[y]     (r = s - k)
// (all adjoints stay symmetric).  Finally, since M_s = (1/T) sum_t y_t^{(x)s}
// with y = x - shift,
//     dL/dx_{t,a} = sum_s (s/T) sum_{u in [n]^{s-1}} GM_s[a, u] prod_k y_{t,u_k},
// a transposed Khatri-Rao contraction evaluated over sorted (s-1)-tuples u
// weighted by their number of distinct orderings, in FP32.  The reverse
// recursion runs in FP64.
#include "cw_internal.h"

namespace cw {

namespace {

constexpr int NT = 256;

// Storage index of the full multi-index with digits (base n) of `f`: sort the
// variables, take the lexicographic rank of the sorted block tuple and the
// in-block offset.  nst[v * (kMaxOrder + 1) + r] = #sorted r-tuples over [v, nbar).
__device__ int64_t storage_index(int64_t f, int s, int n, int b, const int64_t* __restrict__ nst)
{
    int v[kMaxOrder];
    for (int k = s - 1; k >= 0; --k) {
        const int64_t q = f / n;
        v[k] = (int)(f - q * n);
        f = q;
    }
    // insertion sort (s <= 8)
    for (int i = 1; i < s; ++i) {
        const int x = v[i];
        int j = i - 1;
        while (j >= 0 && v[j] > x) {
            v[j + 1] = v[j];
            --j;
        }
        v[j + 1] = x;
    }
    int64_t rank = 0, off = 0;
    int prev = 0;
    for (int k = 0; k < s; ++k) {
        const int jk = v[k] / b;
        for (int u = prev; u < jk; ++u) rank += nst[u * (kMaxOrder + 1) + (s - k - 1)];
        prev = jk;
        off = off * b + (v[k] - jk * b);
    }
    int64_t bs = 1;
    for (int k = 0; k < s; ++k) bs *= b;
    return rank * bs + off;
}

// full[f] = scale * (block[storage(f)] + add[f's single variable] for order 1)
__global__ void __launch_bounds__(NT)
k_expand(const double* __restrict__ blk, int64_t nfull, int s, int n, int b, const int64_t* __restrict__ nst,
         double scale, const float* __restrict__ add1, double* __restrict__ full)
{
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nfull;
         f += (int64_t)gridDim.x * blockDim.x) {
        double x = blk[storage_index(f, s, n, b, nst)] * scale;
        if (add1 != nullptr) x += (double)add1[f];
        full[f] = x;
    }
}

// out[x] += alpha * sum_y G[x * ny + y] * V[y]   (one warp per x, fixed-order lanes)
__global__ void __launch_bounds__(NT)
k_contract(const double* __restrict__ G, const double* __restrict__ V, int64_t nx, int64_t ny, double alpha,
           double* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < nx;
         x += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        double acc = 0.0;
        for (int64_t y = lane; y < ny; y += 32) acc = fma(G[x * ny + y], V[y], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) out[x] += alpha * acc;
    }
}

// dst = 2 w C + dst (G_s from the accumulated higher-order contributions), GM += dst
__global__ void __launch_bounds__(NT)
k_seed(const double* __restrict__ C, double two_w, int64_t nfull, double* __restrict__ G, double* __restrict__ GM)
{
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nfull;
         f += (int64_t)gridDim.x * blockDim.x) {
        const double g = fma(two_w, C[f], G[f]);
        G[f] = g;
        GM[f] += g;
    }
}

// Gc[u][a] = coef * mult(u) * GM[a, u]  for sorted (s-1)-tuples u (FP32), s = order
__global__ void __launch_bounds__(NT)
k_compact(const double* __restrict__ GM, int s, int n, const uint64_t* __restrict__ uvars,
          const float* __restrict__ umult, int nu, double coef, float* __restrict__ Gc)
{
    const int64_t total = (int64_t)nu * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int u = (int)(e / n), a = (int)(e - (int64_t)u * n);
        int64_t f = a;
        const uint64_t vars = uvars[u];
        for (int k = 0; k < s - 1; ++k) f = f * n + (int)((vars >> (8 * k)) & 0xffu);
        Gc[e] = (float)(coef * (double)umult[u] * GM[f]);
    }
}

// dX[t][a] = sum_u prod_k y[t, u_k] * Gc[u][a], y = window row t (oldest first) - shift.
// CTA: 32 window rows; u in chunks of 64 staged in shared memory.
constexpr int AT = 32, AU = 64;
__global__ void __launch_bounds__(NT)
k_grad_x(const float* __restrict__ ring, int64_t T, const int64_t* __restrict__ head_p, int n, int npad,
         const float* __restrict__ shift, const uint64_t* __restrict__ uvars, const uint8_t* __restrict__ unf,
         int nu, const float* __restrict__ Gc, float* __restrict__ dX)
{
    extern __shared__ float sm[];
    float* ys = sm;                  // [AT][npad]
    float* kr = ys + AT * npad;      // [AT][AU]
    float* gs = kr + AT * AU;        // [AU][n]
    const int64_t head = *head_p;
    const int64_t t0 = (int64_t)blockIdx.x * AT;
    for (int e = threadIdx.x; e < AT * npad; e += NT) {
        const int tt = e / npad, v = e - tt * npad;
        const int64_t t = t0 + tt;
        float y = 0.0f;
        if (t < T && v < n) {
            int64_t slot = head + t;
            if (slot >= T) slot -= T;
            y = ring[slot * npad + v] - shift[v];
        }
        ys[e] = y;
    }
    // each thread: row tt = threadIdx.x / 8 (32 rows), columns a = (threadIdx.x % 8) + 8j, j < 32
    const int tt = threadIdx.x >> 3, a0 = threadIdx.x & 7;
    constexpr int NA = kMaxN / 8;
    float acc[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) acc[j] = 0.0f;
    const int na = (n - a0 + 7) / 8;  // columns of this thread
    for (int u0 = 0; u0 < nu; u0 += AU) {
        __syncthreads();
        for (int e = threadIdx.x; e < AT * AU; e += NT) {
            const int r = e / AU, uu = e - r * AU;
            const int u = u0 + uu;
            float p = 0.0f;
            if (u < nu) {
                p = 1.0f;
                const uint64_t vars = uvars[u];
                const int nf = unf[u];
                for (int k = 0; k < nf; ++k) p *= ys[r * npad + (int)((vars >> (8 * k)) & 0xffu)];
            }
            kr[e] = p;
        }
        for (int e = threadIdx.x; e < AU * n; e += NT) {
            const int uu = e / n;
            gs[e] = (u0 + uu < nu) ? Gc[(int64_t)u0 * n + e] : 0.0f;
        }
        __syncthreads();
        for (int uu = 0; uu < AU; ++uu) {
            const float k = kr[tt * AU + uu];
            const float* g = gs + uu * n + a0;
#pragma unroll
            for (int j = 0; j < NA; ++j)
                if (j < na) acc[j] = fmaf(k, g[8 * j], acc[j]);
        }
    }
    const int64_t t = t0 + tt;
    if (t < T) {
#pragma unroll
        for (int j = 0; j < NA; ++j)
            if (j < na) dX[t * n + a0 + 8 * j] = acc[j];
    }
}

inline int grid_for(int64_t work)
{
    int64_t g = (work + NT - 1) / NT;
    return (int)(g < 1 ? 1 : (g > 8192 ? 8192 : g));
}

}  // namespace

cudaError_t launch_expand(const double* blk, int64_t nfull, int s, int n, int b, const int64_t* nst,
                          double scale, const float* add1, double* full, cudaStream_t st)
{
    k_expand<<<grid_for(nfull), NT, 0, st>>>(blk, nfull, s, n, b, nst, scale, add1, full);
    return cudaGetLastError();
}

cudaError_t launch_contract(const double* G, const double* V, int64_t nx, int64_t ny, double alpha,
                            double* out, cudaStream_t st)
{
    k_contract<<<grid_for(nx * 32), NT, 0, st>>>(G, V, nx, ny, alpha, out);
    return cudaGetLastError();
}

cudaError_t launch_seed(const double* C, double two_w, int64_t nfull, double* G, double* GM, cudaStream_t st)
{
    k_seed<<<grid_for(nfull), NT, 0, st>>>(C, two_w, nfull, G, GM);
    return cudaGetLastError();
}

cudaError_t launch_compact(const double* GM, int s, int n, const uint64_t* uvars, const float* umult, int nu,
                           double coef, float* Gc, cudaStream_t st)
{
    k_compact<<<grid_for((int64_t)nu * n), NT, 0, st>>>(GM, s, n, uvars, umult, nu, coef, Gc);
    return cudaGetLastError();
}

cudaError_t launch_grad_x(const float* ring, int64_t T, const int64_t* head, int n, int npad, const float* shift,
                          const uint64_t* uvars, const uint8_t* unf, int nu, const float* Gc, float* dX,
                          cudaStream_t st)
{
    const size_t smem = sizeof(float) * ((size_t)AT * npad + AT * AU + (size_t)AU * n);
    cudaError_t e = smem_opt_in((const void*)k_grad_x, sizeof(float) * (AT * kMaxN + AT * AU + AU * kMaxN));
    if (e != cudaSuccess) return e;
    k_grad_x<<<(int)((T + AT - 1) / AT), NT, smem, st>>>(ring, T, head, n, npad, shift, uvars, unf, nu, Gc, dX);
    return cudaGetLastError();
}

}  // namespace cw
