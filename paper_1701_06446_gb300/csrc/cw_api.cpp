// C ABI of the sliding-window cumulant library: handle state, table upload,
// and the sequence of kernels of one window shift (Algorithm 1).
#include "../../include/cumwin.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cw_internal.h"
#include "cw_layout.h"
#include "cw_tc.h"

using namespace cw;

namespace {

thread_local std::string g_last_error;

int fail_cuda(cudaError_t e, const char* what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? CUMWIN_ENOMEM : CUMWIN_ECUDA;
}

#define CW_TRY(expr)                                    \
    do {                                                \
        cudaError_t _e = (expr);                        \
        if (_e != cudaSuccess) return fail_cuda(_e, #expr); \
    } while (0)

}  // namespace

void cw::set_last_error(const std::string& msg) { g_last_error = msg; }

struct cumwin_s {
    int n = 0, d = 0, b = 0, nbar = 0, npad = 0, prec = 0;
    int64_t T = 0;
    int p = 1;  // nominal shift size (batch of the mixed-form FP32 sums)
    cudaStream_t stream = nullptr;
    int device = 0, sm_count = 0;
    int64_t* head = nullptr;  // device: ring slot of the oldest sample
    bool filled = false;
    std::vector<void*> allocs;

    float* ring = nullptr;      // [T][npad] raw samples
    float* stage = nullptr;     // [2T][npad] X_(+) then X_(-)
    float* hin = nullptr;       // [T][npad] device copy of host X_(+)
    float* shift = nullptr;     // [npad]
    float* shift_zero = nullptr;
    int* status = nullptr;
    double* S[kMaxOrder + 1] = {};
    double* C[kMaxOrder + 1] = {};
    int64_t E[kMaxOrder + 1] = {};
    int64_t Eoff[kMaxOrder + 2] = {};  // offsets of the orders in one concatenated index space

    UpdateArgs upd{};
    UpdTile* tiles = nullptr;
    int ntiles = 0;
    TcPlan tc{};  // tensor-core update plan (mixed forms)

    CumArgs cum[kMaxOrder + 1]{};
    CumLaunch cum_launch[kMaxOrder + 1] = {};
    double* normpart = nullptr;
    int32_t* part_off = nullptr;
    double* fro2 = nullptr;

    // adjoint workspace (allocated by the first cumwin_grad)
    struct Grad {
        bool ready = false;
        double* Cf[kMaxOrder + 1] = {};   // full C_s (order 1 about the shift)
        double* C1true = nullptr;         // full C_1 + shift
        double* Mf[kMaxOrder + 1] = {};   // full M_s, s < d
        double* G[kMaxOrder + 1] = {};    // adjoint of C_s
        double* GM[kMaxOrder + 1] = {};   // adjoint of M_s
        int64_t nf[kMaxOrder + 1] = {};   // n^s
        int64_t* nst = nullptr;
        uint32_t* uvars = nullptr;        // sorted (s-1)-tuples of all orders, concatenated
        float* umult = nullptr;
        uint8_t* unf = nullptr;
        int uoff[kMaxOrder + 2] = {};
        float* Gc = nullptr;              // [nu][n]
    } grad;

    // kernel timing (cumwin_set_timing)
    bool timing = false;
    std::vector<cudaEvent_t> ev;  // 4 per timed shift: start, staged, updated, recovered
    int64_t timed = 0, launches = 0;

    template <class T>
    cudaError_t alloc(T** p, size_t count)
    {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
        if (e != cudaSuccess) return e;
        allocs.push_back(q);
        *p = (T*)q;
        return cudaSuccess;
    }
    template <class T>
    cudaError_t upload(T** p, const std::vector<T>& v)
    {
        cudaError_t e = alloc(p, v.size());
        if (e != cudaSuccess) return e;
        if (!v.empty()) e = cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
        return e;
    }
    void release()
    {
        for (void* q : allocs) cudaFree(q);
        allocs.clear();
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        ev.clear();
    }
    // event slot k of the current timed shift, or null when not timing
    cudaEvent_t mark(int k)
    {
        if (!timing || timed * 4 + k >= (int64_t)ev.size()) return nullptr;
        cudaEvent_t e = ev[timed * 4 + k];
        cudaEventRecord(e, stream);
        return e;
    }
};

namespace {

// Recovery of C_1..C_d and norms.  accum: fold the tensor-core workspace of
// the shift into the sums first (mixed forms, after a push).
int run_cumulants(cumwin_t h, int64_t advance, bool accum = false)
{
    for (int s = 1; s <= h->d; ++s) {
        CumArgs a = h->cum[s];
        a.accum = accum ? 1 : 0;
        CW_TRY(launch_cumulants(a, h->cum_launch[s], h->stream));
    }
    CW_TRY(launch_norm_final(h->normpart, h->part_off, h->d, h->fro2, h->head, advance, h->T,
                             h->stream));
    h->launches += h->d + 1;
    if (h->mark(3) != nullptr) h->timed++;
    return CUMWIN_OK;
}

// Moment sums of the whole window held in the ring buffer (fill, recompute).
int update_window(cumwin_t h)
{
    h->mark(0);
    h->mark(1);
    if (h->prec == CUMWIN_FP64) {
        CW_TRY(launch_update_f64(h->upd, h->tiles, h->ntiles, h->ring, h->T, h->T, h->shift,
                                 h->stream));
        h->launches += 1;
    } else {
        TcAccArgs acc{};
        for (int s = 1; s <= h->d; ++s) acc.S[s] = h->S[s];
        for (int s = 0; s <= h->d + 1; ++s) acc.Eoff[s] = h->Eoff[s];
        acc.d = h->d;
        for (int q = 0; q < h->tc.nbatch; ++q) {
            CW_TRY(tc_update_window_batch(h->tc, h->ring, h->head, q, h->n, h->shift, h->stream));
            CW_TRY(launch_tc_accumulate(h->tc, acc, h->stream));
        }
        h->launches += (int64_t)kTcBatchLaunches * h->tc.nbatch;
    }
    h->mark(2);
    return CUMWIN_OK;
}

// One shift: stage X_(+) / X_(-), move X_(+) into the ring, update the sums.
int update_push(cumwin_t h, const float* x_in, const float* x_out, int p, int64_t ld)
{
    h->mark(0);
    if (h->prec == CUMWIN_FP64) {
        CW_TRY(launch_stage(x_in, ld, x_out, ld, h->ring, h->T, h->head, p, h->n, h->npad,
                            h->stage, h->status, h->stream));
        h->mark(1);
        CW_TRY(launch_update_f64(h->upd, h->tiles, h->ntiles, h->stage, 2 * (int64_t)p, p,
                                 h->shift, h->stream));
        h->launches += 2;
    } else {
        CW_TRY(tc_stage_push(h->tc, x_in, ld, x_out, ld, h->ring, h->head, p, h->n, h->shift,
                             h->stream));
        h->mark(1);
        CW_TRY(tc_gemm_push(h->tc, h->stream));
        h->launches += 3;
    }
    h->mark(2);
    return CUMWIN_OK;
}

int zero_sums(cumwin_t h)
{
    for (int s = 1; s <= h->d; ++s) CW_TRY(launch_zero(h->S[s], h->E[s], h->stream));
    return CUMWIN_OK;
}

int64_t element_index_impl(int n, int b, int order, const int* i)
{
    if (n < 1 || b < 1 || order < 1 || order > kMaxOrder || i == nullptr) return -1;
    int v[kMaxOrder], j[kMaxOrder];
    for (int k = 0; k < order; ++k) {
        if (i[k] < 0 || i[k] >= n) return -1;
        v[k] = i[k];
    }
    std::sort(v, v + order);
    for (int k = 0; k < order; ++k) j[k] = v[k] / b;
    const int nbar = (n + b - 1) / b;
    int64_t off = 0;
    for (int k = 0; k < order; ++k) off = off * b + v[k] % b;
    return rank_sorted(j, order, nbar) * ipow(b, order) + off;
}

}  // namespace

extern "C" {

int cumwin_version(void) { return 100; }

const char* cumwin_strerror(int code)
{
    switch (code) {
    case CUMWIN_OK: return "ok";
    case CUMWIN_EINVAL: return "invalid argument";
    case CUMWIN_ENOMEM: return "device allocation failed";
    case CUMWIN_ECUDA: return "CUDA runtime error";
    case CUMWIN_ESTATE: return "call out of sequence";
    case CUMWIN_ENONFINITE: return "non-finite sample in the window";
    case CUMWIN_ETIMEOUT: return "bounded device wait timed out";
    case CUMWIN_ENOTSUP: return "not supported on this device or build";
    default: return "unknown error";
    }
}

const char* cumwin_last_error(void) { return g_last_error.c_str(); }

int64_t cumwin_layout_size(int n, int b, int order)
{
    if (n < 1 || b < 1 || order < 1 || order > kMaxOrder) return -1;
    const int nbar = (n + b - 1) / b;
    return n_sorted(nbar, order) * ipow(b, order);
}

int64_t cumwin_block_rank(int n, int b, int order, const int* j)
{
    if (n < 1 || b < 1 || order < 1 || order > kMaxOrder || j == nullptr) return -1;
    return rank_sorted(j, order, (n + b - 1) / b);
}

int64_t cumwin_element_index(int n, int b, int order, const int* i)
{
    return element_index_impl(n, b, order, i);
}

int cumwin_selftest_tables(int n, int b, int s)
{
    if (n < 1 || n > kMaxN || b < 1 || s < 1 || s > kMaxOrder) return CUMWIN_EINVAL;
    const int nbar = (n + b - 1) / b;
    const int64_t E = n_sorted(nbar, s) * ipow(b, s);
    if (E > (int64_t)1 << 26) return CUMWIN_EINVAL;
    const int64_t bs = ipow(b, s);
    // 1. update tables: every stored element produced exactly once, at the
    //    storage index of its (row vars ++ col vars) multi-index.
    UpdateTables t = build_update_tables(n, b, s);
    std::vector<int> hits(E, 0);
    const int ncols = (int)t.colvar.size();
    for (int m = 0; m < nbar; ++m) {
        for (int r = t.rowstart[m]; r < t.rowstart[m + 1]; ++r) {
            for (int c = t.colstart[m]; c < ncols; ++c) {
                int vars[kMaxOrder], jj[kMaxOrder];
                for (int k = 0; k < t.h; ++k) vars[k] = (t.rowvar[r] >> (8 * k)) & 0xff;
                for (int k = 0; k < t.sh; ++k) vars[t.h + k] = (t.colvar[c] >> (8 * k)) & 0xff;
                for (int k = 0; k < s; ++k) jj[k] = vars[k] / b;
                const int64_t rk = rank_sorted(jj, s, nbar);
                if (rk < 0) return 1;  // not a sorted block
                int64_t off = 0;
                for (int k = 0; k < s; ++k) off = off * b + vars[k] % b;
                const int64_t want = rk * bs + off;
                const int64_t got = t.rowoff[r] + t.coloff[c];
                if (got != want || got < 0 || got >= E) return 2;
                hits[got]++;
            }
        }
    }
    for (int64_t e = 0; e < E; ++e)
        if (hits[e] != 1) return 3;
    // 2. cumulant tables: sub-block lookups of a synthetic symmetric tensor
    //    f(i) = prod_k (i_k + 1.5) return f of the sub-multi-index.
    if (s >= 2) {
        CumTables ct = build_cum_tables(n, b, s);
        const std::vector<int> blocks = enumerate_sorted(nbar, s);
        const int64_t nb = (int64_t)blocks.size() / s;
        for (int64_t q = 0; q < nb; ++q) {
            const int* j = &blocks[q * s];
            for (int64_t o = 0; o < bs; ++o) {
                int dig[kMaxOrder];
                int64_t rem = o;
                for (int k = s - 1; k >= 0; --k) {
                    dig[k] = (int)(rem % b);
                    rem /= b;
                }
                for (int u = 0; u < ct.nsub; ++u) {
                    const unsigned mask = ct.masks[u];
                    int la = 0, lr = 0;
                    int64_t offA = 0, offR = 0;
                    int va[kMaxOrder], vr[kMaxOrder];
                    for (int k = 0; k < s; ++k) {
                        const int var = j[k] * b + dig[k];
                        if ((mask >> k) & 1u) {
                            offA = offA * b + dig[k];
                            va[la++] = var;
                        } else {
                            offR = offR * b + dig[k];
                            vr[lr++] = var;
                        }
                    }
                    const int64_t ia = (int64_t)ct.subrank[(q * ct.nsub + u) * 2] * ipow(b, la) + offA;
                    const int64_t ir = (int64_t)ct.subrank[(q * ct.nsub + u) * 2 + 1] * ipow(b, lr) + offR;
                    // the storage index of the sub-tuple in its own order must hold
                    // the same multiset of variables
                    int padA = 0, padR = 0;
                    for (int k = 0; k < la; ++k) padA |= va[k] >= n;
                    for (int k = 0; k < lr; ++k) padR |= vr[k] >= n;
                    if (!padA && element_index_impl(n, b, la, va) >= 0) {
                        // same block & offset as canonical storage up to the in-block
                        // permutation: compare the decoded multiset
                        int64_t rk = ia / ipow(b, la), of = ia % ipow(b, la);
                        std::vector<int> jb = enumerate_sorted(nbar, la);
                        int dec[kMaxOrder];
                        int64_t rr = of;
                        for (int k = la - 1; k >= 0; --k) {
                            dec[k] = jb[rk * la + k] * b + (int)(rr % b);
                            rr /= b;
                        }
                        std::sort(dec, dec + la);
                        std::sort(va, va + la);
                        for (int k = 0; k < la; ++k)
                            if (dec[k] != va[k]) return 4;
                    }
                    if (!padR) {
                        int64_t rk = ir / ipow(b, lr), of = ir % ipow(b, lr);
                        std::vector<int> jb = enumerate_sorted(nbar, lr);
                        int dec[kMaxOrder];
                        int64_t rr = of;
                        for (int k = lr - 1; k >= 0; --k) {
                            dec[k] = jb[rk * lr + k] * b + (int)(rr % b);
                            rr /= b;
                        }
                        std::sort(dec, dec + lr);
                        std::sort(vr, vr + lr);
                        for (int k = 0; k < lr; ++k)
                            if (dec[k] != vr[k]) return 5;
                    }
                }
            }
        }
    }
    return 0;
}

int cumwin_create(int n, int d, int b, int64_t T, int p, int precision, void* cuda_stream,
                  cumwin_t* out)
{
    if (out == nullptr) return CUMWIN_EINVAL;
    *out = nullptr;
    if (n < 1 || n > kMaxN || d < 1 || d > kMaxOrder || b < 1 || T < 1) return CUMWIN_EINVAL;
    if (p < 1 || p > T) return CUMWIN_EINVAL;
    if (precision != CUMWIN_FP64 && precision != CUMWIN_MIXED_BF16 && precision != CUMWIN_MIXED_FP16)
        return CUMWIN_EINVAL;
    const int nbar = (n + b - 1) / b;
    if ((int64_t)nbar * b > kMaxN) return CUMWIN_EINVAL;
    if (T > ((int64_t)1 << 40)) return CUMWIN_EINVAL;

    cumwin_s* h = new cumwin_s();
    h->n = n;
    h->d = d;
    h->b = b;
    h->nbar = nbar;
    h->npad = nbar * b;
    h->T = T;
    h->p = p;
    h->prec = precision;
    h->stream = (cudaStream_t)cuda_stream;

    auto bail = [&](int code) {
        h->release();
        delete h;
        return code;
    };
#define CW_CREATE_TRY(expr)                               \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) return bail(fail_cuda(_e, #expr)); \
    } while (0)

    CW_CREATE_TRY(cudaGetDevice(&h->device));
    CW_CREATE_TRY(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device));
    if (precision == CUMWIN_MIXED_FP16) {
        g_last_error = "the FP16 split form is not available in this build";
        return bail(CUMWIN_ENOTSUP);
    }
    if (precision != CUMWIN_FP64) {
        int major = 0, minor = 0;
        CW_CREATE_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->device));
        CW_CREATE_TRY(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, h->device));
        if (!(major == 10 && minor == 3)) {
            g_last_error = "mixed precision needs an sm_103 device";
            return bail(CUMWIN_ENOTSUP);
        }
    }
    const int npad = h->npad;
    CW_CREATE_TRY(h->alloc(&h->ring, (size_t)T * npad));
    CW_CREATE_TRY(h->alloc(&h->stage, (size_t)2 * T * npad));
    CW_CREATE_TRY(h->alloc(&h->hin, (size_t)T * npad));
    CW_CREATE_TRY(h->alloc(&h->shift, npad));
    CW_CREATE_TRY(cudaMemset(h->shift, 0, sizeof(float) * npad));
    CW_CREATE_TRY(h->alloc(&h->status, 1));
    CW_CREATE_TRY(h->alloc(&h->head, 1));
    CW_CREATE_TRY(cudaMemset(h->head, 0, sizeof(int64_t)));
    CW_CREATE_TRY(cudaMemset(h->status, 0, sizeof(int)));
    CW_CREATE_TRY(cudaMemset(h->ring, 0, sizeof(float) * (size_t)T * npad));
    for (int s = 1; s <= d; ++s) {
        h->E[s] = n_sorted(nbar, s) * ipow(b, s);
        if (h->E[s] >= ((int64_t)1 << 31)) {
            g_last_error = "a moment tensor of this size (2^31 stored elements or more) is not supported";
            return bail(CUMWIN_EINVAL);
        }
        CW_CREATE_TRY(h->alloc(&h->S[s], h->E[s]));
        CW_CREATE_TRY(h->alloc(&h->C[s], h->E[s]));
        CW_CREATE_TRY(cudaMemset(h->S[s], 0, sizeof(double) * h->E[s]));
        CW_CREATE_TRY(cudaMemset(h->C[s], 0, sizeof(double) * h->E[s]));
    }

    // update tables and tiles
    h->upd.npad = npad;
    std::vector<UpdTile> tiles;
    std::vector<UpdateTables> ut(d + 1);
    for (int s = 1; s <= d; ++s) {
        ut[s] = build_update_tables(n, b, s);
        const UpdateTables& t = ut[s];
        OrderTables& ot = h->upd.ord[s];
        CW_CREATE_TRY(h->upload((uint32_t**)&ot.rowvar, t.rowvar));
        CW_CREATE_TRY(h->upload((int64_t**)&ot.rowoff, t.rowoff));
        CW_CREATE_TRY(h->upload((uint32_t**)&ot.colvar, t.colvar));
        CW_CREATE_TRY(h->upload((int64_t**)&ot.coloff, t.coloff));
        ot.S = h->S[s];
        ot.h = t.h;
        ot.sh = t.sh;
        ot.nrows = (int32_t)t.rowvar.size();
        ot.ncols = (int32_t)t.colvar.size();
        for (int m = 0; m < nbar; ++m) {
            const int r0 = t.rowstart[m], r1 = t.rowstart[m + 1];
            const int c0 = t.colstart[m], c1 = ot.ncols;
            for (int r = r0; r < r1; r += 64)
                for (int c = c0; c < c1; c += 64) {
                    UpdTile u{};
                    u.s = s;
                    u.row0 = r;
                    u.nrows = std::min(64, r1 - r);
                    u.col0 = c;
                    u.ncols = std::min(64, c1 - c);
                    tiles.push_back(u);
                }
        }
    }
    h->ntiles = (int)tiles.size();
    h->Eoff[1] = 0;
    for (int s = 1; s <= d; ++s) h->Eoff[s + 1] = h->Eoff[s] + h->E[s];
    if (precision == CUMWIN_FP64) {
        CW_CREATE_TRY(h->upload(&h->tiles, tiles));
    } else {
        int rc = tc_plan_create(h->tc, ut, h->upd, h->Eoff, d, n, b, npad, T, p, h->sm_count,
                                precision,
                                h->status,
                                [&](size_t bytes, void** q) { return h->alloc((char**)q, bytes); });
        if (rc != 0) {
            g_last_error = "tensor-core plan: " + std::string(cudaGetErrorString((cudaError_t)rc));
            return bail(CUMWIN_ECUDA);
        }
    }

    // cumulant recovery tables
    std::vector<int32_t> part_off(d + 1, 0);
    for (int s = 1; s <= d; ++s) {
        CumTables ct = build_cum_tables(n, b, s);
        CumArgs& a = h->cum[s];
        for (int k = 1; k <= d; ++k) {
            a.S[k] = h->S[k];
            a.C[k] = h->C[k];
        }
        a.Cout = h->C[s];
        CW_CREATE_TRY(h->upload((int32_t**)&a.subrank, ct.subrank));
        CW_CREATE_TRY(h->upload((double**)&a.mult, ct.mult));
        a.shift = h->shift;
        a.W = h->tc.W;
        a.wslice = h->tc.wslice;
        a.woff = h->Eoff[s];
        a.ksplit = h->tc.ksplit;
        a.accum = 0;
        a.invT = 1.0 / (double)T;
        a.E = h->E[s];
        a.s = s;
        a.b = b;
        a.bs = (int32_t)ipow(b, s);
        a.nsub = ct.nsub;
        for (int u = 0; u < ct.nsub && u < 128; ++u) a.mask[u] = ct.masks[u];
        h->cum_launch[s] = plan_cumulants(s, (int)ipow(b, s), n_sorted(nbar, s), h->sm_count);
        part_off[s] = part_off[s - 1] + h->cum_launch[s].gx * h->cum_launch[s].gy;
    }
    // part_off[s-1]..part_off[s] are the partials of order s
    std::vector<int32_t> po(part_off.begin(), part_off.end());
    CW_CREATE_TRY(h->alloc(&h->normpart, (size_t)part_off[d]));
    for (int s = 1; s <= d; ++s) h->cum[s].normpart = h->normpart + part_off[s - 1];
    CW_CREATE_TRY(h->upload(&h->part_off, po));
    CW_CREATE_TRY(h->alloc(&h->fro2, d));
    CW_CREATE_TRY(cudaMemset(h->fro2, 0, sizeof(double) * d));
    CW_CREATE_TRY(cudaDeviceSynchronize());
#undef CW_CREATE_TRY
    *out = h;
    return CUMWIN_OK;
}

int cumwin_destroy(cumwin_t h)
{
    if (h == nullptr) return CUMWIN_OK;
    cudaStreamSynchronize(h->stream);
    h->release();
    delete h;
    return CUMWIN_OK;
}

int cumwin_set_stream(cumwin_t h, void* cuda_stream)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    h->stream = (cudaStream_t)cuda_stream;
    return CUMWIN_OK;
}

int cumwin_fill(cumwin_t h, const float* X_dev, int64_t ldx)
{
    if (h == nullptr || X_dev == nullptr || ldx < h->n) return CUMWIN_EINVAL;
    CW_TRY(launch_fill_ring(X_dev, ldx, h->ring, h->T, h->n, h->npad, h->status, h->stream));
    CW_TRY(cudaMemsetAsync(h->head, 0, sizeof(int64_t), h->stream));
    if (h->prec != CUMWIN_FP64)
        CW_TRY(launch_column_mean(h->ring, h->T, h->n, h->npad, h->shift, h->stream));
    int rc = zero_sums(h);
    if (rc) return rc;
    rc = update_window(h);
    if (rc) return rc;
    rc = run_cumulants(h, 0);
    if (rc) return rc;
    h->filled = true;
    return CUMWIN_OK;
}

int cumwin_push(cumwin_t h, const float* x_in_dev, const float* x_out_dev, int p, int64_t ld)
{
    if (h == nullptr || x_in_dev == nullptr || p < 1 || p > h->T || ld < h->n) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    if (h->prec != CUMWIN_FP64 && p > h->p) {
        g_last_error = "the mixed forms accept shifts of at most the nominal p given at create";
        return CUMWIN_EINVAL;
    }
    int rc = update_push(h, x_in_dev, x_out_dev, p, ld);
    if (rc) return rc;
    return run_cumulants(h, p, h->prec != CUMWIN_FP64);
}

int cumwin_push_host(cumwin_t h, const float* x_in_host, int p, int64_t ld)
{
    if (h == nullptr || x_in_host == nullptr || p < 1 || p > h->T || ld < h->n) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    CW_TRY(cudaMemcpy2DAsync(h->hin, sizeof(float) * h->npad, x_in_host, sizeof(float) * ld,
                             sizeof(float) * h->n, p, cudaMemcpyHostToDevice, h->stream));
    return cumwin_push(h, h->hin, nullptr, p, h->npad);
}

int cumwin_cumulants(cumwin_t h, int order, double* out_dev)
{
    if (h == nullptr || out_dev == nullptr || order < 1 || order > h->d) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    if (order == 1) {
        CW_TRY(launch_add_shift(h->C[1], h->shift, h->n, h->npad, out_dev, h->stream));
    } else {
        CW_TRY(cudaMemcpyAsync(out_dev, h->C[order], sizeof(double) * h->E[order],
                               cudaMemcpyDeviceToDevice, h->stream));
    }
    return CUMWIN_OK;
}

int cumwin_moments(cumwin_t h, int order, double* out_dev)
{
    if (h == nullptr || out_dev == nullptr || order < 1 || order > h->d) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    CW_TRY(launch_scale(h->S[order], 1.0 / (double)h->T, h->E[order], out_dev, h->stream));
    return CUMWIN_OK;
}

int cumwin_shift(cumwin_t h, float* shift_host)
{
    if (h == nullptr || shift_host == nullptr) return CUMWIN_EINVAL;
    CW_TRY(cudaMemcpyAsync(shift_host, h->shift, sizeof(float) * h->n, cudaMemcpyDeviceToHost,
                           h->stream));
    CW_TRY(cudaStreamSynchronize(h->stream));
    return CUMWIN_OK;
}

int cumwin_norms_device(cumwin_t h, double* fro2_dev)
{
    if (h == nullptr || fro2_dev == nullptr) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    CW_TRY(cudaMemcpyAsync(fro2_dev, h->fro2, sizeof(double) * h->d, cudaMemcpyDeviceToDevice,
                           h->stream));
    return CUMWIN_OK;
}

int cumwin_norms(cumwin_t h, double* fro_host, double* nu_host)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    double z[kMaxOrder];
    int st = 0;
    CW_TRY(cudaMemcpyAsync(z, h->fro2, sizeof(double) * h->d, cudaMemcpyDeviceToHost, h->stream));
    CW_TRY(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CW_TRY(cudaStreamSynchronize(h->stream));
    double fro[kMaxOrder];
    for (int s = 0; s < h->d; ++s) fro[s] = std::sqrt(z[s]);
    if (fro_host)
        for (int s = 0; s < h->d; ++s) fro_host[s] = fro[s];
    if (nu_host)
        for (int s = 1; s <= h->d; ++s)
            nu_host[s - 1] = (s < 3 || h->d < 2) ? NAN : fro[s - 1] / std::pow(fro[1], 0.5 * s);
    if (st & kStatusNonFinite) return CUMWIN_ENONFINITE;
    if (st & kStatusTimeout) return CUMWIN_ETIMEOUT;
    return CUMWIN_OK;
}

int cumwin_recompute(cumwin_t h)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    int rc = zero_sums(h);
    if (rc) return rc;
    rc = update_window(h);
    if (rc) return rc;
    return run_cumulants(h, 0);
}

int cumwin_window(cumwin_t h, float* out_dev)
{
    if (h == nullptr || out_dev == nullptr) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    CW_TRY(launch_window_copy(h->ring, h->T, h->head, h->n, h->npad, out_dev, h->stream));
    return CUMWIN_OK;
}

int cumwin_grad(cumwin_t h, const double* w_host, float* dX_dev)
{
    if (h == nullptr || w_host == nullptr || dX_dev == nullptr) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    const int n = h->n, d = h->d;
    auto& g = h->grad;
    if (!g.ready) {
        int64_t f = 1;
        for (int s = 1; s <= d; ++s) {
            f *= n;
            g.nf[s] = f;
        }
        if (g.nf[d] > ((int64_t)1 << 27)) {
            g_last_error = "the adjoint keeps full n^d tensors; n^d must be at most 2^27";
            return CUMWIN_ENOTSUP;
        }
        for (int s = 1; s <= d; ++s) {
            CW_TRY(h->alloc(&g.Cf[s], g.nf[s]));
            CW_TRY(h->alloc(&g.G[s], g.nf[s]));
            CW_TRY(h->alloc(&g.GM[s], g.nf[s]));
            if (s < d) CW_TRY(h->alloc(&g.Mf[s], g.nf[s]));
        }
        CW_TRY(h->alloc(&g.C1true, n));
        std::vector<int64_t> nst((size_t)(h->nbar + 1) * (kMaxOrder + 1));
        for (int v = 0; v <= h->nbar; ++v)
            for (int r = 0; r <= kMaxOrder; ++r) nst[v * (kMaxOrder + 1) + r] = n_sorted(h->nbar - v, r);
        CW_TRY(h->upload(&g.nst, nst));
        // sorted (s-1)-tuples of variables with their numbers of distinct orderings
        std::vector<uint32_t> uv;
        std::vector<float> um;
        std::vector<uint8_t> unf;
        for (int s = 1; s <= d; ++s) {
            g.uoff[s] = (int)uv.size();
            const int k = s - 1;
            if (k == 0) {
                uv.push_back(0u);
                um.push_back(1.0f);
                unf.push_back(0);
                continue;
            }
            const std::vector<int> tup = enumerate_sorted(n, k);
            for (size_t q = 0; q < tup.size() / k; ++q) {
                uint32_t p = 0;
                for (int i = 0; i < k; ++i) p |= (uint32_t)tup[q * k + i] << (8 * i);
                uv.push_back(p);
                um.push_back((float)block_multiplicity(&tup[q * k], k));
                unf.push_back((uint8_t)k);
            }
        }
        g.uoff[d + 1] = (int)uv.size();
        CW_TRY(h->upload(&g.uvars, uv));
        CW_TRY(h->upload(&g.umult, um));
        CW_TRY(h->upload(&g.unf, unf));
        CW_TRY(h->alloc(&g.Gc, (size_t)uv.size() * n));
        g.ready = true;
    }
    const double invT = 1.0 / (double)h->T;
    cudaStream_t st = h->stream;
    // full tensors of the current window
    for (int s = 1; s <= d; ++s) {
        CW_TRY(launch_expand(h->C[s], g.nf[s], s, n, h->b, g.nst, 1.0, nullptr, g.Cf[s], st));
        if (s < d) CW_TRY(launch_expand(h->S[s], g.nf[s], s, n, h->b, g.nst, invT, nullptr, g.Mf[s], st));
        CW_TRY(cudaMemsetAsync(g.G[s], 0, sizeof(double) * g.nf[s], st));
        CW_TRY(cudaMemsetAsync(g.GM[s], 0, sizeof(double) * g.nf[s], st));
    }
    CW_TRY(launch_expand(h->C[1], n, 1, n, h->b, g.nst, 1.0, h->shift, g.C1true, st));
    // reverse of the subset recursion, highest order first
    for (int s = d; s >= 2; --s) {
        CW_TRY(launch_seed(g.Cf[s], 2.0 * w_host[s], g.nf[s], g.G[s], g.GM[s], st));
        for (int k = 1; k < s; ++k) {
            const int r = s - k;
            const double coef = (double)binom(s - 1, k - 1);
            CW_TRY(launch_contract(g.G[s], g.Mf[r], g.nf[k], g.nf[r], -coef, g.G[k], st));
            CW_TRY(launch_contract(g.G[s], g.Cf[k], g.nf[r], g.nf[k], -coef, g.GM[r], st));
        }
    }
    CW_TRY(launch_seed(g.C1true, 2.0 * w_host[1], n, g.G[1], g.GM[1], st));
    // dL/dX = sum_s (s/T) sum_u mult(u) GM_s[a, u] prod y_{t,u}
    for (int s = 1; s <= d; ++s)
        CW_TRY(launch_compact(g.GM[s], s, n, g.uvars + g.uoff[s], g.umult + g.uoff[s],
                              g.uoff[s + 1] - g.uoff[s], (double)s * invT,
                              g.Gc + (size_t)g.uoff[s] * n, st));
    CW_TRY(launch_grad_x(h->ring, h->T, h->head, n, h->npad, h->shift, g.uvars, g.unf, g.uoff[d + 1], g.Gc,
                         dX_dev, st));
    return CUMWIN_OK;
}

int cumwin_set_timing(cumwin_t h, int enable)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    h->timing = enable != 0;
    h->timed = 0;
    h->launches = 0;
    if (h->timing && h->ev.empty()) {
        h->ev.resize(4 * 65536);
        for (auto& e : h->ev) CW_TRY(cudaEventCreate(&e));
    }
    return CUMWIN_OK;
}

int cumwin_get_timing(cumwin_t h, double* stage_ms, double* update_ms, double* cumulant_ms,
                      int64_t* shifts, int64_t* launches)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    CW_TRY(cudaStreamSynchronize(h->stream));
    double a = 0.0, u = 0.0, c = 0.0;
    for (int64_t k = 0; k < h->timed; ++k) {
        float t0 = 0.f, t1 = 0.f, t2 = 0.f;
        CW_TRY(cudaEventElapsedTime(&t0, h->ev[4 * k], h->ev[4 * k + 1]));
        CW_TRY(cudaEventElapsedTime(&t1, h->ev[4 * k + 1], h->ev[4 * k + 2]));
        CW_TRY(cudaEventElapsedTime(&t2, h->ev[4 * k + 2], h->ev[4 * k + 3]));
        a += t0;
        u += t1;
        c += t2;
    }
    if (stage_ms) *stage_ms = a;
    if (update_ms) *update_ms = u;
    if (cumulant_ms) *cumulant_ms = c;
    if (shifts) *shifts = h->timed;
    if (launches) *launches = h->launches;
    return CUMWIN_OK;
}

int cumwin_status(cumwin_t h)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    int st = 0;
    CW_TRY(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CW_TRY(cudaStreamSynchronize(h->stream));
    if (st & kStatusNonFinite) return CUMWIN_ENONFINITE;
    if (st & kStatusTimeout) return CUMWIN_ETIMEOUT;
    return CUMWIN_OK;
}

}  // extern "C"
