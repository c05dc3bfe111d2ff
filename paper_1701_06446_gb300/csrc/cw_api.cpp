// C ABI of the sliding-window cumulant library: window state, table upload,
// the sequence of kernels of one window shift (Algorithm 1), batches of
// independent windows, and the K-split autotuner.
#include "../../include/cumwin.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
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

#define CW_TRY(expr)                                        \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return fail_cuda(_e, #expr); \
    } while (0)

// The allocator handles take their device memory from (cumwin_set_allocator):
// the caller's callbacks, or cudaMallocAsync on the handle's stream (then
// synchronised, since the creating code touches the memory on other streams)
// and cudaFree.
struct Allocator {
    cumwin_alloc_fn alloc = nullptr;
    cumwin_free_fn free = nullptr;
    void* ctx = nullptr;
};
std::mutex g_alloc_mu;
Allocator g_alloc;

Allocator current_allocator()
{
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    return g_alloc;
}

// Device allocations of one object, all through its allocator, freed together.
struct Arena {
    struct Block {
        void* p;
        size_t bytes;
    };
    std::vector<Block> blocks;
    Allocator al;
    cudaStream_t stream = nullptr;
    size_t total = 0;
    cudaError_t raw(void** q, size_t bytes)
    {
        *q = nullptr;
        if (al.alloc != nullptr) {
            const int rc = al.alloc(al.ctx, bytes, (void*)stream, q);
            if (rc != 0 || *q == nullptr) return cudaErrorMemoryAllocation;
        } else {
            cudaError_t e = cudaMallocAsync(q, bytes, stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) return e;
        }
        blocks.push_back({*q, bytes});
        total += bytes;
        return cudaSuccess;
    }
    template <class T>
    cudaError_t alloc(T** p, size_t count)
    {
        void* q = nullptr;
        cudaError_t e = raw(&q, std::max<size_t>(count, 1) * sizeof(T));
        if (e != cudaSuccess) return e;
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
    template <class T>
    cudaError_t upload(T** p, const T* v, size_t count)
    {
        cudaError_t e = alloc(p, count);
        if (e != cudaSuccess) return e;
        return cudaMemcpy(*p, v, count * sizeof(T), cudaMemcpyHostToDevice);
    }
    void release()
    {
        for (const Block& b : blocks) {
            if (al.free != nullptr) al.free(al.ctx, b.p, b.bytes, (void*)stream);
            else cudaFree(b.p);
        }
        blocks.clear();
        total = 0;
    }
};

}  // namespace

void cw::set_last_error(const std::string& msg) { g_last_error = msg; }

constexpr int kKnormParts = 512;  // partial sums per order of cumwin_norms_k

// Fused recovery of orders 1..dfused (see FusedRecovery); dfused = 0 when the
// device cannot run the cooperative launch, and one launch per order is used.
struct FusedPlan {
    FusedRecovery f{};
    int dfused = 0, grid = 0;
    size_t smem = 0;
    int64_t emax[kMaxOrder + 1] = {};  // largest E_s over the windows
};

struct cumwin_s {
    int n = 0, d = 0, b = 0, nbar = 0, npad = 0, prec = 0;
    int shard = 0, nshards = 1;    // block shard of the top order (cumwin_create_shard)
    int64_t top0 = 0, top1 = -1;   // its lexicographic block range (top1 < 0: all)
    int64_t T = 0;
    int p = 1;  // nominal shift size (batch of the mixed-form FP32 sums)
    cudaStream_t stream = nullptr;
    int device = 0, sm_count = 0;
    int64_t* head = nullptr;      // device: ring slot of the oldest sample, as the staging sees it
    int64_t* head_rec = nullptr;  // device: the same, as the recovery sees it (FIFO slots); the two
                                  // advance once per shift each, in their own kernels
    bool filled = false;
    bool fifo_valid = false;  // the batch-sum FIFO matches the window
    double* fifo64 = nullptr; // FP64 form: [T / p][Eoff[d + 1]] batch sums (UpdateArgs), or null
    Arena mem;

    float* ring = nullptr;   // [T][npad] raw samples
    float* stage = nullptr;  // [2T][npad] X_(+) then X_(-) (FP64 form)
    float* hin[2] = {};      // [T][npad] device copies of host X_(+), used by alternate pushes
    int64_t* nst = nullptr;  // [nbar + 1][kMaxOrder + 1] sorted-tuple counts (full-tensor expansion)
    float* shift = nullptr;  // [npad]
    int* status = nullptr;
    double* S[kMaxOrder + 1] = {};
    double* C[kMaxOrder + 1] = {};
    float2* C2[kMaxOrder + 1] = {};  // two-word copies of the orders below d (mixed forms, d >= 4)
    float2* S2[kMaxOrder + 1] = {};
    int64_t E[kMaxOrder + 1] = {};
    int64_t Eoff[kMaxOrder + 2] = {};  // offsets of the orders in one concatenated index space

    // update tables (FP64 form tiles; tensor-core plan of this window or of its batch)
    std::vector<UpdateTables> ut;
    UpdateArgs upd{};
    UpdTile* tiles = nullptr;
    int ntiles = 0;
    TcPlan tc_own{};
    TcPlan* tc = nullptr;

    // recovery: host arguments per order, device copies
    // [workspace parity][kAccModes][order] (accumulate modes: no workspace /
    // stacked in-out workspace / FIFO)
    CumArgs cum[kMaxOrder + 1]{};
    CumArgs* cum_dev = nullptr;
    CumLaunch cum_launch[kMaxOrder + 1] = {};
    int canon_units[kMaxOrder + 1] = {};  // units of the canonical recovery of each order (0: not used)
    int canon_grid[kMaxOrder + 1] = {};   // its CTAs (CumArgs::unit_begin)
    FusedPlan fused;
    int parts = 0;  // norm partial slots per order
    double* normpart = nullptr;
    double* fro2 = nullptr;
    NormArgs* norm_dev = nullptr;
    TcAccSeg* segs = nullptr;  // workspace segments of this window's orders (own plan)
    int nsegs = 0;
    // scratch of cumwin_norms_k (kKnormParts partials per order) and of
    // cumwin_marginals (the storage indices of the diagonal entries i..i of
    // orders 2..min(d, 4) and the gathered values), allocated at create
    double* knorm_parts = nullptr;
    // drift of the mean from the shift (cumwin_set_auto_recenter): the last
    // measured ratio (device) and a flag the recovery raises in mapped host memory
    double* drift = nullptr;
    int* drift_host = nullptr;   // pinned, mapped
    int* drift_flag_dev = nullptr;
    double drift_limit = 0.0;    // 0: not measured
    int64_t recenters = 0;
    cudaEvent_t ev_drift[2] = {nullptr, nullptr};  // after the recoveries of the last two pushes
    int64_t pushes = 0;
    double* est = nullptr;  // [2d]: ||C_s|| and nu_s staged by cumwin_estimators_enqueue
    int64_t* diag_idx = nullptr;
    double* diag_val = nullptr;

    // adjoint workspace (allocated by the first cumwin_grad)
    struct Grad {
        bool ready = false;
        double* Cf[kMaxOrder + 1] = {};   // full C_s (order 1 about the shift)
        double* C1true = nullptr;         // full C_1 + shift
        double* Mf[kMaxOrder + 1] = {};   // full M_s, s < d
        double* Sblk = nullptr;           // M_s in the block layout, for orders whose sums are not (canonical)
        double* G[kMaxOrder + 1] = {};    // adjoint of C_s
        double* GM[kMaxOrder + 1] = {};   // adjoint of M_s
        int64_t nf[kMaxOrder + 1] = {};   // n^s
        int64_t* nst = nullptr;
        uint64_t* uvars = nullptr;        // sorted (s-1)-tuples of all orders, concatenated (8 bits a variable)
        float* umult = nullptr;
        uint8_t* unf = nullptr;
        int uoff[kMaxOrder + 2] = {};
        float* Gc = nullptr;              // [nu][n]
    } grad;

    // Pipelined shifts (mixed forms, single handles): the recovery of a shift
    // runs on `rstream`, so that the staging, operand build and GEMM of the
    // next shift (on the handle's stream) overlap it.  Shifts alternate
    // between two workspaces (parity); ev_rec[q] marks the end of the last
    // recovery that read workspace q, pend[q] that the handle's stream has
    // not waited for it yet.
    cudaStream_t rstream = nullptr;
    cudaEvent_t ev_gemm = nullptr;
    cudaEvent_t ev_rec[2] = {nullptr, nullptr};
    bool pend[2] = {false, false};
    int par = 0;
    int last = 0;          // workspace of the last pipelined push
    // cumwin_push_host: the host-to-device copy of a push runs on `cstream`
    // into one of two buffers, overlapping the previous pushes' kernels;
    // ev_h2d[q] marks the copy into buffer q, ev_staged[q] the push that last
    // read it
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_h2d[2] = {nullptr, nullptr};
    cudaEvent_t ev_staged[2] = {nullptr, nullptr};
    bool hin_pend[2] = {false, false};
    int hq = 0;
    bool pipeline = true;  // cumwin_set_pipeline

    // kernel timing (cumwin_set_timing)
    bool timing = false;
    bool coarse = false;          // no event between staging and update (cumwin_set_timing 2)
    std::vector<cudaEvent_t> ev;  // 4 per timed shift: start, staged, updated, recovered
    int64_t timed = 0, launches = 0;

    template <class T>
    cudaError_t alloc(T** p, size_t count) { return mem.alloc(p, count); }
    template <class T>
    cudaError_t upload(T** p, const std::vector<T>& v) { return mem.upload(p, v); }
    void release()
    {
        for (cudaStream_t* q : {&rstream, &cstream})
            if (*q != nullptr) {  // their work ends before the memory goes
                cudaStreamSynchronize(*q);
                cudaStreamDestroy(*q);
                *q = nullptr;
            }
        mem.release();
        if (drift_host != nullptr) {
            cudaFreeHost(drift_host);
            drift_host = nullptr;
        }
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        ev.clear();
        for (cudaEvent_t* e : {&ev_gemm, &ev_rec[0], &ev_rec[1], &ev_h2d[0], &ev_h2d[1], &ev_staged[0], &ev_staged[1],
                               &ev_drift[0], &ev_drift[1]})
            if (*e != nullptr) {
                cudaEventDestroy(*e);
                *e = nullptr;
            }
    }
    // event slot k of the current timed shift, or null when not timing
    cudaEvent_t mark(int k, cudaStream_t on = nullptr)
    {
        if (!timing || timed * 4 + k >= (int64_t)ev.size() || (coarse && k == 1)) return nullptr;
        cudaEvent_t e = ev[timed * 4 + k];
        cudaEventRecord(e, on != nullptr ? on : stream);
        return e;
    }
};

struct cumwin_batch_s {
    int nwin = 0, b = 0, p = 0, prec = 0, dmax = 0;
    bool fifo = false;  // regular pushes use the batch-sum FIFO
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    bool filled = false;
    std::vector<cumwin_s*> wins;
    std::vector<int64_t> xoff;  // packed push buffer offsets, [nwin + 1]
    Arena mem;
    TcPlan tc{};
    int* status = nullptr;
    CumArgs* cum_dev = nullptr;  // [kAccModes][kMaxOrder + 1][nwin]
    CumLaunch cum_launch[kMaxOrder + 1] = {};
    FusedPlan fused;
    NormArgs* norm_dev = nullptr;
    double* fro2 = nullptr;      // [nwin][dmax]
    TcAccSeg* segs = nullptr;
    int nsegs = 0;
    int64_t push_launches = 0;  // kernels the last cumwin_batch_push launched
    int shift_grid = 0;          // CTAs of the single-launch shift (0: the phases launch one by one)
    unsigned* shift_bar = nullptr;  // its grid barrier (a counter used by that grid size only)
    bool single = true;          // cumwin_batch_set_single_launch
};

namespace {

// ---------------------------------------------------------------------------
// tuning cache: one line per problem signature, "signature ksplit"
// ---------------------------------------------------------------------------
std::mutex g_tune_mu;

std::string tune_cache_path()
{
    const char* p = std::getenv("CUMWIN_TUNE_CACHE");
    return p ? std::string(p) : std::string();
}

// one line per problem signature: "signature ksplit nmax group" (the last line wins)
struct TileChoice {
    int ksplit = 0, nmax = 0, group = 0;
};

TileChoice tune_cache_get(const std::string& sig)
{
    TileChoice c;
    const std::string path = tune_cache_path();
    if (path.empty()) return c;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream in(line);
        std::string key;
        TileChoice t;
        if (in >> key >> t.ksplit >> t.nmax >> t.group && key == sig) c = t;
    }
    return c;
}

void tune_cache_put(const std::string& sig, const TcPlan& tc)
{
    const std::string path = tune_cache_path();
    if (path.empty()) return;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    std::ofstream f(path, std::ios::app);
    f << sig << ' ' << tc.ksplit << ' ' << tc.nmax << ' ' << tc.group << '\n';
}

// A cached choice, applied to a plan when it is valid for it.
void tune_cache_apply(TcPlan& tc, const TileChoice& c)
{
    if (c.nmax >= 16 && c.nmax <= kTcNmax && c.nmax % 16 == 0 && c.group >= 1 &&
        tc_plan_items(tc, c.nmax, c.group) == 0 && c.ksplit >= 1 && c.ksplit <= tc.ksplit_max)
        tc.ksplit = c.ksplit;
}

std::string plan_signature(const TcPlan& tc, const std::vector<cumwin_s*>& wins, int device)
{
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, device);
    std::ostringstream o;
    o << "cumwin2|" << prop.name << "|prec" << tc.precision << "|p" << tc.p << "|sets" << tc.rsets.size() << "|w";
    uint64_t hsh = 1469598103934665603ull;
    for (const cumwin_s* h : wins) {
        const uint64_t v = ((uint64_t)h->n << 40) ^ ((uint64_t)h->d << 32) ^ ((uint64_t)h->b << 24) ^ (uint64_t)h->T;
        hsh = (hsh ^ v) * 1099511628211ull;
    }
    o << wins.size() << ':' << std::hex << hsh;
    return o.str();
}

// ---------------------------------------------------------------------------
// one window: tables and device state
// ---------------------------------------------------------------------------
int64_t element_index_impl(int n, int b, int order, const int* i);

// Allocates and initialises everything a window needs.  own_tc: build the
// window's own tensor-core plan (mixed forms); batch members leave that to
// the batch.
int window_init(cumwin_s* h, int n, int d, int b, int64_t T, int p, int precision, cudaStream_t stream,
                bool own_tc)
{
    const int nbar = (n + b - 1) / b;
    h->n = n;
    h->d = d;
    h->b = b;
    h->nbar = nbar;
    h->npad = nbar * b;
    h->T = T;
    h->p = p;
    h->prec = precision;
    h->stream = stream;
    h->mem.al = current_allocator();
    h->mem.stream = stream;
    CW_TRY(cudaGetDevice(&h->device));
    CW_TRY(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device));
    if (precision != CUMWIN_FP64) {
        int major = 0, minor = 0;
        CW_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, h->device));
        CW_TRY(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, h->device));
        if (!(major == 10 && minor == 3)) {
            g_last_error = "mixed precision needs an sm_103 device";
            return CUMWIN_ENOTSUP;
        }
    }
    const int npad = h->npad;
    CW_TRY(h->alloc(&h->ring, (size_t)T * npad));
    if (precision == CUMWIN_FP64) CW_TRY(h->alloc(&h->stage, (size_t)2 * T * npad));
    {
        std::vector<int64_t> nst((size_t)(nbar + 1) * (kMaxOrder + 1));
        for (int v = 0; v <= nbar; ++v)
            for (int r = 0; r <= kMaxOrder; ++r) nst[v * (kMaxOrder + 1) + r] = n_sorted(nbar - v, r);
        CW_TRY(h->upload(&h->nst, nst));
    }
    CW_TRY(h->alloc(&h->hin[0], (size_t)T * npad));
    CW_TRY(h->alloc(&h->hin[1], (size_t)T * npad));
    CW_TRY(h->alloc(&h->shift, npad));
    CW_TRY(cudaMemset(h->shift, 0, sizeof(float) * npad));
    CW_TRY(h->alloc(&h->status, 1));
    CW_TRY(cudaMemset(h->status, 0, sizeof(int)));
    CW_TRY(h->alloc(&h->head, 1));
    CW_TRY(cudaMemset(h->head, 0, sizeof(int64_t)));
    CW_TRY(h->alloc(&h->head_rec, 1));
    CW_TRY(cudaMemset(h->head_rec, 0, sizeof(int64_t)));
    CW_TRY(cudaMemset(h->ring, 0, sizeof(float) * (size_t)T * npad));
    h->Eoff[1] = 0;
    for (int s = 1; s <= d; ++s) {
        h->E[s] = n_sorted(nbar, s) * ipow(b, s);
        if (h->E[s] >= ((int64_t)1 << 31)) {
            g_last_error = "a moment tensor of this size (2^31 stored elements or more) is not supported";
            return CUMWIN_EINVAL;
        }
        h->Eoff[s + 1] = h->Eoff[s] + (h->E[s] + 3) / 4 * 4;  // orders start on 16-byte boundaries
        CW_TRY(h->alloc(&h->S[s], h->E[s]));
        CW_TRY(h->alloc(&h->C[s], h->E[s]));
        CW_TRY(cudaMemset(h->S[s], 0, sizeof(double) * h->E[s]));
        CW_TRY(cudaMemset(h->C[s], 0, sizeof(double) * h->E[s]));
    }

    // update tables
    h->upd.npad = npad;
    h->ut.assign(d + 1, UpdateTables{});
    std::vector<UpdTile> tiles;
    // single windows: orders 5-6 with blocks of at least 256 elements compute one
    // element per class of equal entries (CanonTables); their update GEMMs then
    // produce only the rows and columns that canonical elements use, and their sums
    // exist only there (every sub-tuple of a canonical element is canonical in its
    // own block, so the recovery of the orders above reads no other element)
    auto canonical = [&](int s) {
        return own_tc && s >= kCanonMinOrder && s <= kCanonMaxOrder && ipow(b, s) >= kCanonMinBlock &&
               ipow(b, s - 1) <= 0xffff;
    };
    // compressed update tables: the order's sums exist at canonical elements only, which every
    // order above reads when it is canonical too; an order above without the canonical recovery
    // reads all of them (the FP64 sums in the FP64 form; the mixed forms read two-word copies,
    // which k_canon_expand fills in then)
    auto compressed = [&](int s) {
        if (!canonical(s)) return false;
        if (precision != CUMWIN_FP64) return true;
        for (int k = s + 1; k <= d; ++k)
            if (!canonical(k)) return false;
        return true;
    };
    for (int s = 1; s <= d; ++s) {
        h->ut[s] = build_update_tables(n, b, s, compressed(s));
        const UpdateTables& t = h->ut[s];
        OrderTables& ot = h->upd.ord[s];
        CW_TRY(h->upload((uint32_t**)&ot.rowvar, t.rowvar));
        CW_TRY(h->upload((int64_t**)&ot.rowoff, t.rowoff));
        CW_TRY(h->upload((uint32_t**)&ot.colvar, t.colvar));
        CW_TRY(h->upload((int64_t**)&ot.coloff, t.coloff));
        ot.S = h->S[s];
        ot.h = t.h;
        ot.sh = t.sh;
        ot.nrows = (int32_t)t.rowvar.size();
        ot.ncols = (int32_t)t.colvar.size();
        if (precision != CUMWIN_FP64) continue;
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
    if (precision == CUMWIN_FP64) CW_TRY(h->upload(&h->tiles, tiles));
    if (precision == CUMWIN_FP64 && T % p == 0 && T / p >= 1 && T / p <= INT32_MAX) {
        // FIFO of FP64 batch sums when the window is a whole number of batches and the
        // FIFO takes at most a quarter of the free device memory
        const int64_t slots = T / p, per = h->Eoff[d + 1];
        size_t free_b = 0, total_b = 0;
        CW_TRY(cudaMemGetInfo(&free_b, &total_b));
        if ((double)slots * (double)per * sizeof(double) <= (double)free_b / 4) {
            CW_TRY(h->alloc(&h->fifo64, (size_t)(slots * per)));
            h->upd.p = p;
            h->upd.nslots = (int32_t)slots;
            h->upd.fstride = per;
            h->upd.head = h->head;
            for (int s = 1; s <= d; ++s) h->upd.ord[s].F = h->fifo64 + h->Eoff[s];
        }
    }

    // cumulant recovery tables (norm partials and workspace pointers are set later)
    for (int k = 1; k < d; ++k)
        if (h->E[k] >= ((int64_t)1 << 32)) {  // the recovery indexes the lower orders in 32 bits
            g_last_error = "orders below d must hold fewer than 2^32 stored elements";
            return CUMWIN_ENOTSUP;
        }
    const bool twoword = precision != CUMWIN_FP64 && d >= kTwoWordMinOrder;
    if (twoword)
        for (int k = 1; k < d; ++k) {
            CW_TRY(h->alloc(&h->C2[k], (size_t)h->E[k]));
            CW_TRY(h->alloc(&h->S2[k], (size_t)h->E[k]));
        }
    for (int s = 1; s <= d; ++s) {
        CumTables ct = build_cum_tables(n, b, s);
        CumArgs& a = h->cum[s];
        for (int k = 1; k <= d; ++k) {
            a.S[k] = h->S[k];
            a.C[k] = h->C[k];
            a.C2[k] = h->C2[k];
            a.S2[k] = h->S2[k];
        }
        a.split = twoword && s < d;
        a.twoword = twoword && s >= kTwoWordMinOrder;
        a.Cout = h->C[s];
        CW_TRY(h->upload((int32_t**)&a.subrank, ct.subrank));
        CW_TRY(h->upload((double**)&a.mult, ct.mult));
        a.shift = h->shift;
        a.invT = 1.0 / (double)T;
        a.tpow2 = (T & (T - 1)) == 0 ? 1 + (int32_t)__builtin_ctzll((unsigned long long)T) : 0;
        a.E = h->E[s];
        a.s = s;
        a.b = b;
        a.bs = (int32_t)ipow(b, s);
        a.nsub = ct.nsub;
        for (int u = 0; u < ct.nsub && u < 128; ++u) a.mask[u] = ct.masks[u];
        a.W = nullptr;
        a.accum = 0;
        a.bR = (int32_t)ipow(b, s - split_rows(s));
        // the top order's sums follow the workspace order in the mixed forms,
        // so that folding a shift into them is one coalesced pass; so do the
        // canonical orders', which exist at canonical elements only (compressed
        // update tables) and are folded by their recovery
        a.sgemm = precision != CUMWIN_FP64 && (s == d || canonical(s));
        if (precision != CUMWIN_FP64) {
            int32_t* wb = nullptr;
            CW_TRY(h->upload(&wb, build_w_blocks(h->ut[s], n, b)));
            a.wblk = wb;
        }
        h->cum_launch[s] = plan_cumulants(s, (int)ipow(b, s), n_sorted(nbar, s), h->sm_count);
        if (canonical(s)) {
            const bool sh = s == d && h->top1 >= 0;  // a shard recovers its block range of the top order
            // units of up to kCanonGroup blocks, fewer when that leaves k_canon's CTAs under 8 units each
            // (finer units balance them better)
            const int grid = kCanonCtasPerSm * h->sm_count;
            int group = kCanonGroup;
            CanonTables cn = build_canon_tables(n, b, s, kCanonSlice, group, sh ? h->top0 : 0, sh ? h->top1 : -1);
            while (group > 1 && (int64_t)cn.units.size() / 4 < 8LL * grid) {
                group /= 2;
                cn = build_canon_tables(n, b, s, kCanonSlice, group, sh ? h->top0 : 0, sh ? h->top1 : -1);
            }
            CW_TRY(h->upload((int32_t**)&a.blkpat, cn.blkpat));
            CW_TRY(h->upload((int32_t**)&a.can_start, cn.can_start));
            CW_TRY(h->upload((int32_t**)&a.can_off, cn.can_off));
            CW_TRY(h->upload((int32_t**)&a.map_off, cn.map_off));
            CW_TRY(h->upload((int32_t**)&a.can_copies, cn.can_copies));
            if (a.sgemm) {
                CW_TRY(h->upload((int32_t**)&a.can_lr, cn.can_lr));
                CW_TRY(h->upload((int32_t**)&a.map_lr, cn.map_lr));
            }
            CW_TRY(h->upload((int32_t**)&a.dup_start, cn.dup_start));
            int32_t* dd = nullptr;
            CW_TRY(h->upload(&dd, cn.dup));
            a.dup = reinterpret_cast<const int2*>(dd);
            CW_TRY(h->upload((int32_t**)&a.pblocks, cn.pblocks));
            int32_t* du = nullptr;
            CW_TRY(h->upload(&du, cn.units));
            a.units = reinterpret_cast<const int4*>(du);
            a.nunits = (int32_t)(cn.units.size() / 4);
            a.npblocks = (int32_t)cn.pblocks.size();
            a.canon = 1;
            h->canon_grid[s] = std::max(1, std::min(a.nunits, grid));
            for (int k = s + 1; k <= d; ++k) a.split_copies |= canonical(k) ? 0 : 1;
            h->canon_units[s] = a.nunits;
        }
    }
    CW_TRY(h->alloc(&h->fro2, d));
    CW_TRY(cudaMemset(h->fro2, 0, sizeof(double) * d));
    CW_TRY(h->alloc(&h->knorm_parts, (size_t)kKnormParts * d));
    CW_TRY(h->alloc(&h->est, (size_t)2 * d));
    CW_TRY(h->alloc(&h->drift, 1));
    CW_TRY(cudaMemset(h->drift, 0xff, sizeof(double)));  // NaN until measured
    {
        const int dm = std::min(d, 4);
        std::vector<int64_t> idx((size_t)std::max(dm - 1, 1) * n, 0);
        for (int s = 2; s <= dm; ++s)
            for (int i = 0; i < n; ++i) {
                int v[kMaxOrder];
                for (int q = 0; q < s; ++q) v[q] = i;
                idx[(size_t)(s - 2) * n + i] = element_index_impl(n, b, s, v);
            }
        CW_TRY(h->upload(&h->diag_idx, idx));
        CW_TRY(h->alloc(&h->diag_val, idx.size()));
    }

    if (precision != CUMWIN_FP64 && own_tc) {
        TcPlanStream ps{};
        ps.tables = &h->ut;
        ps.upd = &h->upd;
        ps.Eoff = h->Eoff;
        ps.d = d;
        ps.n = n;
        ps.npad = npad;
        ps.T = T;
        ps.ring = h->ring;
        ps.head = h->head;
        ps.shift = h->shift;
        ps.status = h->status;
        ps.xoff = 0;
        ps.top0 = h->top0;
        ps.top1 = h->top1;
        int rc = tc_plan_create(h->tc_own, {ps}, b, p, h->sm_count, precision, h->status, true, true,
                                [&](size_t bytes, void** q) { return h->alloc((char**)q, bytes); });
        if (rc != 0) {
            g_last_error = "tensor-core plan: " + std::string(cudaGetErrorString((cudaError_t)rc));
            return rc == (int)cudaErrorMemoryAllocation ? CUMWIN_ENOMEM : CUMWIN_ECUDA;
        }
        h->tc = &h->tc_own;
    }
    return CUMWIN_OK;
}

// Norm partial slots and the device copies of the recovery arguments of a
// window: `parts` slots per order, stream `index` of plan `tc`.
int window_finish(cumwin_s* h, int parts, const TcPlan* tc, int index)
{
    h->parts = parts;
    CW_TRY(h->alloc(&h->normpart, (size_t)parts * h->d));
    CW_TRY(cudaMemset(h->normpart, 0, sizeof(double) * (size_t)parts * h->d));
    CumArgs arr[2][kAccModes][kMaxOrder + 1] = {};  // [workspace parity][accumulate mode][order]
    for (int s = 1; s <= h->d; ++s) {
        CumArgs& a = h->cum[s];
        a.normpart = h->normpart + (size_t)(s - 1) * parts;
        if (tc != nullptr) {
            a.W = tc->W;
            a.wslice = tc->wslice;
            a.woff = tc->wbase[index] + h->Eoff[s];
            a.ksplit = tc->ksplit;
            if (tc->fifo != nullptr) {
                a.fifo = tc->fifo + tc->fbase[index] + h->Eoff[s];
                a.fstride = h->Eoff[h->d + 1];
                a.head = h->head_rec;
                a.p = h->p;
            }
        }
        for (int q = 0; q < 2; ++q)
            for (int m = 0; m < kAccModes; ++m) {
                arr[q][m][s] = a;
                arr[q][m][s].accum = m;
                if (q == 1 && tc != nullptr && tc->W2 != nullptr) arr[q][m][s].W = tc->W2;
            }
    }
    CW_TRY(h->mem.upload(&h->cum_dev, &arr[0][0][0], 2 * kAccModes * (kMaxOrder + 1)));
    NormArgs na{};
    na.normpart = h->normpart;
    na.fro2 = h->fro2;
    na.head = h->head_rec;
    na.head_stage = h->prec == CUMWIN_FP64 ? h->head : nullptr;  // mixed forms: the build advances it
    na.T = h->T;
    na.parts = parts;
    na.d = h->d;
    na.C1 = h->C[1];
    na.C2 = h->d >= 2 ? h->C[2] : nullptr;
    na.drift = h->drift;
    na.drift_flag = nullptr;  // measured once cumwin_set_auto_recenter enables it
    na.n = h->n;
    na.b = h->b;
    na.nbar = h->nbar;
    CW_TRY(h->mem.upload(&h->norm_dev, &na, 1));
    return CUMWIN_OK;
}

// Work units of the fused recovery over the windows `wins` (shared b), the
// barrier state and the norm partials; leaves fp.dfused = 0 when the device
// cannot run it.  per_sm: CTAs per SM of its grid.  A single window takes 3,
// which leaves room on each SM for a CTA of the next shift's GEMM (pipelined
// shifts) and measured no slower than 4 alone; batches take 4.
int fused_setup(FusedPlan& fp, const std::vector<cumwin_s*>& wins, int b, int sm_count,
                const NormArgs* norm_dev, int* status, Arena& mem, int per_sm)
{
    int dmax = 0, device = 0, coop = 0;
    for (const cumwin_s* h : wins) {
        dmax = std::max(dmax, h->d);
        for (int s = 1; s <= h->d; ++s) fp.emax[s] = std::max(fp.emax[s], h->E[s]);
    }
    CW_TRY(cudaGetDevice(&device));
    CW_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
    fp.dfused = 0;
    if (!coop) return CUMWIN_OK;
    const int df = std::min(dmax, kFusedMax);
    const int nwin = (int)wins.size();
    FusedRecovery& f = fp.f;
    f.nwin = nwin;
    std::vector<int64_t> ustart((size_t)(kFusedMax + 1) * (nwin + 1), 0);
    int64_t utot = 0;
    for (int s = 1; s <= df; ++s) {
        int64_t nbmax = 0;
        for (const cumwin_s* h : wins)
            if (s <= h->d) nbmax = std::max<int64_t>(nbmax, n_sorted(h->nbar, s));
        const CumLaunch L = plan_cumulants(s, (int)ipow(b, s), nbmax, sm_count);
        f.slots[s] = L.slots;
        f.gy[s] = L.gy;
        f.upoff[s] = utot;
        int64_t* us = &ustart[(size_t)s * (nwin + 1)];
        for (int w = 0; w < nwin; ++w) {
            const cumwin_s* h = wins[w];
            const int64_t nb = s <= h->d ? n_sorted(h->nbar, s) : 0;
            us[w + 1] = us[w] + (nb + L.slots - 1) / L.slots * L.gy;
        }
        f.utot[s] = us[nwin];
        utot += us[nwin];
    }
    // fold segments: (window, order) with the order's stored elements
    std::vector<int64_t> abeg(1, 0);
    std::vector<int32_t> aarg;
    // the order-4 sums kept in workspace order (windows whose top order is 4)
    // are folded alongside orders 1-3 (vector pass); every other segment first
    for (int pass = 0; pass < 2; ++pass) {
        for (int w = 0; w < nwin; ++w)
            for (int s = 1; s <= std::min(df, wins[w]->d); ++s) {
                const bool late = s == 4 && wins[w]->cum[s].sgemm;
                if (late != (pass == 1)) continue;
                aarg.push_back(s * nwin + w);
                // order-4 segments start at multiples of four (vector fold)
                abeg.push_back(abeg.back() + (pass == 1 ? (wins[w]->E[s] + 3) / 4 * 4 : wins[w]->E[s]));
            }
        if (pass == 0) {
            f.nseg_lo = (int32_t)aarg.size();
            abeg.back() = (abeg.back() + 3) / 4 * 4;  // the order-4 range starts at a multiple of four
        }
    }
    f.nseg = (int32_t)aarg.size();
    fp.smem = fused_smem_bytes(f, df);
    fp.grid = fused_grid(df, fp.smem, sm_count, per_sm);
    if (fp.grid < 1) return CUMWIN_OK;
    int64_t* dus = nullptr;
    CW_TRY(mem.upload(&dus, ustart));
    f.ustart = dus;
    int64_t* dab = nullptr;
    int32_t* daa = nullptr;
    CW_TRY(mem.upload(&dab, abeg));
    CW_TRY(mem.upload(&daa, aarg));
    f.abeg = dab;
    f.aarg = daa;
    CW_TRY(mem.alloc(&f.upart, (size_t)std::max<int64_t>(utot, 1)));
    CW_TRY(mem.alloc(&f.bar, kBarrierWords));
    CW_TRY(cudaMemset(f.bar, 0, kBarrierWords * sizeof(unsigned)));
    f.norm = norm_dev;
    f.status = status;
    fp.dfused = df;
    return CUMWIN_OK;
}

// Recovery of orders 1..d and norms of the windows of `fp` / `cum_dev`
// ([mode][order][nwin]); accum: how the tensor-core workspace of the shift is
// folded into the sums first (CumArgs::accum; 0 = it is not).  Returns the
// number of launches through *launches.
int recover(const FusedPlan& fp, const CumArgs* cum_dev, const CumLaunch* cum_launch, const NormArgs* norm_dev,
            int nwin, int d, int64_t advance, int accum, int sm_count, cudaStream_t st, int64_t* launches,
            const int* canon_grid = nullptr)
{
    const CumArgs* args = cum_dev + (size_t)accum * (kMaxOrder + 1) * nwin;
    int s0 = 1;
    if (fp.dfused > 0) {
        FusedRecovery f = fp.f;
        f.args = args;
        f.advance = advance;
        f.advance_heads = d <= fp.dfused && advance != 0;
        f.fold = accum != 0;
        CW_TRY(launch_recover_fused(f, fp.dfused, fp.grid, fp.smem, st));
        *launches += 1;
        s0 = fp.dfused + 1;
    }
    for (int s = s0; s <= d; ++s) {
        if (s == kTwoWordMinOrder) {  // two-word copies of the lower orders for the orders from here on
            const int s_hi = kTwoWordMinOrder - 1;
            int64_t maxE = 1;
            for (int k = 1; k <= s_hi; ++k) maxE = std::max(maxE, fp.emax[k]);
            CW_TRY(launch_split(args, nwin, s_hi, maxE, sm_count, st));
            *launches += 1;
        }
        const bool canon = canon_grid != nullptr && canon_grid[s] > 0;
        // the top order (workspace order) is folded first; canonical orders (workspace
        // order too) are folded by k_canon at their canonical elements
        if (accum != 0 && !canon) {
            CW_TRY(launch_fold_linear(args + (size_t)s * nwin, nwin, fp.emax[s], sm_count, st));
            *launches += 1;
        }
        if (canon) {  // one window, canonical elements
            // grids within the order's norm partial slots (gx * gy of its launch shape)
            const int slots = cum_launch[s].gx * cum_launch[s].gy;
            CW_TRY(launch_canon(s, args + s, canon_grid[s], st));
            CW_TRY(launch_canon_expand(args + s, slots, st));
            *launches += 2;
        } else {
            CW_TRY(launch_cumulants(s, args + (size_t)s * nwin, nwin, cum_launch[s], st));
            *launches += 1;
        }
    }
    if (s0 <= d) {
        CW_TRY(launch_norm_final(norm_dev, nwin, advance, s0, st));
        *launches += 1;
    }
    return CUMWIN_OK;
}

int run_cumulants(cumwin_t h, int64_t advance, int accum = 0, int parity = 0, cudaStream_t on = nullptr)
{
    cudaStream_t st = on != nullptr ? on : h->stream;
    const int rc = recover(h->fused, h->cum_dev + (size_t)parity * kAccModes * (kMaxOrder + 1), h->cum_launch,
                           h->norm_dev, 1, h->d, advance, accum, h->sm_count, st, &h->launches, h->canon_grid);
    if (rc) return rc;
    if (h->mark(3, st) != nullptr) h->timed++;
    return CUMWIN_OK;
}

bool capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// The handle's stream waits for the recoveries still running on the
// recovery stream (no host synchronisation).  Under stream capture the wait
// becomes an external-event node of the graph and the recoveries stay
// pending for the eager work that follows the capture.
cudaError_t wait_recovery(cumwin_t h, int q)
{
    if (!h->pend[q]) return cudaSuccess;
    if (capturing(h->stream)) return cudaStreamWaitEvent(h->stream, h->ev_rec[q], cudaEventWaitExternal);
    const cudaError_t e = cudaStreamWaitEvent(h->stream, h->ev_rec[q], 0);
    if (e == cudaSuccess) h->pend[q] = false;
    return e;
}

cudaError_t join(cumwin_t h)
{
    for (int q = 0; q < 2; ++q) {
        const cudaError_t e = wait_recovery(h, q);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Shifts overlap the recovery of the previous one in the mixed forms, unless
// switched off, timed phase by phase, or captured into a graph.
bool pipelined(cumwin_t h)
{
    return h->pipeline && h->rstream != nullptr && !h->timing && !capturing(h->stream);
}

std::vector<TcAccSeg> acc_segments(const std::vector<cumwin_s*>& wins, const TcPlan& tc)
{
    std::vector<TcAccSeg> segs;
    for (size_t i = 0; i < wins.size(); ++i) {
        const cumwin_s* h = wins[i];
        for (int s = 1; s <= h->d; ++s) {
            TcAccSeg g{};
            g.S = h->S[s];
            g.wblk = h->cum[s].wblk;
            g.begin = tc.wbase[i] + h->Eoff[s];
            g.E = h->cum[s].sgemm ? h->ut[s].wsize : h->E[s];  // sums in workspace order: its slots
            g.bs = (int32_t)ipow(h->b, s);
            g.bR = h->cum[s].bR;
            g.head = h->head_rec;
            g.p = h->p;
            g.sgemm = h->cum[s].sgemm;
            if (tc.fifo != nullptr) {
                g.fifo = tc.fifo + tc.fbase[i] + h->Eoff[s];
                g.fstride = h->Eoff[h->d + 1];
                g.nslots = (int32_t)(h->T / h->p);
            }
            segs.push_back(g);
        }
    }
    return segs;
}

// Moment sums of the whole window held in the ring buffer (fill, recompute).
int update_window(cumwin_t h)
{
    h->mark(0);
    h->mark(1);
    if (h->prec == CUMWIN_FP64 && h->fifo64 != nullptr) {
        // batch by batch from the ring's head: each batch's sums enter S and its FIFO slot
        for (int q = 0; q < h->upd.nslots; ++q) {
            CW_TRY(launch_window_rows(h->ring, h->T, h->head, (int64_t)q * h->p, h->p, h->npad, h->stage,
                                      h->stream));
            CW_TRY(launch_update_f64(h->upd, h->tiles, h->ntiles, h->stage, h->p, h->p, h->shift,
                                     kUpdFifoStore, q, h->stream));
        }
        h->launches += 2LL * h->upd.nslots;
        h->fifo_valid = true;
    } else if (h->prec == CUMWIN_FP64) {
        CW_TRY(launch_update_f64(h->upd, h->tiles, h->ntiles, h->ring, h->T, h->T, h->shift,
                                 kUpdNoFifo, 0, h->stream));
        h->launches += 1;
    } else {
        for (int q = 0; q < h->tc->nbatch; ++q) {
            CW_TRY(tc_update_window_batch(*h->tc, q, h->stream));
            CW_TRY(launch_tc_accumulate(*h->tc, h->segs, h->nsegs, q, h->stream));
        }
        h->launches += 4LL * h->tc->nbatch;
        h->fifo_valid = h->tc->fifo != nullptr;
    }
    h->mark(2);
    return CUMWIN_OK;
}

// One shift: stage X_(+) / X_(-), move X_(+) into the ring, update the sums.
// *accum: how the recovery folds the shift's workspace in (CumArgs::accum).
// A shift of the nominal p with the leaving rows taken from the ring uses the
// batch-sum FIFO when there is one; any other shift recomputes the leaving
// half and retires the FIFO until the next fill or recompute.
int update_push(cumwin_t h, const float* x_in, const float* x_out, int p, int64_t ld, int* accum, int parity)
{
    *accum = 0;
    h->mark(0);
    if (h->prec == CUMWIN_FP64) {
        const bool fifo = h->fifo64 != nullptr && h->fifo_valid && x_out == nullptr && p == h->p;
        if (!fifo) h->fifo_valid = false;
        CW_TRY(launch_stage(x_in, ld, x_out, ld, h->ring, h->T, h->head, p, h->n, h->npad,
                            h->stage, h->status, h->stream));
        h->mark(1);
        // FIFO: only X_(+) is multiplied (the staged X_(-) rows are not read)
        CW_TRY(launch_update_f64(h->upd, h->tiles, h->ntiles, h->stage, fifo ? (int64_t)p : 2 * (int64_t)p, p,
                                 h->shift, fifo ? kUpdFifoShift : kUpdNoFifo, 0, h->stream));
    } else {
        const bool fifo = h->tc->fifo != nullptr && h->fifo_valid && x_out == nullptr && p == h->p;
        if (!fifo) h->fifo_valid = false;
        CW_TRY(tc_stage_push(*h->tc, x_in, x_out, ld, p, !fifo, h->stream));
        h->mark(1);
        CW_TRY(tc_gemm_push(*h->tc, !fifo, parity, h->stream));
        *accum = fifo ? 2 : 1;
    }
    h->launches += 2 + (h->prec != CUMWIN_FP64);
    h->mark(2);
    return CUMWIN_OK;
}

int zero_sums(cumwin_t h)
{
    for (int s = 1; s <= h->d; ++s) CW_TRY(launch_zero(h->S[s], h->E[s], h->stream));
    return CUMWIN_OK;
}

int fill_prepare(cumwin_t h, const float* X_dev, int64_t ldx)
{
    CW_TRY(launch_fill_ring(X_dev, ldx, h->ring, h->T, h->n, h->npad, h->status, h->stream));
    CW_TRY(cudaMemsetAsync(h->head, 0, sizeof(int64_t), h->stream));
    CW_TRY(cudaMemsetAsync(h->head_rec, 0, sizeof(int64_t), h->stream));
    if (h->prec != CUMWIN_FP64)
        CW_TRY(launch_column_mean(h->ring, h->T, h->n, h->npad, h->shift, h->stream));
    return zero_sums(h);
}

int check_args(int n, int d, int b, int64_t T, int p, int precision)
{
    if (n < 1 || n > kMaxN || d < 1 || d > kMaxOrder || b < 1 || T < 1) return CUMWIN_EINVAL;
    if (p < 1 || p > T) return CUMWIN_EINVAL;
    if (precision != CUMWIN_FP64 && precision != CUMWIN_MIXED_BF16 && precision != CUMWIN_MIXED_FP16)
        return CUMWIN_EINVAL;
    const int nbar = (n + b - 1) / b;
    if ((int64_t)nbar * b > kMaxN) return CUMWIN_EINVAL;
    if (T > ((int64_t)1 << 40)) return CUMWIN_EINVAL;
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

int cumwin_version(void) { return 110; }

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

static void nu_from_fro(const double* fro, int d, double* nu);

int cumwin_estimators_from_fro2(int d, const double* fro2_host, double* fro_host, double* nu_host)
{
    if (d < 1 || d > kMaxOrder || fro2_host == nullptr) return CUMWIN_EINVAL;
    double fro[kMaxOrder];
    for (int s = 0; s < d; ++s) fro[s] = std::sqrt(fro2_host[s]);
    if (fro_host)
        for (int s = 0; s < d; ++s) fro_host[s] = fro[s];
    if (nu_host) nu_from_fro(fro, d, nu_host);
    return CUMWIN_OK;
}

int cumwin_set_allocator(cumwin_alloc_fn alloc, cumwin_free_fn free_fn, void* ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return CUMWIN_EINVAL;
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.free = free_fn;
    g_alloc.ctx = alloc != nullptr ? ctx : nullptr;
    return CUMWIN_OK;
}

int64_t cumwin_device_bytes(cumwin_t h)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    return (int64_t)h->mem.total;
}

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
    std::vector<int> hits(E, 0), whits(E, 0);
    const std::vector<int64_t> roww = build_w_rows(t);
    const std::vector<int32_t> wblk = build_w_blocks(t, n, b);
    const int64_t bsh = ipow(b, t.sh);
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
                // workspace slot: the row form (epilogue) and the block form
                // (recovery) agree, and the slots cover [0, E) once
                const int64_t w = roww[r] + c;
                const int64_t wb = wblk[2 * rk] + (off / bsh) * wblk[2 * rk + 1] + off % bsh;
                if (w != wb || w < 0 || w >= E) return 6;
                whits[w]++;
            }
        }
    }
    for (int64_t e = 0; e < E; ++e)
        if (hits[e] != 1 || whits[e] != 1) return 3;
    // 2. canonical tables: the canonical offset of every stored element holds the
    //    same multiset of variables, is its own canonical offset, appears once in
    //    its pattern's list, and the units cover every (block, canonical element)
    //    of every pattern exactly once
    if (s >= 2 && E <= (int64_t)1 << 22) {
        const CanonTables cn = build_canon_tables(n, b, s, kCanonSlice, kCanonGroup);
        const std::vector<int> blocks = enumerate_sorted(nbar, s);
        const int64_t nb = (int64_t)blocks.size() / s;
        int64_t canon = 0;
        std::vector<int> seen(E, 0);
        for (size_t u = 0; u < cn.units.size(); u += 4) {
            const int q = cn.units[u], sl = cn.units[u + 1], g = cn.units[u + 2], cnt = cn.units[u + 3];
            const int c0 = cn.can_start[q] + sl * kCanonSlice;
            const int c1 = std::min(cn.can_start[q + 1], c0 + kCanonSlice);
            for (int k = 0; k < cnt; ++k) {
                const int blk = cn.pblocks[g + k];
                if (cn.blkpat[blk] != q) return 7;
                for (int c = c0; c < c1; ++c) seen[(int64_t)blk * bs + cn.can_off[c]]++;
            }
        }
        for (int64_t q = 0; q < nb; ++q) {
            const int* j = &blocks[q * s];
            const int pat = cn.blkpat[q];
            for (int64_t o = 0; o < bs; ++o) {
                const int64_t co = cn.map_off[(size_t)pat * bs + o];
                if (co < 0 || co >= bs || cn.map_off[(size_t)pat * bs + co] != co) return 8;
                int va[kMaxOrder], vb[kMaxOrder];
                int64_t ra = o, rb = co;
                for (int k = s - 1; k >= 0; --k) {
                    va[k] = j[k] * b + (int)(ra % b);
                    vb[k] = j[k] * b + (int)(rb % b);
                    ra /= b;
                    rb /= b;
                }
                std::sort(va, va + s);
                std::sort(vb, vb + s);
                for (int k = 0; k < s; ++k)
                    if (va[k] != vb[k]) return 9;
                const int64_t e = q * bs + o;
                if ((co == o) != (seen[e] == 1) || seen[e] > 1) return 10;
                canon += co == o;
            }
        }
        if (canon != cn.canonical) return 11;
        // 4. compressed update tables: the workspace slots are [0, wsize) once each,
        //    every canonical element is produced once, and at the slot its rank pair
        //    (can_lr, map_lr of every offset of its class) gives
        const UpdateTables tc = build_update_tables(n, b, s, true);
        const std::vector<int64_t> rowc = build_w_rows(tc);
        const std::vector<int32_t> wblc = build_w_blocks(tc, n, b);
        std::vector<int64_t> slot_of(E, -1);
        std::vector<int> chits(tc.wsize, 0);
        const int ncc = (int)tc.colvar.size();
        for (int m = 0; m < nbar; ++m)
            for (int r = tc.rowstart[m]; r < tc.rowstart[m + 1]; ++r)
                for (int c = tc.colstart[m]; c < ncc; ++c) {
                    int vars[kMaxOrder], jj[kMaxOrder];
                    for (int k = 0; k < tc.h; ++k) vars[k] = (tc.rowvar[r] >> (8 * k)) & 0xff;
                    for (int k = 0; k < tc.sh; ++k) vars[tc.h + k] = (tc.colvar[c] >> (8 * k)) & 0xff;
                    for (int k = 0; k < s; ++k) jj[k] = vars[k] / b;
                    const int64_t rk = rank_sorted(jj, s, nbar);
                    int64_t off = 0;
                    for (int k = 0; k < s; ++k) off = off * b + vars[k] % b;
                    const int64_t e = rk * bs + off, w = rowc[r] + c;
                    if (rk < 0 || tc.rowoff[r] + tc.coloff[c] != e || w < 0 || w >= tc.wsize) return 12;
                    if (slot_of[e] >= 0) return 13;
                    slot_of[e] = w;
                    chits[w]++;
                }
        for (int64_t w = 0; w < tc.wsize; ++w)
            if (chits[w] != 1) return 14;
        for (int64_t q = 0; q < nb; ++q) {
            const int pat = cn.blkpat[q];
            for (int64_t o = 0; o < bs; ++o) {
                const int64_t co = cn.map_off[(size_t)pat * bs + o];
                const int lr = cn.map_lr[(size_t)pat * bs + o];
                const int64_t w = wblc[2 * q] + (int64_t)((unsigned)lr >> 16) * wblc[2 * q + 1] + (lr & 0xffff);
                if (lr < 0 || slot_of[q * bs + co] != w) return 15;
            }
        }
        for (int q = 0; q < cn.npat; ++q)
            for (int c = cn.can_start[q]; c < cn.can_start[q + 1]; ++c)
                if (cn.can_lr[c] != cn.map_lr[(size_t)q * bs + cn.can_off[c]]) return 15;
    }
    // 3. cumulant tables: sub-block lookups of a synthetic symmetric tensor
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
    return cumwin_create_shard(n, d, b, T, p, precision, cuda_stream, 0, 1, out);
}

int cumwin_shard_blocks(int n, int b, int d, int shard, int nshards, int64_t* begin, int64_t* end)
{
    if (n < 1 || b < 1 || d < 1 || d > kMaxOrder || nshards < 1 || shard < 0 || shard >= nshards ||
        begin == nullptr || end == nullptr)
        return CUMWIN_EINVAL;
    shard_blocks((n + b - 1) / b, d, shard, nshards, begin, end);
    return CUMWIN_OK;
}

int cumwin_create_shard(int n, int d, int b, int64_t T, int p, int precision, void* cuda_stream, int shard,
                        int nshards, cumwin_t* out)
{
    if (out == nullptr) return CUMWIN_EINVAL;
    *out = nullptr;
    int rc = check_args(n, d, b, T, p, precision);
    if (rc) return rc;
    if (nshards < 1 || shard < 0 || shard >= nshards) return CUMWIN_EINVAL;
    if (nshards > 1 && (precision == CUMWIN_FP64 || d < kCanonMinOrder || d > kCanonMaxOrder ||
                        ipow(b, d) < kCanonMinBlock)) {
        g_last_error = "block shards need a mixed form and a top order of 5 or 6 with b^d >= 256";
        return CUMWIN_ENOTSUP;
    }
    cumwin_s* h = new cumwin_s();
    h->shard = shard;
    h->nshards = nshards;
    if (nshards > 1) shard_blocks((n + b - 1) / b, d, shard, nshards, &h->top0, &h->top1);
    rc = window_init(h, n, d, b, T, p, precision, (cudaStream_t)cuda_stream, true);
    int parts = 1;
    for (int s = 1; s <= d; ++s) {
        parts = std::max(parts, h->cum_launch[s].gx * h->cum_launch[s].gy);
        if (h->canon_units[s] > 0) parts = std::max(parts, kCanonCtasPerSm * h->sm_count);  // k_canon's grid
    }
    if (rc == CUMWIN_OK && h->tc != nullptr) {
        tune_cache_apply(*h->tc, tune_cache_get(plan_signature(*h->tc, {h}, h->device)));
    }
    if (rc == CUMWIN_OK) rc = window_finish(h, parts, h->tc, 0);
    if (rc == CUMWIN_OK) rc = fused_setup(h->fused, {h}, b, h->sm_count, h->norm_dev, h->status, h->mem, 3);
    if (rc == CUMWIN_OK) {  // the copy stream of cumwin_push_host
        cudaError_t e = cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking);
        for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
            e = cudaEventCreateWithFlags(&h->ev_h2d[q], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_staged[q], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) rc = fail_cuda(e, "create");
    }
    if (rc == CUMWIN_OK && h->tc != nullptr) {  // the recovery stream of pipelined shifts
        cudaError_t e = cudaStreamCreateWithFlags(&h->rstream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_gemm, cudaEventDisableTiming);
        for (int q = 0; q < 2 && e == cudaSuccess; ++q)
            e = cudaEventCreateWithFlags(&h->ev_rec[q], cudaEventDisableTiming);
        if (e != cudaSuccess) rc = fail_cuda(e, "create");
    }
    if (rc == CUMWIN_OK && h->tc != nullptr) {
        std::vector<TcAccSeg> segs = acc_segments({h}, *h->tc);
        h->nsegs = (int)segs.size();
        cudaError_t e = h->mem.upload(&h->segs, segs);
        if (e != cudaSuccess) rc = fail_cuda(e, "create");
    }
    if (rc == CUMWIN_OK) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = fail_cuda(e, "create");
    }
    if (rc != CUMWIN_OK) {
        h->release();
        delete h;
        return rc;
    }
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
    cudaStream_t next = (cudaStream_t)cuda_stream;
    if (next == h->stream) return CUMWIN_OK;
    // later work on the new stream follows everything issued so far on the old
    // one and the pending recoveries.  When either stream is under capture the
    // capturer orders the streams (a graph cannot wait on a temporary event).
    if (!capturing(h->stream) && !capturing(next)) {
        cudaEvent_t e = nullptr;
        CW_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        cudaError_t err = cudaEventRecord(e, h->stream);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(next, e, 0);
        cudaEventDestroy(e);  // released once the wait is resolved
        CW_TRY(err);
    }
    h->stream = next;
    h->mem.stream = next;
    CW_TRY(join(h));
    return CUMWIN_OK;
}

int cumwin_fill(cumwin_t h, const float* X_dev, int64_t ldx)
{
    if (h == nullptr || X_dev == nullptr || ldx < h->n) return CUMWIN_EINVAL;
    CW_TRY(join(h));
    int rc = fill_prepare(h, X_dev, ldx);
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
    const bool drift_on = h->drift_host != nullptr && h->drift_limit > 0.0 && !capturing(h->stream);
    if (drift_on) {
        // the flag of the recovery two pushes back is in place once its event completes: the
        // host runs at most two shifts ahead of the device while the policy is on
        if (h->pushes >= 2) CW_TRY(cudaEventSynchronize(h->ev_drift[h->pushes & 1]));
        if (*(volatile int*)h->drift_host != 0) {
            // a recovery found the mean drifted from the shift: re-centre before this shift
            // (after the pending recoveries, so that none of them raises the flag again)
            CW_TRY(join(h));
            if (h->rstream != nullptr) CW_TRY(cudaStreamSynchronize(h->rstream));
            CW_TRY(cudaStreamSynchronize(h->stream));
            *(volatile int*)h->drift_host = 0;
            const int rr = cumwin_recenter(h);
            if (rr) return rr;
            h->recenters++;
        }
    }
    int accum = 0;
    const bool pipe = pipelined(h);
    const int q = pipe ? h->par : 0;
    CW_TRY(wait_recovery(h, q));  // the recovery that last read workspace q
    int rc = update_push(h, x_in_dev, x_out_dev, p, ld, &accum, q);
    if (rc) return rc;
    if (!pipe) {
        CW_TRY(join(h));
        rc = run_cumulants(h, p, accum);
        if (rc == CUMWIN_OK && drift_on) {
            CW_TRY(cudaEventRecord(h->ev_drift[h->pushes & 1], h->stream));
            h->pushes++;
        }
        return rc;
    }
    // the recovery of this shift on the recovery stream, after its GEMM
    CW_TRY(cudaEventRecord(h->ev_gemm, h->stream));
    CW_TRY(cudaStreamWaitEvent(h->rstream, h->ev_gemm, 0));
    rc = run_cumulants(h, p, accum, q, h->rstream);
    if (rc) return rc;
    CW_TRY(cudaEventRecord(h->ev_rec[q], h->rstream));
    if (drift_on) {
        CW_TRY(cudaEventRecord(h->ev_drift[h->pushes & 1], h->rstream));
        h->pushes++;
    }
    h->pend[q] = true;
    h->last = q;
    h->par ^= 1;
    return CUMWIN_OK;
}

int cumwin_norms_enqueue(cumwin_t h, double* fro2_out, int* status_out)
{
    if (h == nullptr || (fro2_out == nullptr && status_out == nullptr)) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    // behind the last pipelined recovery on the recovery stream (and counted
    // in its event, so that cumwin_join covers the copies), else on the
    // handle's stream
    const bool behind = h->pend[h->last] && !capturing(h->stream);
    cudaStream_t st = behind ? h->rstream : h->stream;
    if (!behind) CW_TRY(join(h));
    if (fro2_out != nullptr)
        CW_TRY(cudaMemcpyAsync(fro2_out, h->fro2, sizeof(double) * h->d, cudaMemcpyDefault, st));
    if (status_out != nullptr)
        CW_TRY(cudaMemcpyAsync(status_out, h->status, sizeof(int), cudaMemcpyDefault, st));
    if (behind) CW_TRY(cudaEventRecord(h->ev_rec[h->last], h->rstream));
    return CUMWIN_OK;
}

int cumwin_estimators_enqueue(cumwin_t h, double* fro_out, double* nu_out, int* status_out)
{
    if (h == nullptr || (fro_out == nullptr && nu_out == nullptr && status_out == nullptr)) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    // as cumwin_norms_enqueue: behind the last pipelined recovery when there is one
    const bool behind = h->pend[h->last] && !capturing(h->stream);
    cudaStream_t st = behind ? h->rstream : h->stream;
    if (!behind) CW_TRY(join(h));
    if (fro_out != nullptr || nu_out != nullptr) {
        EstArgs a{};
        a.fro = h->est;
        a.nu = h->est + h->d;
        a.d = h->d;
        CW_TRY(launch_estimators(h->fro2, a, st));
        if (fro_out != nullptr)
            CW_TRY(cudaMemcpyAsync(fro_out, h->est, sizeof(double) * h->d, cudaMemcpyDefault, st));
        if (nu_out != nullptr)
            CW_TRY(cudaMemcpyAsync(nu_out, h->est + h->d, sizeof(double) * h->d, cudaMemcpyDefault, st));
    }
    if (status_out != nullptr)
        CW_TRY(cudaMemcpyAsync(status_out, h->status, sizeof(int), cudaMemcpyDefault, st));
    if (behind) CW_TRY(cudaEventRecord(h->ev_rec[h->last], h->rstream));
    return CUMWIN_OK;
}

int cumwin_loss(cumwin_t h, const double* w_host, double* L_dev)
{
    if (h == nullptr || w_host == nullptr || L_dev == nullptr) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    CW_TRY(join(h));
    EstArgs a{};
    a.loss = L_dev;
    a.d = h->d;
    for (int s = 1; s <= h->d; ++s) a.w[s] = w_host[s];
    CW_TRY(launch_estimators(h->fro2, a, h->stream));
    return CUMWIN_OK;
}

int cumwin_set_auto_recenter(cumwin_t h, double limit)
{
    if (h == nullptr || !(limit >= 0.0) || !std::isfinite(limit)) return CUMWIN_EINVAL;
    if (h->prec == CUMWIN_FP64) {
        g_last_error = "the FP64 form accumulates raw moments without a shift";
        return CUMWIN_ENOTSUP;
    }
    if (h->d < 2) return CUMWIN_EINVAL;
    CW_TRY(join(h));
    CW_TRY(cudaStreamSynchronize(h->stream));
    if (limit > 0.0 && h->drift_host == nullptr) {
        CW_TRY(cudaHostAlloc((void**)&h->drift_host, sizeof(int), cudaHostAllocMapped));
        CW_TRY(cudaHostGetDevicePointer((void**)&h->drift_flag_dev, h->drift_host, 0));
        for (cudaEvent_t& e : h->ev_drift) CW_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    h->pushes = 0;
    if (h->drift_host != nullptr) *(volatile int*)h->drift_host = 0;
    h->drift_limit = limit;
    NormArgs na{};
    CW_TRY(cudaMemcpy(&na, h->norm_dev, sizeof(NormArgs), cudaMemcpyDeviceToHost));
    na.drift_flag = limit > 0.0 ? h->drift_flag_dev : nullptr;
    na.drift_limit = limit;
    CW_TRY(cudaMemcpy(h->norm_dev, &na, sizeof(NormArgs), cudaMemcpyHostToDevice));
    return CUMWIN_OK;
}

int cumwin_drift(cumwin_t h, double* ratio_host, int64_t* recenters)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    CW_TRY(join(h));
    if (ratio_host != nullptr) {
        CW_TRY(cudaMemcpyAsync(ratio_host, h->drift, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CW_TRY(cudaStreamSynchronize(h->stream));
    }
    if (recenters != nullptr) *recenters = h->recenters;
    return CUMWIN_OK;
}

int cumwin_join(cumwin_t h)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    CW_TRY(join(h));
    return CUMWIN_OK;
}

int cumwin_set_pipeline(cumwin_t h, int enable)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    CW_TRY(join(h));
    h->pipeline = enable != 0;
    return CUMWIN_OK;
}

int cumwin_fifo(cumwin_t h)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    const bool has = h->fifo64 != nullptr || (h->tc != nullptr && h->tc->fifo != nullptr);
    return has && h->fifo_valid ? 1 : 0;
}

int cumwin_push_host(cumwin_t h, const float* x_in_host, int p, int64_t ld)
{
    if (h == nullptr || x_in_host == nullptr || p < 1 || p > h->T || ld < h->n) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    if (h->cstream == nullptr || capturing(h->stream)) {  // one stream: the copy, then the push
        CW_TRY(cudaMemcpy2DAsync(h->hin[0], sizeof(float) * h->npad, x_in_host, sizeof(float) * ld,
                                 sizeof(float) * h->n, p, cudaMemcpyHostToDevice, h->stream));
        return cumwin_push(h, h->hin[0], nullptr, p, h->npad);
    }
    // the copy into buffer q waits for the push that last read it and overlaps
    // the kernels of the pushes before; the push waits for the copy
    const int q = h->hq;
    if (h->hin_pend[q]) CW_TRY(cudaStreamWaitEvent(h->cstream, h->ev_staged[q], 0));
    CW_TRY(cudaMemcpy2DAsync(h->hin[q], sizeof(float) * h->npad, x_in_host, sizeof(float) * ld,
                             sizeof(float) * h->n, p, cudaMemcpyHostToDevice, h->cstream));
    CW_TRY(cudaEventRecord(h->ev_h2d[q], h->cstream));
    CW_TRY(cudaStreamWaitEvent(h->stream, h->ev_h2d[q], 0));
    const int rc = cumwin_push(h, h->hin[q], nullptr, p, h->npad);
    if (rc) return rc;
    CW_TRY(cudaEventRecord(h->ev_staged[q], h->stream));  // after the push's staging read the buffer
    h->hin_pend[q] = true;
    h->hq = q ^ 1;
    return CUMWIN_OK;
}

int cumwin_cumulants(cumwin_t h, int order, double* out_dev)
{
    if (h == nullptr || out_dev == nullptr || order < 1 || order > h->d) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    CW_TRY(join(h));
    if (order == 1) {
        CW_TRY(launch_add_shift(h->C[1], h->shift, h->n, h->npad, out_dev, h->stream));
    } else {
        CW_TRY(cudaMemcpyAsync(out_dev, h->C[order], sizeof(double) * h->E[order],
                               cudaMemcpyDeviceToDevice, h->stream));
    }
    return CUMWIN_OK;
}

int cumwin_full(cumwin_t h, int order, double* out_dev)
{
    if (h == nullptr || out_dev == nullptr || order < 1 || order > h->d) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    int64_t nf = 1;
    for (int s = 0; s < order; ++s) {
        nf *= h->n;
        if (nf > ((int64_t)1 << 36)) {
            g_last_error = "the full tensor would hold more than 2^36 elements";
            return CUMWIN_EINVAL;
        }
    }
    CW_TRY(join(h));
    CW_TRY(launch_expand(h->C[order], nf, order, h->n, h->b, h->nst, 1.0, order == 1 ? h->shift : nullptr, out_dev,
                         h->stream));
    return CUMWIN_OK;
}

int cumwin_moments(cumwin_t h, int order, double* out_dev)
{
    if (h == nullptr || out_dev == nullptr || order < 1 || order > h->d) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    CW_TRY(join(h));
    // kept in workspace order, or at canonical elements only: gather back to the block layout
    if (h->cum[order].sgemm || h->cum[order].canon)
        CW_TRY(launch_gather_sums(h->cum_dev + order, h->E[order], 1.0 / (double)h->T, out_dev, h->stream));
    else
        CW_TRY(launch_scale(h->S[order], 1.0 / (double)h->T, h->E[order], out_dev, h->stream));
    return CUMWIN_OK;
}

int cumwin_shift(cumwin_t h, float* shift_host)
{
    if (h == nullptr || shift_host == nullptr) return CUMWIN_EINVAL;
    CW_TRY(join(h));
    CW_TRY(cudaMemcpyAsync(shift_host, h->shift, sizeof(float) * h->n, cudaMemcpyDeviceToHost,
                           h->stream));
    CW_TRY(cudaStreamSynchronize(h->stream));
    return CUMWIN_OK;
}

int cumwin_norms_device(cumwin_t h, double* fro2_dev)
{
    if (h == nullptr || fro2_dev == nullptr) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    CW_TRY(join(h));
    CW_TRY(cudaMemcpyAsync(fro2_dev, h->fro2, sizeof(double) * h->d, cudaMemcpyDeviceToDevice,
                           h->stream));
    return CUMWIN_OK;
}

int cumwin_norms_k(cumwin_t h, double k, double* out_host)
{
    if (h == nullptr || out_host == nullptr || !(k >= 1.0) || !std::isfinite(k)) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    CW_TRY(join(h));
    double* parts = h->knorm_parts;  // kKnormParts per order, allocated at create
    for (int s = 1; s <= h->d; ++s) {
        const int np = (int)std::max<int64_t>(1, std::min<int64_t>(kKnormParts, (h->E[s] + 255) / 256));
        CW_TRY(launch_knorm(h->cum_dev + s, h->E[s], k, parts + (size_t)(s - 1) * kKnormParts, np, h->stream));
    }
    std::vector<double> host((size_t)kKnormParts * h->d, 0.0);
    CW_TRY(cudaMemcpyAsync(host.data(), parts, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, h->stream));
    CW_TRY(cudaStreamSynchronize(h->stream));
    for (int s = 1; s <= h->d; ++s) {
        const int np = (int)std::max<int64_t>(1, std::min<int64_t>(kKnormParts, (h->E[s] + 255) / 256));
        double z = 0.0;
        for (int q = 0; q < np; ++q) z += host[(size_t)(s - 1) * kKnormParts + q];
        out_host[s - 1] = std::pow(z, 1.0 / k);
    }
    return CUMWIN_OK;
}

int cumwin_marginals(cumwin_t h, double* skew_host, double* kurt_host)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    CW_TRY(join(h));
    const int n = h->n, dm = std::min(h->d, 4);
    std::vector<double> diag((size_t)(dm + 1) * n, NAN);
    if (dm >= 2) {  // the diagonal entries C_s[i..i], s = 2..dm, through the index table of create
        for (int s = 2; s <= dm; ++s)
            CW_TRY(launch_gather_idx(h->C[s], h->diag_idx + (size_t)(s - 2) * n, n, h->diag_val + (size_t)(s - 2) * n,
                                     h->stream));
        CW_TRY(cudaMemcpyAsync(diag.data() + 2 * (size_t)n, h->diag_val, sizeof(double) * (size_t)(dm - 1) * n,
                               cudaMemcpyDeviceToHost, h->stream));
        CW_TRY(cudaStreamSynchronize(h->stream));
    }
    for (int i = 0; i < n; ++i) {
        const double v2 = diag[2 * (size_t)n + i];
        const bool ok = dm >= 2 && v2 > 0.0;
        if (skew_host) skew_host[i] = ok && dm >= 3 ? diag[3 * (size_t)n + i] / std::pow(v2, 1.5) : NAN;
        if (kurt_host) kurt_host[i] = ok && dm >= 4 ? diag[4 * (size_t)n + i] / (v2 * v2) : NAN;
    }
    return CUMWIN_OK;
}

static void nu_from_fro(const double* fro, int d, double* nu)
{
    for (int s = 1; s <= d; ++s)
        nu[s - 1] = (s < 3 || d < 2) ? NAN : fro[s - 1] / std::pow(fro[1], 0.5 * s);
}

int cumwin_norms(cumwin_t h, double* fro_host, double* nu_host)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    CW_TRY(join(h));
    double z[kMaxOrder];
    int st = 0;
    CW_TRY(cudaMemcpyAsync(z, h->fro2, sizeof(double) * h->d, cudaMemcpyDeviceToHost, h->stream));
    CW_TRY(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CW_TRY(cudaStreamSynchronize(h->stream));
    double fro[kMaxOrder];
    for (int s = 0; s < h->d; ++s) fro[s] = std::sqrt(z[s]);
    if (fro_host)
        for (int s = 0; s < h->d; ++s) fro_host[s] = fro[s];
    if (nu_host) nu_from_fro(fro, h->d, nu_host);
    if (st & kStatusNonFinite) return CUMWIN_ENONFINITE;
    if (st & kStatusTimeout) return CUMWIN_ETIMEOUT;
    return CUMWIN_OK;
}

int cumwin_recompute(cumwin_t h)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    CW_TRY(join(h));
    int rc = zero_sums(h);
    if (rc) return rc;
    rc = update_window(h);
    if (rc) return rc;
    return run_cumulants(h, 0);
}

int cumwin_recenter(cumwin_t h)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    CW_TRY(join(h));
    if (h->prec != CUMWIN_FP64)  // the new shift: the current window's column means
        CW_TRY(launch_column_mean(h->ring, h->T, h->n, h->npad, h->shift, h->stream));
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
    CW_TRY(join(h));
    CW_TRY(launch_window_copy(h->ring, h->T, h->head, h->n, h->npad, out_dev, h->stream));
    return CUMWIN_OK;
}

int cumwin_grad(cumwin_t h, const double* w_host, float* dX_dev)
{
    if (h == nullptr || w_host == nullptr || dX_dev == nullptr) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    if (h->nshards > 1) {
        g_last_error = "the adjoint needs the whole top-order tensor, not a block shard";
        return CUMWIN_ENOTSUP;
    }
    CW_TRY(join(h));
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
        int64_t eblk = 0;
        for (int s = 1; s <= d; ++s) {
            CW_TRY(h->alloc(&g.Cf[s], g.nf[s]));
            CW_TRY(h->alloc(&g.G[s], g.nf[s]));
            CW_TRY(h->alloc(&g.GM[s], g.nf[s]));
            if (s < d) CW_TRY(h->alloc(&g.Mf[s], g.nf[s]));
            if (s < d && (h->cum[s].sgemm || h->cum[s].canon)) eblk = std::max(eblk, h->E[s]);
        }
        if (eblk > 0) CW_TRY(h->alloc(&g.Sblk, eblk));
        CW_TRY(h->alloc(&g.C1true, n));
        g.nst = h->nst;
        // sorted (s-1)-tuples of variables with their numbers of distinct orderings
        std::vector<uint64_t> uv;
        std::vector<float> um;
        std::vector<uint8_t> unf;
        for (int s = 1; s <= d; ++s) {
            g.uoff[s] = (int)uv.size();
            const int k = s - 1;
            if (k == 0) {
                uv.push_back(0ull);
                um.push_back(1.0f);
                unf.push_back(0);
                continue;
            }
            const std::vector<int> tup = enumerate_sorted(n, k);
            for (size_t q = 0; q < tup.size() / k; ++q) {
                uint64_t p = 0;  // up to kMaxOrder - 1 = 7 variables of 8 bits
                for (int i = 0; i < k; ++i) p |= (uint64_t)tup[q * k + i] << (8 * i);
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
        if (s < d) {
            // the sums of a canonical order are kept at its canonical elements only (in workspace order
            // in the mixed forms): gather every stored element from its canonical one first
            const double* src = h->S[s];
            if (h->cum[s].sgemm || h->cum[s].canon) {
                CW_TRY(launch_gather_sums(h->cum_dev + s, h->E[s], 1.0, g.Sblk, st));
                src = g.Sblk;
            }
            CW_TRY(launch_expand(src, g.nf[s], s, n, h->b, g.nst, invT, nullptr, g.Mf[s], st));
        }
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

// The recovery's copies of the K-split of the handle's plan.
static int sync_ksplit(cumwin_t h)
{
    const int ks = h->tc->ksplit;
    for (int s = 1; s <= h->d; ++s) h->cum[s].ksplit = ks;
    CumArgs arr[2][kAccModes][kMaxOrder + 1] = {};
    for (int s = 1; s <= h->d; ++s)
        for (int q = 0; q < 2; ++q)
            for (int m = 0; m < kAccModes; ++m) {
                arr[q][m][s] = h->cum[s];
                arr[q][m][s].accum = m;
                if (q == 1 && h->tc->W2 != nullptr) arr[q][m][s].W = h->tc->W2;
            }
    CW_TRY(cudaMemcpy(h->cum_dev, &arr[0][0][0], sizeof(arr), cudaMemcpyHostToDevice));
    return CUMWIN_OK;
}

int cumwin_set_tiles(cumwin_t h, int ksplit, int nmax, int group)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    if (h->tc == nullptr) return CUMWIN_OK;  // the FP64 form has no tensor-core update
    if (ksplit < 1 || ksplit > h->tc->ksplit_max || nmax < 16 || nmax > kTcNmax || nmax % 16 != 0 || group < 1)
        return CUMWIN_EINVAL;
    CW_TRY(join(h));
    CW_TRY(cudaDeviceSynchronize());  // no GEMM of this handle reads the items while they change
    const int rc = tc_plan_items(*h->tc, nmax, group);
    if (rc) return fail_cuda((cudaError_t)rc, "tc_plan_items");
    h->tc->ksplit = ksplit;
    return sync_ksplit(h);
}

int cumwin_tune(cumwin_t h, int reps, int* ksplit_out)
{
    if (h == nullptr || reps < 1) return CUMWIN_EINVAL;
    if (!h->filled) return CUMWIN_ESTATE;
    CW_TRY(join(h));
    if (h->tc == nullptr) {
        if (ksplit_out) *ksplit_out = 0;
        return CUMWIN_OK;  // nothing to tune in the FP64 form
    }
    const bool leaving = !(h->tc->fifo != nullptr && h->fifo_valid);
    const int ks = tc_autotune(*h->tc, reps, leaving, h->stream, nullptr);
    if (ks < 0) return fail_cuda((cudaError_t)(-ks), "tc_autotune");
    const int rc = sync_ksplit(h);
    if (rc) return rc;
    tune_cache_put(plan_signature(*h->tc, {h}, h->device), *h->tc);
    if (ksplit_out) *ksplit_out = ks;
    return CUMWIN_OK;
}

int cumwin_get_tiles(cumwin_t h, int* ksplit, int* nmax, int* group)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    const TcPlan* tc = h->tc;
    if (ksplit) *ksplit = tc ? tc->ksplit : 0;
    if (nmax) *nmax = tc ? tc->nmax : 0;
    if (group) *group = tc ? tc->group : 0;
    return CUMWIN_OK;
}

int cumwin_set_timing(cumwin_t h, int enable)
{
    if (h == nullptr) return CUMWIN_EINVAL;
    CW_TRY(join(h));
    h->timing = enable != 0;
    h->coarse = enable == 2;
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
    CW_TRY(join(h));
    CW_TRY(cudaStreamSynchronize(h->stream));
    double a = 0.0, u = 0.0, c = 0.0;
    for (int64_t k = 0; k < h->timed; ++k) {
        float t0 = 0.f, t1 = 0.f, t2 = 0.f;
        if (h->coarse) {  // staging counted in the update
            CW_TRY(cudaEventElapsedTime(&t1, h->ev[4 * k], h->ev[4 * k + 2]));
        } else {
            CW_TRY(cudaEventElapsedTime(&t0, h->ev[4 * k], h->ev[4 * k + 1]));
            CW_TRY(cudaEventElapsedTime(&t1, h->ev[4 * k + 1], h->ev[4 * k + 2]));
        }
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
    CW_TRY(join(h));
    int st = 0;
    CW_TRY(cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CW_TRY(cudaStreamSynchronize(h->stream));
    if (st & kStatusNonFinite) return CUMWIN_ENONFINITE;
    if (st & kStatusTimeout) return CUMWIN_ETIMEOUT;
    return CUMWIN_OK;
}

// ---------------------------------------------------------------------------
// batches of independent windows
// ---------------------------------------------------------------------------
int cumwin_batch_destroy(cumwin_batch_t B)
{
    if (B == nullptr) return CUMWIN_OK;
    cudaStreamSynchronize(B->stream);
    for (cumwin_s* h : B->wins) {
        h->release();
        delete h;
    }
    B->mem.release();
    delete B;
    return CUMWIN_OK;
}

int cumwin_batch_create(int nwin, const int* n, const int* d, const int64_t* T, int b, int p, int precision,
                        void* cuda_stream, cumwin_batch_t* out)
{
    if (out == nullptr || n == nullptr || d == nullptr || T == nullptr || nwin < 1 || nwin > 65535)
        return CUMWIN_EINVAL;
    *out = nullptr;
    if (precision == CUMWIN_FP64) {
        g_last_error = "batches run the tensor-core forms";
        return CUMWIN_ENOTSUP;
    }
    for (int i = 0; i < nwin; ++i) {
        const int rc = check_args(n[i], d[i], b, T[i], p, precision);
        if (rc) return rc;
    }
    cumwin_batch_s* B = new cumwin_batch_s();
    B->nwin = nwin;
    B->b = b;
    B->p = p;
    B->prec = precision;
    B->stream = (cudaStream_t)cuda_stream;
    B->mem.al = current_allocator();
    B->mem.stream = B->stream;
    auto bail = [&](int code) {
        cumwin_batch_destroy(B);
        return code;
    };
    B->xoff.assign(nwin + 1, 0);
    std::vector<TcPlanStream> ps(nwin);
    for (int i = 0; i < nwin; ++i) {
        cumwin_s* h = new cumwin_s();
        B->wins.push_back(h);
        const int rc = window_init(h, n[i], d[i], b, T[i], p, precision, B->stream, false);
        if (rc) return bail(rc);
        B->dmax = std::max(B->dmax, d[i]);
        B->sm_count = h->sm_count;
        B->xoff[i + 1] = B->xoff[i] + (int64_t)p * n[i];
        TcPlanStream& q = ps[i];
        q.tables = &h->ut;
        q.upd = &h->upd;
        q.Eoff = h->Eoff;
        q.d = d[i];
        q.n = n[i];
        q.npad = h->npad;
        q.T = T[i];
        q.ring = h->ring;
        q.head = h->head;
        q.shift = h->shift;
        q.status = h->status;
        q.xoff = B->xoff[i];
    }
    cudaError_t e0 = B->mem.alloc(&B->status, 1);
    if (e0 != cudaSuccess) return bail(fail_cuda(e0, "alloc"));
    cudaMemset(B->status, 0, sizeof(int));
    int rc = tc_plan_create(B->tc, ps, b, p, B->sm_count, precision, B->status, true, false,
                            [&](size_t bytes, void** q) { return B->mem.alloc((char**)q, bytes); });
    if (rc != 0) {
        g_last_error = "tensor-core plan: " + std::string(cudaGetErrorString((cudaError_t)rc));
        return bail(rc == (int)cudaErrorMemoryAllocation ? CUMWIN_ENOMEM : CUMWIN_ECUDA);
    }
    tune_cache_apply(B->tc, tune_cache_get(plan_signature(B->tc, B->wins, B->wins[0]->device)));
    // recovery launch shapes over all windows (b is shared, so b^s is too)
    int parts = 1;
    for (int s = 1; s <= B->dmax; ++s) {
        int64_t nb = 0;
        for (cumwin_s* h : B->wins)
            if (s <= h->d) nb = std::max<int64_t>(nb, n_sorted(h->nbar, s));
        B->cum_launch[s] = plan_cumulants(s, (int)ipow(b, s), nb, B->sm_count);
        parts = std::max(parts, B->cum_launch[s].gx * B->cum_launch[s].gy);
    }
    B->fifo = B->tc.fifo != nullptr;
    std::vector<CumArgs> arr((size_t)kAccModes * (kMaxOrder + 1) * nwin);
    std::vector<NormArgs> na(nwin);
    cudaError_t e = B->mem.alloc(&B->fro2, (size_t)nwin * B->dmax);
    if (e != cudaSuccess) return bail(fail_cuda(e, "alloc"));
    for (int i = 0; i < nwin; ++i) {
        cumwin_s* h = B->wins[i];
        h->fro2 = B->fro2 + (size_t)i * B->dmax;
        h->tc = &B->tc;
        rc = window_finish(h, parts, &B->tc, i);
        if (rc) return bail(rc);
        for (int s = 1; s <= B->dmax; ++s) {
            for (int acc = 0; acc < kAccModes; ++acc) {
                CumArgs a{};
                if (s <= h->d) {
                    a = h->cum[s];
                    a.accum = acc;
                }  // else E = 0: the kernel skips this window
                arr[((size_t)acc * (kMaxOrder + 1) + s) * nwin + i] = a;
            }
        }
        na[i].normpart = h->normpart;
        na[i].fro2 = h->fro2;
        na[i].head = h->head_rec;
        na[i].head_stage = nullptr;  // the operand build advances it
        na[i].T = h->T;
        na[i].parts = parts;
        na[i].d = h->d;
    }
    e = B->mem.upload(&B->cum_dev, arr);
    if (e == cudaSuccess) e = B->mem.upload(&B->norm_dev, na);
    if (e == cudaSuccess) {
        rc = fused_setup(B->fused, B->wins, b, B->sm_count, B->norm_dev, B->status, B->mem, 4);
        if (rc) return bail(rc);
        // a shift as one cooperative launch when every order is in the fused recovery
        // and one 1024-thread CTA fits on every SM
        if (B->fused.dfused > 0 && B->dmax <= B->fused.dfused &&
            batch_shift_blocks_per_sm(precision, B->fused.dfused) >= 1) {
            e = B->mem.alloc(&B->shift_bar, kBarrierWords);
            if (e == cudaSuccess) e = cudaMemset(B->shift_bar, 0, kBarrierWords * sizeof(unsigned));
            if (e == cudaSuccess) B->shift_grid = B->sm_count;
        }
    }
    std::vector<TcAccSeg> segs = acc_segments(B->wins, B->tc);
    B->nsegs = (int)segs.size();
    if (e == cudaSuccess) e = B->mem.upload(&B->segs, segs);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return bail(fail_cuda(e, "batch create"));
    *out = B;
    return CUMWIN_OK;
}

int64_t cumwin_batch_offset(cumwin_batch_t B, int window)
{
    if (B == nullptr || window < 0 || window > B->nwin) return -1;
    return B->xoff[window];
}

static int batch_recover(cumwin_batch_t B, int64_t advance, int accum, int64_t* launches = nullptr)
{
    int64_t L = 0;
    const int rc = recover(B->fused, B->cum_dev, B->cum_launch, B->norm_dev, B->nwin, B->dmax, advance, accum,
                           B->sm_count, B->stream, &L);
    if (launches != nullptr) *launches = L;
    return rc;
}

int cumwin_batch_fill(cumwin_batch_t B, const float* const* X_dev)
{
    if (B == nullptr || X_dev == nullptr) return CUMWIN_EINVAL;
    for (int i = 0; i < B->nwin; ++i)
        if (X_dev[i] == nullptr) return CUMWIN_EINVAL;
    for (int i = 0; i < B->nwin; ++i) {
        cumwin_s* h = B->wins[i];
        h->stream = B->stream;
        const int rc = fill_prepare(h, X_dev[i], h->n);
        if (rc) return rc;
    }
    for (int q = 0; q < B->tc.nbatch; ++q) {
        CW_TRY(tc_update_window_batch(B->tc, q, B->stream));
        CW_TRY(launch_tc_accumulate(B->tc, B->segs, B->nsegs, q, B->stream));
    }
    const int rc = batch_recover(B, 0, 0);
    if (rc) return rc;
    for (cumwin_s* h : B->wins) h->filled = true;
    B->filled = true;
    return CUMWIN_OK;
}

int cumwin_batch_push(cumwin_batch_t B, const float* x_dev)
{
    if (B == nullptr || x_dev == nullptr) return CUMWIN_EINVAL;
    if (!B->filled) return CUMWIN_ESTATE;
    if (B->single && B->shift_grid > 0) {
        // staging, operand build, GEMM and recovery as the phases of one launch
        const TcPlan& tc = B->tc;
        BatchShiftArgs a{};
        a.sdesc = tc.sdesc;
        a.xin = x_dev;
        a.p = B->p;
        a.P = tc.P;
        a.nstreams = tc.nstreams;
        a.tiles_x = (tc.P + 31) / 32;
        a.tiles_y = (tc.npad_max + 31) / 32;
        a.leaving = B->fifo ? 0 : 1;
        a.scaled = tc.precision == 2;
        a.Kcap = tc.Kcap;
        a.vmax = tc.vmax;
        a.nvmax = tc.vmax != nullptr ? 2 * (int64_t)tc.npad_max * tc.nstreams : 0;
        a.opvars = tc.opvars;
        a.oprows = tc.oprows;
        a.ops = tc.ops;
        a.opexp = tc.opexp;
        a.nkb = (a.leaving ? 2 : 1) * tc.P / 8;
        a.gemm = tc_gemm_args(tc, a.leaving != 0, 0);
        FusedRecovery f = B->fused.f;
        const int accum = B->fifo ? 2 : 1;
        f.args = B->cum_dev + (size_t)accum * (kMaxOrder + 1) * B->nwin;
        f.advance = B->p;
        f.advance_heads = 1;
        f.fold = 1;
        f.bar = B->shift_bar;  // the recovery's own launches use another grid size
        CW_TRY(launch_batch_shift(tc, a, f, B->fused.dfused, B->shift_grid, B->stream));
        B->push_launches = 1;
        return CUMWIN_OK;
    }
    CW_TRY(tc_stage_push(B->tc, x_dev, nullptr, -1, B->p, !B->fifo, B->stream));  // staging + operand build
    CW_TRY(tc_gemm_push(B->tc, !B->fifo, 0, B->stream));
    int64_t L = 0;
    const int rc = batch_recover(B, B->p, B->fifo ? 2 : 1, &L);
    B->push_launches = 3 + L;
    return rc;
}

int cumwin_batch_cumulants(cumwin_batch_t B, int window, int order, double* out_dev)
{
    if (B == nullptr || window < 0 || window >= B->nwin) return CUMWIN_EINVAL;
    cumwin_s* h = B->wins[window];
    h->stream = B->stream;
    return cumwin_cumulants(h, order, out_dev);
}

int cumwin_batch_norms(cumwin_batch_t B, double* fro_host, double* nu_host)
{
    if (B == nullptr) return CUMWIN_EINVAL;
    if (!B->filled) return CUMWIN_ESTATE;
    std::vector<double> z((size_t)B->nwin * B->dmax);
    int st = 0;
    CW_TRY(cudaMemcpyAsync(z.data(), B->fro2, sizeof(double) * z.size(), cudaMemcpyDeviceToHost, B->stream));
    CW_TRY(cudaMemcpyAsync(&st, B->status, sizeof(int), cudaMemcpyDeviceToHost, B->stream));
    CW_TRY(cudaStreamSynchronize(B->stream));
    for (int i = 0; i < B->nwin; ++i) {
        const int d = B->wins[i]->d;
        double fro[kMaxOrder];
        for (int s = 0; s < B->dmax; ++s) fro[s] = s < d ? std::sqrt(z[(size_t)i * B->dmax + s]) : NAN;
        if (fro_host)
            for (int s = 0; s < B->dmax; ++s) fro_host[(size_t)i * B->dmax + s] = fro[s];
        if (nu_host) {
            double nu[kMaxOrder];
            nu_from_fro(fro, d, nu);
            for (int s = 0; s < B->dmax; ++s) nu_host[(size_t)i * B->dmax + s] = s < d ? nu[s] : NAN;
        }
    }
    for (cumwin_s* h : B->wins) {
        int ws = 0;
        CW_TRY(cudaMemcpy(&ws, h->status, sizeof(int), cudaMemcpyDeviceToHost));
        st |= ws;
    }
    if (st & kStatusNonFinite) return CUMWIN_ENONFINITE;
    if (st & kStatusTimeout) return CUMWIN_ETIMEOUT;
    return CUMWIN_OK;
}

int cumwin_batch_tune(cumwin_batch_t B, int reps, int* ksplit_out)
{
    if (B == nullptr || reps < 1) return CUMWIN_EINVAL;
    if (!B->filled) return CUMWIN_ESTATE;
    const int ks = tc_autotune(B->tc, reps, !B->fifo, B->stream, nullptr);
    if (ks < 0) return fail_cuda((cudaError_t)(-ks), "tc_autotune");
    std::vector<CumArgs> arr((size_t)kAccModes * (kMaxOrder + 1) * B->nwin);
    CW_TRY(cudaMemcpy(arr.data(), B->cum_dev, sizeof(CumArgs) * arr.size(), cudaMemcpyDeviceToHost));
    for (CumArgs& a : arr) a.ksplit = ks;
    CW_TRY(cudaMemcpy(B->cum_dev, arr.data(), sizeof(CumArgs) * arr.size(), cudaMemcpyHostToDevice));
    for (cumwin_s* h : B->wins)
        for (int s = 1; s <= h->d; ++s) h->cum[s].ksplit = ks;
    tune_cache_put(plan_signature(B->tc, B->wins, B->wins[0]->device), B->tc);
    if (ksplit_out) *ksplit_out = ks;
    return CUMWIN_OK;
}

int cumwin_batch_get_tiles(cumwin_batch_t B, int* ksplit, int* nmax, int* group)
{
    if (B == nullptr) return CUMWIN_EINVAL;
    if (ksplit) *ksplit = B->tc.ksplit;
    if (nmax) *nmax = B->tc.nmax;
    if (group) *group = B->tc.group;
    return CUMWIN_OK;
}

int cumwin_batch_set_single_launch(cumwin_batch_t B, int enable)
{
    if (B == nullptr) return CUMWIN_EINVAL;
    B->single = enable != 0;
    return B->shift_grid > 0 ? 1 : 0;
}

int cumwin_batch_fifo(cumwin_batch_t B)
{
    if (B == nullptr) return CUMWIN_EINVAL;
    return B->fifo ? 1 : 0;
}

int64_t cumwin_batch_launches(cumwin_batch_t B)
{
    return B == nullptr ? CUMWIN_EINVAL : B->push_launches;
}

int cumwin_batch_status(cumwin_batch_t B)
{
    if (B == nullptr) return CUMWIN_EINVAL;
    return cumwin_batch_norms(B, nullptr, nullptr);
}

}  // extern "C"
