// Moment-sum update on the 5th-generation tensor cores (Eqs. 6-7, Algorithm 2),
// for one or many independent windows at once.
//
// See cw_tc.h for the pipeline.  This file holds the staging kernels, the
// Khatri-Rao operand builder, the warp-specialized persistent tcgen05 GEMM,
// the host planner and the K-split autotuner.  Every mbarrier wait is
// bounded: on a timeout the CTA records kStatusTimeout, drains the copies and
// MMAs it issued (bounded), frees its tensor memory and returns.
#include <climits>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <map>

#include "cw_device.cuh"
#include "cw_tc.h"
#include "cw_tc_device.cuh"
#include "tc_ptx.cuh"

namespace cw {

namespace {

using namespace ptx;

using namespace tcdev;

// Staging (cw_tc_device.cuh): one 32 x 32 tile per CTA, blockIdx.z = stream.
__global__ void __launch_bounds__(256)
k_tc_stage_push(const TcStreamDesc* __restrict__ sdesc, const float* __restrict__ xin_base,
                const float* __restrict__ xout_base, int64_t ld_arg, int p, int P, int64_t Kcap, int leaving,
                int scaled)
{
    __shared__ float tin[32][33], tout[32][33];
    grid_dep_launch();  // the operand build may launch now; it waits for this grid
    stage_push_tile<false>(sdesc, xin_base, xout_base, ld_arg, p, P, Kcap, leaving, scaled, blockIdx.x, blockIdx.y,
                           blockIdx.z, tin, tout);
}

// Window rows [q*p, q*p + p) (window order, oldest first) into samples [0, P);
// blockIdx.y = stream.
__global__ void __launch_bounds__(256)
k_tc_stage_batch(const TcStreamDesc* __restrict__ sdesc, int q, int p, int P, int64_t Kcap, int scaled)
{
    grid_dep_launch();
    const TcStreamDesc sd = sdesc[blockIdx.y];
    const int64_t head = *sd.head;
    const int64_t total = (int64_t)sd.npad * P;
    // P is a multiple of 64 and the stride a multiple of 32, so the 32 lanes of a
    // warp always take the same variable in the same iteration (the reduction below)
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(e / P);
        const int r = (int)(e - (int64_t)v * P);
        const int64_t w = (int64_t)q * p + r;
        float x = 0.0f;
        if (r < p && w < sd.T && v < sd.n) {
            int64_t slot = head + w;
            if (slot >= sd.T) slot -= sd.T;
            x = sd.ring[slot * sd.npad + v] - sd.shift[v];
        }
        sd.XT[(int64_t)v * Kcap + r] = x;
        if (scaled) {  // FP16 form: largest |sample| of the variable in this batch
            const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(x)));
            if ((threadIdx.x & 31) == 0 && m != 0u && v < sd.n)
                atomicMax(reinterpret_cast<unsigned*>(sd.vmax) + v, m);
        }
    }
}

// Operand build (cw_tc_device.cuh); advances the staging ring heads.  A
// persistent grid of kBuildCtasPerSm CTAs per SM, so that each thread builds
// many items and the next item's row descriptor load overlaps the current one.
constexpr int kBuildCtasPerSm = 4;
template <bool BF16>
__global__ void __launch_bounds__(256, kBuildCtasPerSm)
k_kr_build(const TcStreamDesc* __restrict__ sdesc, int64_t Kcap, const uint64_t* __restrict__ opvars,
           int64_t rows, int nkb, uint16_t* __restrict__ ops, int nstreams, int64_t advance, int P,
           int32_t* __restrict__ opexp)
{
    grid_dep_launch();  // the GEMM may launch now; its TMA warp waits for this grid
    grid_dep_wait();    // the staged samples come from the previous kernel
    // the staging of this shift is complete: its ring heads move on (the
    // recovery keeps its own head, so it may still run on another stream)
    if (advance != 0 && blockIdx.x == 0)
        for (int i = threadIdx.x; i < nstreams; i += blockDim.x) {
            int64_t* hp = sdesc[i].head;
            *hp = (*hp + advance) % sdesc[i].T;
        }
    kr_build_range<BF16>(sdesc, Kcap, opvars, rows, nkb, ops, P, opexp, blockIdx.x * blockDim.x + threadIdx.x,
                         gridDim.x * blockDim.x);
}

// The GEMM (cw_tc_device.cuh): persistent, one CTA per SM.  The bound of 4
// CTAs per SM only caps the registers at 80 (shared memory allows one CTA per
// SM); uncapped (124 registers) pipelined shifts were about 1 us slower.  The
// GEMM of the next shift still starts only as the previous shift's recovery
// leaves an SM: to start beside the recovery's three CTAs it needs 64
// registers and the largest shared-memory split on both sides, which slowed
// the host-driven streaming loop.
template <bool BF16>
__global__ void __launch_bounds__(GEMM_THREADS, 4)
k_kr_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB32,
          const __grid_constant__ CUtensorMap mapB64, const __grid_constant__ CUtensorMap mapB128,
          const TcGemmArgs args)
{
    extern __shared__ unsigned char dsm_raw[];
    kr_gemm_body<BF16, false>(&mapA, &mapB32, &mapB64, &mapB128, args, dsm_raw);
}

// Batch q of the window: S += (double)D_in for every (stream, order) segment,
// D_in = sum_k W[k][0] at the element's workspace slot; with a FIFO, D_in is
// also kept (workspace order) in slot (head / p + q) mod nslots, the batch's
// slot from then on.  Sums kept in workspace order are indexed by the slot.
// Threads run over storage elements (e) so the FP64 sums are read and
// written contiguously.
__global__ void __launch_bounds__(256)
k_tc_accumulate(const float* __restrict__ W, int64_t wslice, int ksplit, const TcAccSeg* __restrict__ segs,
                int nsegs, int q)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < wslice;
         e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nsegs - 1;  // last segment with begin <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (segs[mid].begin <= e) lo = mid;
            else hi = mid - 1;
        }
        const TcAccSeg& g = segs[lo];
        const int64_t el = e - g.begin;
        if (el >= g.E) continue;
        int64_t slot = el;  // sums in workspace order: element = slot
        if (!g.sgemm) {
            const int32_t blk = (int32_t)(el / g.bs), a = (int32_t)(el - (int64_t)blk * g.bs);
            const int32_t aL = a / g.bR, aR = a - aL * g.bR;
            slot = (int64_t)g.wblk[2 * blk] + (int64_t)aL * g.wblk[2 * blk + 1] + aR;
        }
        const float din = sum_in_partials(W + g.begin + slot, wslice, ksplit);
        g.S[el] += f32_to_f64(din);
        if (g.fifo != nullptr && q < g.nslots) {
            const int64_t f = (*g.head / g.p + q) % g.nslots;
            g.fifo[f * g.fstride + slot] = din;
        }
    }
}

// Launch configuration with programmatic stream serialization: the kernel may
// start while the previous one on the stream runs (it waits with
// grid_dep_wait before reading what that one wrote).
void pdl_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute (&attr)[1], dim3 grid, dim3 block, size_t smem,
                cudaStream_t st)
{
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
}

inline int grid_for(int64_t work)
{
    int64_t g = (work + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 16384));
}

cudaError_t launch_gemm(const TcPlan& plan, float* W, int nplus, int nminus, int minus_k, cudaStream_t st)
{
    TcGemmArgs a{};
    a.ord = plan.ord;
    a.items = plan.items;
    a.opexp = plan.precision == 2 ? plan.opexp : nullptr;
    a.oprows = plan.oprows;
    a.W = W;
    a.wslice = plan.wslice;
    a.nitems = plan.nitems;
    a.ksplit = plan.ksplit;
    a.nplus = nplus;
    a.nminus = nminus;
    a.minus_k = minus_k;
    a.status = plan.status;
    const int units = plan.nitems * plan.ksplit;
    const int grid = units < plan.sm_count ? units : plan.sm_count;
    if (grid < 1) return cudaSuccess;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    pdl_config(cfg, attr, dim3(grid), dim3(GEMM_THREADS), GEMM_SMEM, st);
    if (plan.precision == 1)
        return cudaLaunchKernelEx(&cfg, k_kr_gemm<true>, plan.mapA, plan.mapB[0], plan.mapB[1], plan.mapB[2], a);
    return cudaLaunchKernelEx(&cfg, k_kr_gemm<false>, plan.mapA, plan.mapB[0], plan.mapB[1], plan.mapB[2], a);
}

cudaError_t launch_build(const TcPlan& plan, int nsamples, int64_t advance, cudaStream_t st)
{
    const int nkb = nsamples / 8;
    const int64_t work = plan.oprows * nkb;
    const int grid = std::min(grid_for(work), kBuildCtasPerSm * std::max(plan.sm_count, 1));
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    pdl_config(cfg, attr, dim3(grid), dim3(256), 0, st);
    if (plan.precision == 1)
        return cudaLaunchKernelEx(&cfg, k_kr_build<true>, (const TcStreamDesc*)plan.sdesc, plan.Kcap,
                                  (const uint64_t*)plan.opvars, plan.oprows, nkb, plan.ops, plan.nstreams, advance,
                                  plan.P, plan.opexp);
    return cudaLaunchKernelEx(&cfg, k_kr_build<false>, (const TcStreamDesc*)plan.sdesc, plan.Kcap,
                              (const uint64_t*)plan.opvars, plan.oprows, nkb, plan.ops, plan.nstreams, advance,
                              plan.P, plan.opexp);
}

// --------------------------------------------------------------------------
// planning (host)
// --------------------------------------------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (fn == nullptr) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Operand array [part][row][Kcap] (16-bit), boxes of 64 samples x boxrows rows
// landing in shared memory in the 128-byte-swizzled K-major layout.
int encode_operand_map(CUtensorMap* map, void* base, int64_t rows, int64_t Kcap, int boxrows)
{
    EncodeTiledFn enc = get_encode_fn();
    if (enc == nullptr) return (int)cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)Kcap, (cuuint64_t)rows, 2};
    const cuuint64_t strides[2] = {(cuuint64_t)Kcap * 2, (cuuint64_t)rows * Kcap * 2};
    const cuuint32_t box[3] = {(cuuint32_t)KC, (cuuint32_t)boxrows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return (int)cudaErrorInvalidValue;
    return 0;
}

int b_box_rows(int nrows) { return nrows <= 32 ? 32 : nrows <= 64 ? 64 : 128; }

// Per-K-chunk cost model of one item (cycles): tensor time of 3 MMAs of
// 128 x N x KC against the operand bytes streamed in, plus a fixed overhead.
double item_chunk_cost(int nrows)
{
    const int NB = (nrows + 15) & ~15;
    const double mma = 3.0 * TM * NB * KC / 4096.0;
    const double tma = (2.0 * A_PART + 2.0 * 128 * b_box_rows(nrows)) / 128.0;
    return std::max(mma, tma) + 60.0;
}

}  // namespace

int tc_plan_create(TcPlan& plan, const std::vector<TcPlanStream>& streams, int b, int p, int sm_count,
                   int precision, int* status, bool fifo, bool double_w, const DevAlloc& alloc)
{
    (void)b;
    plan.precision = precision;
    plan.nstreams = (int)streams.size();
    plan.p = p;
    plan.P = (p + KC - 1) / KC * KC;
    plan.Kcap = 2 * (int64_t)plan.P;
    plan.status = status;
    plan.sm_count = sm_count;
    if (plan.nstreams < 1 || plan.nstreams > (1 << 20)) return (int)cudaErrorInvalidValue;

    // per-stream staging buffers and descriptors
    std::vector<TcStreamDesc> sdesc(plan.nstreams);
    plan.nbatch = 0;
    plan.nbatch_stream.assign(plan.nstreams, 0);
    for (const TcPlanStream& S : streams) plan.npad_max = std::max(plan.npad_max, S.npad);
    if (precision == 2) {
        cudaError_t e = alloc(sizeof(float) * 2 * (size_t)plan.npad_max * plan.nstreams, (void**)&plan.vmax);
        if (e != cudaSuccess) return (int)e;
    }
    for (int i = 0; i < plan.nstreams; ++i) {
        const TcPlanStream& S = streams[i];
        TcStreamDesc& sd = sdesc[i];
        cudaError_t e = alloc(sizeof(float) * (size_t)S.npad * plan.Kcap, (void**)&sd.XT);
        if (e != cudaSuccess) return (int)e;
        e = cudaMemset(sd.XT, 0, sizeof(float) * (size_t)S.npad * plan.Kcap);
        if (e != cudaSuccess) return (int)e;
        sd.ring = S.ring;
        sd.head = S.head;
        sd.shift = S.shift;
        sd.status = S.status;
        sd.T = S.T;
        sd.xoff = S.xoff;
        sd.n = S.n;
        sd.npad = S.npad;
        sd.vmax = plan.vmax != nullptr ? plan.vmax + (size_t)2 * plan.npad_max * i : nullptr;
        plan.nbatch_stream[i] = (int)((S.T + p - 1) / p);
        plan.nbatch = std::max(plan.nbatch, plan.nbatch_stream[i]);
    }
    cudaError_t e = alloc(sizeof(TcStreamDesc) * sdesc.size(), (void**)&plan.sdesc);
    if (e != cudaSuccess) return (int)e;
    e = cudaMemcpy(plan.sdesc, sdesc.data(), sizeof(TcStreamDesc) * sdesc.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return (int)e;

    // operand sets per stream: key (factors, grouped?) -> first row; singles
    // and the empty product have one ordering
    std::vector<uint64_t> opvars;
    std::vector<TcOrder> ord((size_t)plan.nstreams * (kMaxOrder + 1));
    plan.wbase.assign(plan.nstreams, 0);
    int64_t wtot = 0;
    double useful = 0, issued = 0;
    for (int i = 0; i < plan.nstreams; ++i) {
        const TcPlanStream& S = streams[i];
        // key: (factors, grouped + 2 * compressed); sets of at most one factor
        // have a single ordering and nothing to compress
        std::map<std::pair<int, int>, int64_t> setoff;
        auto add_set = [&](int k, int grouped, bool compressed, const std::vector<uint32_t>& vars) -> int64_t {
            const std::pair<int, int> key(k, k <= 1 ? 0 : grouped + 2 * (int)compressed);
            auto it = setoff.find(key);
            if (it != setoff.end()) return it->second;
            const int64_t off = (int64_t)opvars.size();
            for (uint32_t v : vars)
                opvars.push_back((uint64_t)v | ((uint64_t)k << 32) | ((uint64_t)i << 40));
            setoff[key] = off;
            return off;
        };
        plan.wbase[i] = wtot;
        for (int s = 1; s <= S.d; ++s) {
            const UpdateTables& t = (*S.tables)[s];
            const OrderTables& ot = S.upd->ord[s];
            TcOrder& o = ord[(size_t)i * (kMaxOrder + 1) + s];
            o.woff = wtot + S.Eoff[s];
            const std::vector<int64_t> roww = build_w_rows(t);
            {
                int64_t* dw = nullptr;
                e = alloc(sizeof(int64_t) * std::max<size_t>(roww.size(), 1), (void**)&dw);
                if (e != cudaSuccess) return (int)e;
                e = cudaMemcpy(dw, roww.data(), sizeof(int64_t) * roww.size(), cudaMemcpyHostToDevice);
                if (e != cudaSuccess) return (int)e;
                o.roww = dw;
            }
            const int64_t loff = add_set(t.h, 1, t.compressed, t.rowvar);
            const int64_t roff = add_set(t.sh, 0, t.compressed, t.colvar);
            const int nbar = (int)t.colstart.size();
            const int ncols = (int)t.colvar.size();
            std::vector<int32_t> colmin(t.rowvar.size());
            for (int m = 0; m < nbar; ++m)
                for (int r = t.rowstart[m]; r < t.rowstart[m + 1]; ++r) colmin[r] = t.colstart[m];
            int32_t* dcm = nullptr;
            e = alloc(sizeof(int32_t) * std::max<size_t>(colmin.size(), 1), (void**)&dcm);
            if (e != cudaSuccess) return (int)e;
            e = cudaMemcpy(dcm, colmin.data(), sizeof(int32_t) * colmin.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return (int)e;
            o.rowcolmin = dcm;

            // row ranges: groups larger than NMAX rows are split; consecutive small
            // groups are merged (invalid pairs are masked) while that lowers the
            // modelled cost
            struct Range { int r0, r1, c0; };
            std::vector<Range> ranges;
            // a block shard of the top order keeps, per group, the rows of the left tuples
            // whose blocks (jL ++ any sorted jR) meet [top0, top1): a contiguous run of the
            // group's rows, as the blocks of consecutive left tuples follow each other
            std::vector<int> keep0(t.rowstart.begin(), t.rowstart.end() - 1), keep1(t.rowstart.begin() + 1,
                                                                                        t.rowstart.end());
            if (s == S.d && S.top1 >= 0 && t.sh > 0) {
                for (int m = 0; m < nbar; ++m) {
                    keep0[m] = INT_MAX;
                    keep1[m] = INT_MIN;
                }
                const std::vector<int> left = enumerate_sorted(nbar, t.h);
                std::vector<int> full(s);
                for (size_t q = 0; q < left.size() / t.h; ++q) {
                    const int* jl = &left[q * t.h];
                    const int m = jl[t.h - 1];
                    for (int k = 0; k < t.h; ++k) full[k] = jl[k];
                    for (int k = t.h; k < s; ++k) full[k] = m;
                    const int64_t lo = rank_sorted(full.data(), s, nbar);
                    for (int k = t.h; k < s; ++k) full[k] = nbar - 1;
                    const int64_t hi = rank_sorted(full.data(), s, nbar);
                    if (hi < S.top0 || lo >= S.top1) continue;
                    keep0[m] = std::min(keep0[m], t.leftrow[q]);
                    keep1[m] = std::max(keep1[m], t.leftrow[q] + t.leftcnt[q]);
                }
            }
            for (int m = 0; m < nbar; ++m) {
                const int r0 = keep0[m], r1 = keep1[m];
                if (r1 <= r0 || t.colstart[m] >= ncols) continue;
                for (int r = r0; r < r1; r += NMAX) ranges.push_back({r, std::min(r1, r + NMAX), t.colstart[m]});
            }
            auto cost = [&](const Range& R) {
                const int span = ncols - R.c0;
                return ((span + TM - 1) / TM) * item_chunk_cost(R.r1 - R.r0);
            };
            std::vector<Range> merged;
            for (const Range& R : ranges) {
                if (!merged.empty()) {
                    Range& L = merged.back();
                    if (L.r1 == R.r0 && R.r1 - L.r0 <= NMAX) {
                        Range M{L.r0, R.r1, L.c0};
                        if (cost(M) <= cost(L) + cost(R)) {
                            L = M;
                            continue;
                        }
                    }
                }
                merged.push_back(R);
            }
            TcRangeSet rs;
            rs.s = s;
            rs.stream = i;
            rs.ncols = ncols;
            rs.loff = loff;
            rs.roff = roff;
            rs.rowstart = t.rowstart;
            rs.colstart = t.colstart;
            rs.roww = roww;
            rs.colmin = colmin;
            for (const Range& R : merged) rs.ranges.push_back({R.r0, R.r1, R.c0});
            if (!rs.ranges.empty()) plan.rsets.push_back(std::move(rs));
        }
        wtot += S.Eoff[S.d + 1];
    }
    plan.wslice = wtot;
    // the higher orders (the largest GEMMs) first; the small ones fill the tail
    std::stable_sort(plan.rsets.begin(), plan.rsets.end(),
                     [](const TcRangeSet& x, const TcRangeSet& y) { return x.s > y.s; });
    (void)useful;
    (void)issued;
    // room for the items of the finest tile shape the autotuner tries
    int64_t cap = 0;
    for (const TcRangeSet& rs : plan.rsets)
        for (const TcRangeSet::Range& R : rs.ranges)
            cap += (int64_t)((R.r1 - R.r0 + 63) / 64 + 1) * ((rs.ncols - R.c0 + TM - 1) / TM);
    plan.items_cap = (int)std::max<int64_t>(1, cap);
    e = alloc(sizeof(TcItem) * (size_t)plan.items_cap, (void**)&plan.items);
    if (e != cudaSuccess) return (int)e;
    {
        const int rc = tc_plan_items(plan, NMAX, 8);
        if (rc) return rc;
    }

    // K-splits: a few units per persistent CTA, at least 2 chunks per split,
    // the workspace (2 x ksplit x wslice floats) within 256 MB
    const int chunks = plan.P / KC;
    int64_t kmem = ((int64_t)256 << 20) / std::max<int64_t>(1, 8 * plan.wslice);
    plan.ksplit_max = (int)std::max<int64_t>(1, std::min<int64_t>(kmem, std::max(1, chunks / 2)));
    // default: the largest power of two keeping at most one unit per CTA
    // (powers of two divide the chunk count, so no split is left empty).  Each
    // split adds one FP32 image of the sums that the recovery reads back, so
    // fewer splits are preferred (see tc_autotune).
    int ks = 1;
    while (2 * ks <= plan.ksplit_max && (int64_t)plan.nitems * 2 * ks <= (int64_t)sm_count) ks *= 2;
    plan.ksplit = ks;

    e = alloc(sizeof(TcOrder) * ord.size(), (void**)&plan.ord);
    if (e != cudaSuccess) return (int)e;
    e = cudaMemcpy(plan.ord, ord.data(), sizeof(TcOrder) * ord.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return (int)e;

    // operand array and its tensor maps
    plan.oprows = (int64_t)opvars.size();
    if (plan.oprows * (plan.Kcap / 8) >= ((int64_t)1 << 31) || plan.oprows >= ((int64_t)1 << 31))
        return (int)cudaErrorInvalidValue;
    if (precision == 2) {
        e = alloc(sizeof(int32_t) * 2 * (size_t)plan.oprows, (void**)&plan.opexp);
        if (e != cudaSuccess) return (int)e;
        e = cudaMemset(plan.opexp, 0, sizeof(int32_t) * 2 * (size_t)plan.oprows);
        if (e != cudaSuccess) return (int)e;
    }
    e = alloc(sizeof(uint64_t) * opvars.size(), (void**)&plan.opvars);
    if (e != cudaSuccess) return (int)e;
    e = cudaMemcpy(plan.opvars, opvars.data(), sizeof(uint64_t) * opvars.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return (int)e;
    const size_t opbytes = sizeof(uint16_t) * 2 * (size_t)plan.Kcap * plan.oprows;
    e = alloc(opbytes, (void**)&plan.ops);
    if (e != cudaSuccess) return (int)e;
    e = cudaMemset(plan.ops, 0, opbytes);
    if (e != cudaSuccess) return (int)e;
    int rc = encode_operand_map(&plan.mapA, plan.ops, plan.oprows, plan.Kcap, TM);
    if (rc) return rc;
    for (int k = 0; k < 3; ++k) {
        rc = encode_operand_map(&plan.mapB[k], plan.ops, plan.oprows, plan.Kcap, 32 << k);
        if (rc) return rc;
    }

    // workspace for the largest K-split the autotuner may pick
    e = alloc(sizeof(float) * 2 * (size_t)plan.ksplit_max * plan.wslice, (void**)&plan.W);
    if (e != cudaSuccess) return (int)e;
    e = cudaMemset(plan.W, 0, sizeof(float) * 2 * (size_t)plan.ksplit_max * plan.wslice);
    if (e != cudaSuccess) return (int)e;
    if (double_w) {  // a second workspace: the GEMM of one shift while the recovery of the last reads the first
        e = alloc(sizeof(float) * 2 * (size_t)plan.ksplit_max * plan.wslice, (void**)&plan.W2);
        if (e != cudaSuccess) return (int)e;
        e = cudaMemset(plan.W2, 0, sizeof(float) * 2 * (size_t)plan.ksplit_max * plan.wslice);
        if (e != cudaSuccess) return (int)e;
    }

    // batch-sum FIFO: T_i / p slots of every stream's sums (workspace order)
    plan.fbase.assign(plan.nstreams, 0);
    if (fifo) {
        bool ok = true;
        int64_t ftot = 0;
        for (int i = 0; i < plan.nstreams; ++i) {
            if (streams[i].T % p != 0) ok = false;
            plan.fbase[i] = ftot;
            ftot += streams[i].T / p * streams[i].Eoff[streams[i].d + 1];
        }
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) ok = false;
        if (ok && (size_t)ftot * sizeof(float) <= free_b / 4) {
            e = alloc(sizeof(float) * (size_t)std::max<int64_t>(ftot, 1), (void**)&plan.fifo);
            if (e != cudaSuccess) return (int)e;
            e = cudaMemset(plan.fifo, 0, sizeof(float) * (size_t)std::max<int64_t>(ftot, 1));
            if (e != cudaSuccess) return (int)e;
        }
    }

    e = cudaFuncSetAttribute(k_kr_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM);
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(k_kr_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM);
    if (e != cudaSuccess) return (int)e;
    plan.ready = 1;
    return 0;
}

int tc_plan_items(TcPlan& plan, int nmax, int group)
{
    if (nmax < 16 || nmax > NMAX || nmax % 16 != 0 || group < 1) return (int)cudaErrorInvalidValue;
    std::vector<TcItem> items;
    double issued = 0.0, useful = 0.0;
    for (const TcRangeSet& rs : plan.rsets) {
        // row tiles: every range cut into pieces of at most nmax rows
        std::vector<TcRangeSet::Range> tiles;
        for (const TcRangeSet::Range& R : rs.ranges) {
            // a tile's columns start at the first valid column of its first row (the
            // smallest of its rows': groups, in row order, start at increasing columns),
            // so that a tile inside one group has no masked column
            for (int r = R.r0; r < R.r1; r += nmax)
                tiles.push_back({r, std::min(R.r1, r + nmax), std::max(R.c0, (int)rs.colmin[r])});
            for (int r = R.r0; r < R.r1; ++r) useful += 3.0 * std::max(0, rs.ncols - rs.colmin[r]);
        }
        // super-blocks of `group` row tiles; inside one, by column position, then row tile
        for (size_t g0 = 0; g0 < tiles.size(); g0 += (size_t)group) {
            const size_t g1 = std::min(tiles.size(), g0 + (size_t)group);
            std::vector<std::pair<int, int>> order;  // (column, tile)
            for (size_t k = g0; k < g1; ++k)
                for (int c = tiles[k].c0; c < rs.ncols; c += TM) order.push_back({c, (int)k});
            std::stable_sort(order.begin(), order.end());
            for (const auto& ck : order) {
                const TcRangeSet::Range& R = tiles[ck.second];
                const int c = ck.first;
                TcItem it{};
                it.s = rs.s;
                it.row0 = R.r0;
                it.nrows = R.r1 - R.r0;
                it.col0 = c;
                it.ncols = std::min(TM, rs.ncols - c);
                it.brow = (int32_t)(rs.loff + R.r0);
                it.acol = (int32_t)(rs.roff + c);
                it.bbox = b_box_rows(it.nrows);
                it.stream = rs.stream;
                // rows of one group: the slots of a row follow from the first row's
                const int m0 = (int)(std::upper_bound(rs.rowstart.begin(), rs.rowstart.end(), R.r0) -
                                     rs.rowstart.begin()) - 1;
                it.fast = R.r1 <= rs.rowstart[m0 + 1] ? 1 : 0;
                it.wwidth = (int32_t)(rs.ncols - rs.colstart[m0]);
                it.wrow0 = (int32_t)rs.roww[R.r0];
                items.push_back(it);
                issued += 3.0 * TM * ((it.nrows + 15) & ~15);
            }
        }
    }
    if ((int)items.size() > plan.items_cap) return (int)cudaErrorInvalidValue;
    const cudaError_t e = cudaMemcpy(plan.items, items.data(), sizeof(TcItem) * items.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return (int)e;
    plan.nitems = (int)items.size();
    plan.nmax = nmax;
    plan.group = group;
    plan.useful_macs_per_sample = useful;
    plan.issued_macs_per_sample = issued;
    return 0;
}

cudaError_t tc_stage_push(const TcPlan& plan, const float* xin, const float* xout, int64_t ld, int p,
                          bool leaving, cudaStream_t st)
{
    if (p > plan.p) return cudaErrorInvalidValue;
    const dim3 grid((plan.P + 31) / 32, (plan.npad_max + 31) / 32, plan.nstreams);
    const int scaled = plan.precision == 2;
    if (scaled) {  // the per-variable maxima of this staging start from zero
        const cudaError_t e0 = cudaMemsetAsync(plan.vmax, 0, sizeof(float) * 2 * (size_t)plan.npad_max *
                                                                 plan.nstreams, st);
        if (e0 != cudaSuccess) return e0;
    }
    k_tc_stage_push<<<grid, 256, 0, st>>>(plan.sdesc, xin, xout, ld, p, plan.P, plan.Kcap, leaving ? 1 : 0, scaled);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_build(plan, (leaving ? 2 : 1) * plan.P, p, st);
}

TcGemmArgs tc_gemm_args(const TcPlan& plan, bool leaving, int parity)
{
    TcGemmArgs a{};
    a.ord = plan.ord;
    a.items = plan.items;
    a.opexp = plan.precision == 2 ? plan.opexp : nullptr;
    a.oprows = plan.oprows;
    a.W = parity != 0 && plan.W2 != nullptr ? plan.W2 : plan.W;
    a.wslice = plan.wslice;
    a.nitems = plan.nitems;
    a.ksplit = plan.ksplit;
    a.nplus = plan.P / KC;
    a.nminus = leaving ? plan.P / KC : 0;
    a.minus_k = plan.P;
    a.status = plan.status;
    return a;
}

cudaError_t tc_gemm_push(const TcPlan& plan, bool leaving, int parity, cudaStream_t st)
{
    float* W = parity != 0 && plan.W2 != nullptr ? plan.W2 : plan.W;
    return launch_gemm(plan, W, plan.P / KC, leaving ? plan.P / KC : 0, plan.P, st);
}

cudaError_t tc_update_window_batch(const TcPlan& plan, int q, cudaStream_t st)
{
    const int gx = std::max(1, std::min(64, (plan.npad_max * plan.P + 255) / 256));
    const int scaled = plan.precision == 2;
    if (scaled) {
        const cudaError_t e0 = cudaMemsetAsync(plan.vmax, 0, sizeof(float) * 2 * (size_t)plan.npad_max *
                                                                 plan.nstreams, st);
        if (e0 != cudaSuccess) return e0;
    }
    k_tc_stage_batch<<<dim3(gx, plan.nstreams), 256, 0, st>>>(plan.sdesc, q, plan.p, plan.P, plan.Kcap, scaled);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_build(plan, plan.P, 0, st);
    if (e != cudaSuccess) return e;
    return launch_gemm(plan, plan.W, plan.P / KC, 0, 0, st);
}

cudaError_t launch_tc_accumulate(const TcPlan& plan, const TcAccSeg* segs_dev, int nsegs, int q,
                                 cudaStream_t st)
{
    k_tc_accumulate<<<grid_for(plan.wslice), 256, 0, st>>>(plan.W, plan.wslice, plan.ksplit, segs_dev, nsegs, q);
    return cudaGetLastError();
}

int tc_autotune(TcPlan& plan, int reps, bool leaving, cudaStream_t st, double* best_ms)
{
    const int chunks = plan.P / KC;
    const int mchunks = leaving ? chunks : 0;
    // the item list is rewritten below: no GEMM queued before may still read it
    {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return -(int)e;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return -(int)cudaErrorUnknown;
    // average time of `reps` GEMM launches of the current shape (after one warm-up)
    auto time_gemm = [&](double* ms_out) -> cudaError_t {
        cudaError_t e = launch_gemm(plan, plan.W, chunks, mchunks, plan.P, st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_gemm(plan, plan.W, chunks, mchunks, plan.P, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        *ms_out = ms;
        return e;
    };
    auto fail = [&](cudaError_t e) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return -(int)e;
    };
    // 1. the tile shape at one K-split: rows per item and super-block height
    plan.ksplit = 1;
    int best_nmax = plan.nmax, best_group = plan.group;
    double best_t = 1e30;
    for (int nmax : {NMAX, NMAX / 2})
        for (int group : {1, 4, 8, 16}) {
            int rc = tc_plan_items(plan, nmax, group);
            if (rc) return fail((cudaError_t)rc);
            double ms = 0.0;
            const cudaError_t e = time_gemm(&ms);
            if (e != cudaSuccess) return fail(e);
            if (ms < best_t) {
                best_t = ms;
                best_nmax = nmax;
                best_group = group;
            }
        }
    {
        const int rc = tc_plan_items(plan, best_nmax, best_group);
        if (rc) return fail((cudaError_t)rc);
    }
    // 2. the K-split for that shape: the fewest splits within 10% of the fastest
    // (every split costs the recovery one more read of the workspace, which this
    // timing does not see)
    std::vector<double> times;
    double fastest = 1e30;
    for (int ks = 1; ks <= plan.ksplit_max && ks <= chunks; ks *= 2) {
        plan.ksplit = ks;
        double ms = 0.0;
        const cudaError_t e = time_gemm(&ms);
        if (e != cudaSuccess) return fail(e);
        times.push_back(ms);
        fastest = std::min(fastest, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int best = 1;
    double chosen = fastest;
    for (size_t i = 0, ks = 1; i < times.size(); ++i, ks *= 2)
        if (times[i] <= 1.10 * fastest) {
            best = (int)ks;
            chosen = times[i];
            break;
        }
    plan.ksplit = best;
    if (best_ms) *best_ms = chosen / std::max(1, reps);
    return best;
}

}  // namespace cw
