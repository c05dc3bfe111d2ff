// Device code of the tensor-core update shared by its own kernels
// (k_update_tc.cu) and the single-launch batch shift (k_cumulants.cu): the
// staging tile, the Khatri-Rao operand build and the warp-specialised tcgen05
// GEMM, as functions of a (virtual) CTA.  See cw_tc.h for the pipeline.
#pragma once

#include <climits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cw_device.cuh"
#include "cw_tc.h"
#include "tc_ptx.cuh"

namespace cw {
namespace tcdev {

using namespace ptx;

constexpr int KC = kTcKC, TM = kTcM, NMAX = kTcNmax, STAGES = kTcStages;
constexpr int GEMM_THREADS = 192;  // warp 0: TMA, warp 1: MMA, warps 2-5: epilogue
constexpr long long kWaitLimit = 1LL << 32;  // clock cycles (~2 s)
static_assert(KC * 2 == 128, "one K-chunk is one 128-byte swizzle row of bf16");

constexpr int A_PART = TM * 128;      // bytes of one 16-bit part of an A tile (128 rows x 128 B)
constexpr int B_PART = NMAX * 128;    // bytes of one 16-bit part of a B tile (up to NMAX rows)
constexpr int STAGE_BYTES = 2 * A_PART + 2 * B_PART;
constexpr size_t GEMM_SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
constexpr size_t gemm_smem(int nst) { return (size_t)nst * STAGE_BYTES + 1024; }

// ---------------------------------------------------------------------------
// staging: shifted samples, transposed to [variable][sample]
// ---------------------------------------------------------------------------
// Samples [0, P) of the K axis hold X_(+), [P, 2P) hold X_(-) (when
// `leaving`), zero beyond p.
// Each (virtual) CTA moves a tile of 32 samples x 32 variables of one stream
// through shared memory so that both the row-major reads and the
// variable-major writes are coalesced; the thread that reads X_(-) from a ring
// slot also writes X_(+) into it.
// One tile (bx: sample tile, by: variable tile, bz: stream) by a (virtual)
// CTA of 256 threads, through tin / tout (32 x 33 floats each).
template <bool V>
__device__ __forceinline__ void stage_push_tile(const TcStreamDesc* __restrict__ sdesc,
                                                const float* __restrict__ xin_base,
                                                const float* __restrict__ xout_base, int64_t ld_arg, int p, int P,
                                                int64_t Kcap, int leaving, int scaled, int bx, int by, int bz,
                                                float (*tin)[33], float (*tout)[33])
{
    const TcStreamDesc sd = sdesc[bz];
    const int r0 = bx * 32, v0 = by * 32;
    if (v0 >= sd.npad) return;
    const int64_t head = *sd.head;
    const int64_t ld = ld_arg < 0 ? sd.n : ld_arg;
    const float* x_in = xin_base + sd.xoff;
    const float* x_out = xout_base != nullptr ? xout_base + sd.xoff : nullptr;
    const int tid = vtid<V>();
    const int tx = tid & 31, ty = tid >> 5;  // 32 x 8
    bool badv = false;
    for (int rr = ty; rr < 32; rr += 8) {
        const int r = r0 + rr, v = v0 + tx;
        float xin = 0.0f, xo = 0.0f;
        if (r < p && v < sd.npad) {
            int64_t slot = head + r;
            if (slot >= sd.T) slot -= sd.T;
            const float raw_in = v < sd.n ? x_in[(int64_t)r * ld + v] : 0.0f;
            float raw_out = 0.0f;
            if (leaving) {
                if (x_out != nullptr) raw_out = v < sd.n ? x_out[(int64_t)r * ld + v] : 0.0f;
                else raw_out = sd.ring[slot * sd.npad + v];
            }
            sd.ring[slot * sd.npad + v] = raw_in;
            badv |= !isfinite(raw_in);
            if (v < sd.n) {
                xin = raw_in - sd.shift[v];
                xo = raw_out - sd.shift[v];
            }
        }
        tin[rr][tx] = xin;
        tout[rr][tx] = xo;
    }
    vsync<V>();
    if (scaled && ty == 0 && v0 + tx < sd.n) {  // FP16 form: largest |sample| per variable and half
        float mi = 0.0f, mo = 0.0f;
        for (int rr = 0; rr < 32; ++rr) {
            mi = fmaxf(mi, fabsf(tin[rr][tx]));
            mo = fmaxf(mo, fabsf(tout[rr][tx]));
        }
        // non-negative floats order as their bit patterns
        if (mi > 0.0f) atomicMax(reinterpret_cast<unsigned*>(sd.vmax) + v0 + tx, __float_as_uint(mi));
        if (leaving && mo > 0.0f)
            atomicMax(reinterpret_cast<unsigned*>(sd.vmax) + sd.npad + v0 + tx, __float_as_uint(mo));
    }
    for (int vv = ty; vv < 32; vv += 8) {
        const int v = v0 + vv, r = r0 + tx;
        if (v < sd.npad && r < P) {
            sd.XT[(int64_t)v * Kcap + r] = tin[tx][vv];
            if (leaving) sd.XT[(int64_t)v * Kcap + P + r] = tout[tx][vv];
        }
    }
    if (badv) atomicOr(sd.status, kStatusNonFinite);
    vsync<V>();  // tin / tout may be refilled by the next tile
}

// Exponent e of the power-of-two scale 2^-e that maps |x| <= m into [0, 1):
// m = f * 2^e with f in [0.5, 1); 0 for m = 0 (or subnormal), clamped so that
// 2^-e is a normal float.
__device__ __forceinline__ int scale_exp(float m)
{
    const int ex = (int)((__float_as_uint(m) >> 23) & 0xffu);
    if (ex == 0) return 0;
    return min(125, max(-125, ex - 126));
}

__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((unsigned)(127 + k) << 23); }

// x * 2^k, exact unless the result leaves the float range (|k| <= 250).
__device__ __forceinline__ float scale_pow2(float x, int k)
{
    const int k1 = k / 2, k2 = k - k1;
    return __fmul_rn(__fmul_rn(x, pow2f(k1)), pow2f(k2));
}

// ---------------------------------------------------------------------------
// Khatri-Rao operand rows: product over the row's variables of 8 consecutive
// samples, split into 16-bit hi + lo, stored at [part][row][sample]
// (samples contiguous, Kcap per row).
// ---------------------------------------------------------------------------
// A row has at most this many factors (its variables are packed 8 bits each
// into 32 bits; a factor of order s <= 8 takes at most ceil(s / 2) of them).
constexpr int kMaxRowFactors = 4;

// Row `row`, samples [8 kb, 8 kb + 8).  The factors' loads are issued
// together (unrolled over the largest factor count); the products are formed
// in factor order, so the result does not depend on the unrolling.
template <bool BF16>
__device__ __forceinline__ void kr_build_item(const TcStreamDesc* __restrict__ sdesc, int64_t Kcap,
                                              uint64_t w, int64_t row, int kb, int64_t rows,
                                              uint16_t* __restrict__ ops, int P, int32_t* __restrict__ opexp)
{
    const uint32_t vars = (uint32_t)w;
    const int nf = (int)((w >> 32) & 0xffu);
    const TcStreamDesc* sd = &sdesc[(int)(w >> 40)];
    const float* XT = sd->XT;
    const int half = 8 * kb >= P ? 1 : 0;  // entering or leaving samples
    float4 a[kMaxRowFactors], c[kMaxRowFactors];
#pragma unroll
    for (int f = 0; f < kMaxRowFactors; ++f) {
        if (f < nf) {
            const int var = (int)((vars >> (8 * f)) & 0xffu);
            const float* xr = XT + (int64_t)var * Kcap + 8 * kb;
            a[f] = *reinterpret_cast<const float4*>(xr);
            c[f] = *reinterpret_cast<const float4*>(xr + 4);
        }
    }
    float p[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) p[t] = 1.0f;
    int esum = 0;
#pragma unroll
    for (int f = 0; f < kMaxRowFactors; ++f) {
        if (f < nf) {
            float4 x = a[f], y = c[f];
            if constexpr (!BF16) {  // every factor scaled into [-1, 1] by a power of two (exact)
                const int var = (int)((vars >> (8 * f)) & 0xffu);
                const int e = scale_exp(sd->vmax[half * sd->npad + var]);
                const float sc = pow2f(-e);
                esum += e;
                x.x *= sc; x.y *= sc; x.z *= sc; x.w *= sc;
                y.x *= sc; y.y *= sc; y.z *= sc; y.w *= sc;
            }
            p[0] *= x.x; p[1] *= x.y; p[2] *= x.z; p[3] *= x.w;
            p[4] *= y.x; p[5] *= y.y; p[6] *= y.z; p[7] *= y.w;
        }
    }
    if constexpr (!BF16) {
        if (8 * kb == half * P) opexp[(int64_t)half * rows + row] = esum;  // the row's scale, once per half
    }
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if constexpr (BF16) {
            const __nv_bfloat162 hv = __floats2bfloat162_rn(p[2 * q], p[2 * q + 1]);
            const float2 hf = __bfloat1622float2(hv);
            const __nv_bfloat162 lv = __floats2bfloat162_rn(p[2 * q] - hf.x, p[2 * q + 1] - hf.y);
            h[q] = *reinterpret_cast<const uint32_t*>(&hv);
            l[q] = *reinterpret_cast<const uint32_t*>(&lv);
        } else {
            const __half2 hv = __floats2half2_rn(p[2 * q], p[2 * q + 1]);
            const float2 hf = __half22float2(hv);
            const __half2 lv = __floats2half2_rn(p[2 * q] - hf.x, p[2 * q + 1] - hf.y);
            h[q] = *reinterpret_cast<const uint32_t*>(&hv);
            l[q] = *reinterpret_cast<const uint32_t*>(&lv);
        }
    }
    const int64_t part = rows * Kcap;  // elements of one part
    const int64_t o = row * Kcap + 8 * kb;
    *reinterpret_cast<uint4*>(ops + o) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(ops + part + o) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Row `row`, 256-sample chunk kc, as one warp: lane l forms samples
// 256 kc + 4 l + [0, 4) and 256 kc + 128 + 4 l + [0, 4), so that every load
// instruction of the warp reads 512 contiguous bytes of a staged variable and
// every store writes 256 contiguous bytes of a part (half as many L1
// wavefronts as 8 consecutive samples per lane).  The chunk lies inside one
// half (entering or leaving samples): P is a multiple of 256.  Products in
// factor order, bitwise those of kr_build_item.
template <bool BF16>
__device__ __forceinline__ void kr_build_chunk(const TcStreamDesc* __restrict__ sdesc, int64_t Kcap,
                                               uint64_t w, int64_t row, int kc, int lane, int64_t rows,
                                               uint16_t* __restrict__ ops, int P, int32_t* __restrict__ opexp)
{
    const uint32_t vars = (uint32_t)w;
    const int nf = (int)((w >> 32) & 0xffu);
    const TcStreamDesc* sd = &sdesc[(int)(w >> 40)];
    const float* XT = sd->XT;
    const int s0 = 256 * kc;
    const int half = s0 >= P ? 1 : 0;  // entering or leaving samples
    float4 a[kMaxRowFactors], c[kMaxRowFactors];
#pragma unroll
    for (int f = 0; f < kMaxRowFactors; ++f) {
        if (f < nf) {
            const int var = (int)((vars >> (8 * f)) & 0xffu);
            const float* xr = XT + (int64_t)var * Kcap + s0 + 4 * lane;
            a[f] = *reinterpret_cast<const float4*>(xr);
            c[f] = *reinterpret_cast<const float4*>(xr + 128);
        }
    }
    float p[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) p[t] = 1.0f;
    int esum = 0;
#pragma unroll
    for (int f = 0; f < kMaxRowFactors; ++f) {
        if (f < nf) {
            float4 x = a[f], y = c[f];
            if constexpr (!BF16) {  // every factor scaled into [-1, 1] by a power of two (exact)
                const int var = (int)((vars >> (8 * f)) & 0xffu);
                const int e = scale_exp(sd->vmax[half * sd->npad + var]);
                const float sc = pow2f(-e);
                esum += e;
                x.x *= sc; x.y *= sc; x.z *= sc; x.w *= sc;
                y.x *= sc; y.y *= sc; y.z *= sc; y.w *= sc;
            }
            p[0] *= x.x; p[1] *= x.y; p[2] *= x.z; p[3] *= x.w;
            p[4] *= y.x; p[5] *= y.y; p[6] *= y.z; p[7] *= y.w;
        }
    }
    if constexpr (!BF16) {
        if (lane == 0 && s0 == half * P) opexp[(int64_t)half * rows + row] = esum;  // once per half
    }
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if constexpr (BF16) {
            const __nv_bfloat162 hv = __floats2bfloat162_rn(p[2 * q], p[2 * q + 1]);
            const float2 hf = __bfloat1622float2(hv);
            const __nv_bfloat162 lv = __floats2bfloat162_rn(p[2 * q] - hf.x, p[2 * q + 1] - hf.y);
            h[q] = *reinterpret_cast<const uint32_t*>(&hv);
            l[q] = *reinterpret_cast<const uint32_t*>(&lv);
        } else {
            const __half2 hv = __floats2half2_rn(p[2 * q], p[2 * q + 1]);
            const float2 hf = __half22float2(hv);
            const __half2 lv = __floats2half2_rn(p[2 * q] - hf.x, p[2 * q + 1] - hf.y);
            h[q] = *reinterpret_cast<const uint32_t*>(&hv);
            l[q] = *reinterpret_cast<const uint32_t*>(&lv);
        }
    }
    const int64_t part = rows * Kcap;  // elements of one part
    const int64_t o = row * Kcap + s0 + 4 * lane;
    *reinterpret_cast<uint2*>(ops + o) = make_uint2(h[0], h[1]);
    *reinterpret_cast<uint2*>(ops + o + 128) = make_uint2(h[2], h[3]);
    *reinterpret_cast<uint2*>(ops + part + o) = make_uint2(l[0], l[1]);
    *reinterpret_cast<uint2*>(ops + part + o + 128) = make_uint2(l[2], l[3]);
}

// Elements [begin, rows * nkb) with the given stride of the build (begin = the
// thread's index, stride a multiple of 32): each is one row and 8 consecutive
// samples.  Element e -> (chunk of cw 8-sample steps, row, step): the 32 lanes
// of a warp write 32 consecutive steps of one row (512 contiguous bytes per
// part), consecutive warps take consecutive rows of the same chunk, so that the
// CTAs running at once read the staged samples of one chunk (npad x 8 cw
// floats) from L1.
template <bool BF16>
__device__ __forceinline__ void kr_build_range(const TcStreamDesc* __restrict__ sdesc, int64_t Kcap,
                                               const uint64_t* __restrict__ opvars, int64_t rows, int nkb,
                                               uint16_t* __restrict__ ops, int P, int32_t* __restrict__ opexp,
                                               int begin, int stride)
{
    // rows * nkb < 2^31 (checked on the host): 32-bit index arithmetic
    const int total = (int)(rows * nkb);
    if (nkb % 32 == 0) {
        // chunks of 32 steps: one (chunk, row) per warp and round, lane = step; the
        // next round's row descriptor is loaded before this round's item is built,
        // so that its latency overlaps the item instead of preceding the next one
        const int lane = begin & 31;
        const int nw = total >> 5, nrows = (int)rows, ws = stride >> 5;
        int wi = begin >> 5;
        if (wi >= nw) return;
        int kc = wi / nrows, row = wi - kc * nrows;
        uint64_t w = opvars[row];
        for (;;) {
            const int wn = wi + ws;
            int kcn = 0, rown = 0;
            uint64_t wnext = 0;
            if (wn < nw) {
                kcn = wn / nrows;
                rown = wn - kcn * nrows;
                wnext = opvars[rown];
            }
            if (P % 256 == 0) kr_build_chunk<BF16>(sdesc, Kcap, w, row, kc, lane, rows, ops, P, opexp);
            else kr_build_item<BF16>(sdesc, Kcap, w, row, 32 * kc + lane, rows, ops, P, opexp);
            if (wn >= nw) break;
            wi = wn;
            kc = kcn;
            row = rown;
            w = wnext;
        }
        return;
    }
    const int cw = nkb;  // fewer or ragged steps: one chunk
    const int rw = (int)rows * cw;
    for (int e = begin; e < total; e += stride) {
        const int kc = e / rw;
        const int rem = e - kc * rw;
        const int row = rem / cw;
        const int kb = kc * cw + (rem - row * cw);
        kr_build_item<BF16>(sdesc, Kcap, opvars[row], row, kb, rows, ops, P, opexp);
    }
}

// The build of kr_build_range in a register-lean form for the single-launch
// batch shift, whose build shares the launch's registers with the GEMM and
// recovery phases (the unrolled loads of kr_build_range tripled its spills):
// one row and 8 consecutive samples per element, factors loaded one after
// the other.  Bitwise the same operands.
template <bool BF16>
__device__ __forceinline__ void kr_build_range_lean(const TcStreamDesc* __restrict__ sdesc, int64_t Kcap,
                                               const uint64_t* __restrict__ opvars, int64_t rows, int nkb,
                                               uint16_t* __restrict__ ops, int P, int32_t* __restrict__ opexp,
                                               int begin, int stride)
{
    // rows * nkb < 2^31 (checked on the host): 32-bit index arithmetic
    const int total = (int)(rows * nkb);
    const int64_t part = rows * Kcap;  // elements of one part
    // item e -> (chunk of cw 8-sample steps, row, step): the 32 lanes of a warp write
    // 32 consecutive steps of one row (512 contiguous bytes per part), consecutive
    // warps take consecutive rows of the same chunk, so that the CTAs running at
    // once read the staged samples of one chunk (npad x 8 cw floats) from L1
    const int cw = nkb % 32 == 0 ? 32 : nkb;
    const int rw = (int)rows * cw;
    for (int e = begin; e < total; e += stride) {
        const int kc = e / rw;
        const int rem = e - kc * rw;
        const int row = rem / cw;
        const int kb = kc * cw + (rem - row * cw);
        const uint64_t w = opvars[row];
        const uint32_t vars = (uint32_t)w;
        const int nf = (int)((w >> 32) & 0xffu);
        const TcStreamDesc* sd = &sdesc[(int)(w >> 40)];
        const float* XT = sd->XT;
        float p[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) p[t] = 1.0f;
        const int half = 8 * kb >= P ? 1 : 0;  // entering or leaving samples
        int esum = 0;
        for (int f = 0; f < nf; ++f) {
            const int var = (int)((vars >> (8 * f)) & 0xffu);
            const float* xr = XT + (int64_t)var * Kcap + 8 * kb;
            float4 a = *reinterpret_cast<const float4*>(xr);
            float4 c = *reinterpret_cast<const float4*>(xr + 4);
            if constexpr (!BF16) {  // every factor scaled into [-1, 1] by a power of two (exact)
                const int e = scale_exp(sd->vmax[half * sd->npad + var]);
                const float sc = pow2f(-e);
                esum += e;
                a.x *= sc; a.y *= sc; a.z *= sc; a.w *= sc;
                c.x *= sc; c.y *= sc; c.z *= sc; c.w *= sc;
            }
            p[0] *= a.x; p[1] *= a.y; p[2] *= a.z; p[3] *= a.w;
            p[4] *= c.x; p[5] *= c.y; p[6] *= c.z; p[7] *= c.w;
        }
        if constexpr (!BF16) {
            if (8 * kb == half * P) opexp[(int64_t)half * rows + row] = esum;  // the row's scale, once per half
        }
        uint32_t h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if constexpr (BF16) {
                const __nv_bfloat162 hv = __floats2bfloat162_rn(p[2 * q], p[2 * q + 1]);
                const float2 hf = __bfloat1622float2(hv);
                const __nv_bfloat162 lv = __floats2bfloat162_rn(p[2 * q] - hf.x, p[2 * q + 1] - hf.y);
                h[q] = *reinterpret_cast<const uint32_t*>(&hv);
                l[q] = *reinterpret_cast<const uint32_t*>(&lv);
            } else {
                const __half2 hv = __floats2half2_rn(p[2 * q], p[2 * q + 1]);
                const float2 hf = __half22float2(hv);
                const __half2 lv = __floats2half2_rn(p[2 * q] - hf.x, p[2 * q + 1] - hf.y);
                h[q] = *reinterpret_cast<const uint32_t*>(&hv);
                l[q] = *reinterpret_cast<const uint32_t*>(&lv);
            }
        }
        const int64_t o = (int64_t)row * Kcap + 8 * kb;
        *reinterpret_cast<uint4*>(ops + o) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(ops + part + o) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// 3-D TMA load: box {64 samples, rows, 1} at (k, row, part), 128-byte swizzle.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int k,
                                            int row, int part)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(k), "r"(row), "r"(part)
        : "memory");
}

// ---------------------------------------------------------------------------
// the GEMM: persistent, one CTA per SM looping over (item, K-split) units.
// Warp 0 streams A/B tiles through the STAGES-deep ring continuously across
// units; warp 1 issues the MMAs into one of two TMEM accumulator sets
// (columns [256*ab, 256*ab + 256): D_in then D_out); warps 2-5 drain the
// other set into the workspace while the next unit's MMAs run.
// ---------------------------------------------------------------------------
struct UnitRange {
    int nplus, nminus, p0, m0;
};

__device__ __forceinline__ UnitRange unit_range(const TcGemmArgs& args, int split)
{
    UnitRange r;
    const int cps_p = (args.nplus + args.ksplit - 1) / args.ksplit;
    const int p0 = min(args.nplus, split * cps_p), p1 = min(args.nplus, p0 + cps_p);
    const int cps_m = (args.nminus + args.ksplit - 1) / args.ksplit;
    const int m0 = min(args.nminus, split * cps_m), m1 = min(args.nminus, m0 + cps_m);
    r.nplus = p1 - p0;
    r.nminus = m1 - m0;
    r.p0 = p0;
    r.m0 = m0;
    return r;
}

// The bound of 4 CTAs per SM only caps the registers at 80 (shared memory allows
// one CTA per SM); uncapped (124 registers) pipelined shifts were about 1 us
// slower.  The GEMM of the next shift still starts only as the previous shift's
// recovery leaves an SM: to start beside the recovery's three CTAs it needs 64
// registers and the largest shared-memory split on both sides, which slowed the
// host-driven streaming loop.
// CTA-wide barrier of the GEMM's 192 threads: __syncthreads in its own
// kernel, a named barrier (id 5) inside the single-launch batch shift.
template <bool MEGA>
__device__ __forceinline__ void gemm_sync()
{
    if constexpr (MEGA) {
        asm volatile("bar.sync 5, %0;" ::"n"(GEMM_THREADS) : "memory");
    } else {
        __syncthreads();
    }
}

// The GEMM on threads 0..GEMM_THREADS-1 of a CTA; dsm_raw: NST stages of
// dynamic shared memory (gemm_smem(NST) bytes).
template <bool BF16, bool MEGA, int NST = STAGES>
__device__ __forceinline__ void kr_gemm_body(const CUtensorMap* mapA_p, const CUtensorMap* mapB32_p,
                                             const CUtensorMap* mapB64_p, const CUtensorMap* mapB128_p,
                                             const TcGemmArgs& args, unsigned char* dsm_raw)
{
    const CUtensorMap& mapA = *mapA_p;
    const CUtensorMap& mapB32 = *mapB32_p;
    const CUtensorMap& mapB64 = *mapB64_p;
    const CUtensorMap& mapB128 = *mapB128_p;
    unsigned char* dsm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t bar_full[NST], bar_empty[NST];
    __shared__ __align__(8) uint64_t bar_accfull[2], bar_accempty[2], bar_final;
    __shared__ uint32_t s_tbase;
    __shared__ int s_abort;
    __shared__ int64_t s_roww[4][NMAX];      // one copy per epilogue warp
    __shared__ int32_t s_rowcolmin[4][NMAX];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nunits = args.nitems * args.ksplit;

    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&bar_full[s], 1);
            mbar_init(&bar_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bar_accfull[b], 1);
            mbar_init(&bar_accempty[b], 4);  // one arrival per epilogue warp
        }
        mbar_init(&bar_final, 1);
        s_abort = 0;
        fence_mbar_init();
    }
    if (warp == 0 && lane == 0) {
        prefetch_tensormap(&mapA);
        prefetch_tensormap(&mapB32);
        prefetch_tensormap(&mapB64);
        prefetch_tensormap(&mapB128);
    }
    if (warp == 1) {
        tmem_alloc(&s_tbase, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    gemm_sync<MEGA>();
    tc_fence_after();
    const uint32_t tbase = s_tbase;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            grid_dep_wait();  // the operands come from the previous kernel
            uint32_t g = 0;
            bool stop = false;
            for (int u = blockIdx.x; u < nunits && !stop; u += gridDim.x) {
                const TcItem item = args.items[u / args.ksplit];
                const UnitRange R = unit_range(args, u % args.ksplit);
                const CUtensorMap* mapB = item.bbox == 32 ? &mapB32 : item.bbox == 64 ? &mapB64 : &mapB128;
                const uint32_t bytes = 2u * A_PART + 2u * (uint32_t)item.bbox * 128u;
                const int nch = R.nplus + R.nminus;
                for (int q = 0; q < nch; ++q, ++g) {
                    const uint32_t st = g % NST, use = g / NST;
                    if (g >= NST && !mbar_wait(&bar_empty[st], (use - 1) & 1, kWaitLimit)) {
                        atomicOr(args.status, kStatusTimeout);
                        s_abort = 1;
                        stop = true;
                        break;
                    }
                    if (*(volatile int*)&s_abort) {
                        stop = true;
                        break;
                    }
                    const int k = q < R.nplus ? (R.p0 + q) * KC : args.minus_k + (R.m0 + q - R.nplus) * KC;
                    unsigned char* sa = dsm + st * STAGE_BYTES;
                    unsigned char* sb = sa + 2 * A_PART;
                    mbar_arrive_expect_tx(&bar_full[st], bytes);
                    tma_load_3d(sa, &mapA, &bar_full[st], k, item.acol, 0);
                    tma_load_3d(sa + A_PART, &mapA, &bar_full[st], k, item.acol, 1);
                    tma_load_3d(sb, mapB, &bar_full[st], k, item.brow, 0);
                    tma_load_3d(sb + B_PART, mapB, &bar_full[st], k, item.brow, 1);
                }
            }
            // drain: every issued load has landed before the CTA may exit (bounded)
            for (uint32_t q = g > NST ? g - NST : 0; q < g; ++q)
                mbar_wait(&bar_full[q % NST], (q / NST) & 1, kWaitLimit);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            uint32_t g = 0, it = 0;
            bool stop = false;
            for (int u = blockIdx.x; u < nunits && !stop; u += gridDim.x, ++it) {
                const TcItem item = args.items[u / args.ksplit];
                const UnitRange R = unit_range(args, u % args.ksplit);
                const int nch = R.nplus + R.nminus;
                const uint32_t ab = it & 1, ause = it >> 1;
                if (it >= 2 && !mbar_wait(&bar_accempty[ab], (ause - 1) & 1, kWaitLimit)) {
                    atomicOr(args.status, kStatusTimeout);
                    s_abort = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t idesc = idesc_f16(TM, (item.nrows + 15) & ~15, BF16);
                for (int q = 0; q < nch; ++q, ++g) {
                    const uint32_t st = g % NST, use = g / NST;
                    if (!mbar_wait(&bar_full[st], use & 1, kWaitLimit)) {
                        atomicOr(args.status, kStatusTimeout);
                        s_abort = 1;
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const bool plus = q < R.nplus;
                    const bool first = (q == 0) || (q == R.nplus);
                    const uint32_t d = tbase + ab * 256u + (plus ? 0u : (uint32_t)NMAX);
                    const uint32_t sa = smem_u32(dsm + st * STAGE_BYTES);
                    const uint32_t sb = sa + 2 * A_PART;
#pragma unroll
                    for (int ks = 0; ks < KC / 16; ++ks) {
                        const uint64_t ah = smem_desc_sw128(sa + ks * 32);
                        const uint64_t al = smem_desc_sw128(sa + A_PART + ks * 32);
                        const uint64_t bh = smem_desc_sw128(sb + ks * 32);
                        const uint64_t bl = smem_desc_sw128(sb + B_PART + ks * 32);
                        tc_mma_f16(d, ah, bh, idesc, (first && ks == 0) ? 0u : 1u);
                        tc_mma_f16(d, ah, bl, idesc, 1u);
                        tc_mma_f16(d, al, bh, idesc, 1u);
                    }
                    tc_commit(&bar_empty[st]);
                }
                tc_commit(&bar_accfull[ab]);
            }
            // every MMA issued by this CTA has completed before TMEM is freed (bounded)
            tc_commit(&bar_final);
            mbar_wait(&bar_final, 0, kWaitLimit);
        }
    } else {
        // ---------------- epilogue: TMEM -> FP32 workspace ----------------
        const int ew = warp - 2;  // 0..3
        const int quarter = warp & 3;
        const bool scaled = args.opexp != nullptr;
        if (scaled) grid_dep_wait();  // the row scales come from the operand build
        uint32_t it = 0;
        for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++it) {
            const TcItem item = args.items[u / args.ksplit];
            const int split = u % args.ksplit;
            const UnitRange R = unit_range(args, split);
            const TcOrder& od = args.ord[item.stream * (kMaxOrder + 1) + item.s];
            const uint32_t ab = it & 1;
            // this warp's copy of the row tables of an item that spans groups
            int64_t* roww = s_roww[ew];
            int32_t* rowcolmin = s_rowcolmin[ew];
            if (!item.fast) {
                __syncwarp();
                for (int r = lane; r < NMAX; r += 32) {
                    const bool v = r < item.nrows;
                    roww[r] = v ? od.roww[item.row0 + r] : 0;
                    rowcolmin[r] = v ? od.rowcolmin[item.row0 + r] : INT_MAX;
                }
                __syncwarp();
            }
            const bool ok = mbar_wait(&bar_accfull[ab], (it >> 1) & 1, kWaitLimit);
            if (!ok || *(volatile int*)&s_abort) {
                if (!ok && lane == 0) atomicOr(args.status, kStatusTimeout);
                s_abort = 1;
                break;
            }
            tc_fence_after();
            const int i = 32 * quarter + lane;
            const bool ivalid = i < item.ncols;
            const int cglob = item.col0 + i;
            float* Win = args.W + (int64_t)(2 * split) * args.wslice + od.woff;
            float* Wout = Win + args.wslice;
            const int NB = (item.nrows + 15) & ~15;
            // FP16 form: the exponents of this lane's column (A row) scale, per half
            int ec0 = 0, ec1 = 0;
            if (scaled && ivalid) {
                ec0 = args.opexp[item.acol + i];
                if (args.nminus > 0) ec1 = args.opexp[args.oprows + item.acol + i];
            }
            // 16 rows per round: one TMEM load per accumulator, one wait, then
            // one coalesced 64-byte store per row (lanes = consecutive slots)
            for (int jb = 0; jb < NB; jb += 16) {
                uint32_t d0[16], d1[16];
                const uint32_t ta = tbase + ab * 256u + ((uint32_t)(32 * quarter) << 16) + (uint32_t)jb;
                if (R.nplus > 0) tmem_ld16p(ta, d0);
                if (R.nminus > 0) tmem_ld16p(ta + (uint32_t)NMAX, d1);
                tmem_ld_wait();
                if (scaled) {  // undo the operand scales: D * 2^(row exponent + column exponent), exact
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        const int r = min(jb + t, item.nrows - 1);
                        d0[t] = __float_as_uint(scale_pow2(__uint_as_float(d0[t]), ec0 + args.opexp[item.brow + r]));
                        if (args.nminus > 0)
                            d1[t] = __float_as_uint(
                                scale_pow2(__uint_as_float(d1[t]), ec1 + args.opexp[args.oprows + item.brow + r]));
                    }
                }
                if (item.fast) {
                    const int64_t w0 = (int64_t)item.wrow0 + (int64_t)jb * item.wwidth + cglob;
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        if (ivalid && jb + t < item.nrows) {
                            const int64_t e = w0 + (int64_t)t * item.wwidth;
                            Win[e] = R.nplus > 0 ? __uint_as_float(d0[t]) : 0.0f;
                            if (args.nminus > 0) Wout[e] = R.nminus > 0 ? __uint_as_float(d1[t]) : 0.0f;
                        }
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        const int r = jb + t;
                        if (ivalid && r < item.nrows && cglob >= rowcolmin[r]) {
                            const int64_t e = roww[r] + cglob;
                            Win[e] = R.nplus > 0 ? __uint_as_float(d0[t]) : 0.0f;
                            if (args.nminus > 0) Wout[e] = R.nminus > 0 ? __uint_as_float(d1[t]) : 0.0f;
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_accempty[ab]);
        }
    }
    tc_fence_before();
    gemm_sync<MEGA>();
    if (warp == 1) tmem_dealloc(tbase, 512);
}


}  // namespace tcdev
}  // namespace cw
