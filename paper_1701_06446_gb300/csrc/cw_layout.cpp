// Host-side block-layout arithmetic and the tables of the update and
// cumulant-recovery kernels.
#include "cw_layout.h"

#include <algorithm>
#include <cmath>

#include "cw_internal.h"

namespace cw {

int64_t binom(int64_t n, int64_t k)
{
    if (k < 0 || n < 0 || k > n) return 0;
    k = std::min(k, n - k);
    int64_t r = 1;
    for (int64_t i = 1; i <= k; ++i) r = r * (n - k + i) / i;  // exact at every step
    return r;
}

int64_t n_sorted(int nbar, int s)
{
    if (s == 0) return 1;
    return binom((int64_t)nbar + s - 1, s);
}

int64_t ipow(int64_t b, int e)
{
    int64_t r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

int64_t rank_sorted(const int* j, int s, int nbar)
{
    int64_t r = 0;
    int prev = 0;
    for (int k = 0; k < s; ++k) {
        if (j[k] < prev || j[k] >= nbar) return -1;
        // tuples that agree on positions < k and hold v < j[k] at position k:
        // the remaining s-k-1 positions are any sorted tuple over [v, nbar)
        for (int v = prev; v < j[k]; ++v) r += n_sorted(nbar - v, s - k - 1);
        prev = j[k];
    }
    return r;
}

std::vector<int> enumerate_sorted(int nbar, int s)
{
    std::vector<int> out;
    if (s == 0) return out;
    std::vector<int> j(s, 0);
    for (;;) {
        out.insert(out.end(), j.begin(), j.end());
        int k = s - 1;
        while (k >= 0 && j[k] == nbar - 1) --k;
        if (k < 0) break;
        j[k]++;
        for (int q = k + 1; q < s; ++q) j[q] = j[k];
    }
    return out;
}

double block_multiplicity(const int* j, int s)
{
    double f = 1.0;
    for (int i = 2; i <= s; ++i) f *= i;
    int run = 1;
    for (int k = 1; k <= s; ++k) {
        if (k < s && j[k] == j[k - 1]) {
            run++;
        } else {
            for (int i = 2; i <= run; ++i) f /= i;
            run = 1;
        }
    }
    return f;
}

static uint32_t pack_vars(const int* v, int cnt)
{
    uint32_t p = 0;
    for (int k = 0; k < cnt; ++k) p |= (uint32_t)v[k] << (8 * k);
    return p;
}

int run_mask(const int* j, int k)
{
    int m = 0;
    for (int i = 1; i < k; ++i)
        if (j[i] == j[i - 1]) m |= 1 << i;
    return m;
}

std::vector<int32_t> half_ranks(int b, int k, int mask)
{
    const int64_t bk = ipow(b, k);
    std::vector<int32_t> rk(bk, -1);
    int32_t next = 0;
    int dig[kMaxOrder];
    for (int64_t a = 0; a < bk; ++a) {
        int64_t rem = a;
        for (int i = k - 1; i >= 0; --i) {
            dig[i] = (int)(rem % b);
            rem /= b;
        }
        bool ok = true;
        for (int i = 1; i < k && ok; ++i) ok = !((mask >> i) & 1) || dig[i] >= dig[i - 1];
        if (ok) rk[a] = next++;
    }
    return rk;
}

static std::vector<int64_t> group_bases(const UpdateTables& t);

UpdateTables build_update_tables(int n, int b, int s, bool compressed)
{
    UpdateTables t;
    const int nbar = (n + b - 1) / b;
    const int h = split_rows(s), sh = s - h;
    t.s = s;
    t.h = h;
    t.sh = sh;
    t.compressed = compressed;
    // rank tables of the runs masks (compressed tables keep the offsets of rank >= 0)
    std::vector<std::vector<int32_t>> lranks(1 << kMaxOrder), rranks(1 << kMaxOrder);
    auto keep = [&](std::vector<std::vector<int32_t>>& cache, int k, int mask, int64_t a) {
        if (!compressed) return true;
        if (cache[mask].empty()) cache[mask] = half_ranks(b, k, mask);
        return cache[mask][a] >= 0;
    };
    const int64_t bs = ipow(b, s), bh = ipow(b, h), bsh = ipow(b, sh);
    auto off_first_below = [&](int m) -> int64_t {  // sorted sh-tuples whose first entry < m
        if (sh == 0) return 0;
        return n_sorted(nbar, sh) - n_sorted(nbar - m, sh);
    };

    // left rows, grouped by the last block index m
    const std::vector<int> left = enumerate_sorted(nbar, h);
    const int64_t nleft = (int64_t)left.size() / h;
    t.rowstart.assign(nbar + 1, 0);
    std::vector<int> full(s), vars(kMaxOrder);
    t.leftrow.assign(nleft, 0);
    t.leftcnt.assign(nleft, 0);
    for (int m = 0; m < nbar; ++m) {
        t.rowstart[m] = (int32_t)t.rowvar.size();
        const int64_t off_m = off_first_below(m);
        for (int64_t q = 0; q < nleft; ++q) {
            const int* jl = &left[q * h];
            if (jl[h - 1] != m) continue;
            t.leftrow[q] = (int32_t)t.rowvar.size();
            for (int k = 0; k < h; ++k) full[k] = jl[k];
            for (int k = h; k < s; ++k) full[k] = m;
            const int64_t P = rank_sorted(full.data(), s, nbar);
            const int lm = run_mask(jl, h);
            for (int64_t a = 0; a < bh; ++a) {
                if (!keep(lranks, h, lm, a)) continue;
                int64_t rem = a;
                for (int k = h - 1; k >= 0; --k) {
                    vars[k] = jl[k] * b + (int)(rem % b);
                    rem /= b;
                }
                t.rowvar.push_back(pack_vars(vars.data(), h));
                t.rowoff.push_back((P - off_m) * bs + a * bsh);
            }
            t.leftcnt[q] = (int32_t)t.rowvar.size() - t.leftrow[q];
        }
    }
    t.rowstart[nbar] = (int32_t)t.rowvar.size();

    // right columns, lexicographic
    t.colstart.assign(nbar, 0);
    if (sh == 0) {
        t.colvar.push_back(0u);
        t.coloff.push_back(0);
        t.rightcol.assign(1, 0);
    } else {
        const std::vector<int> right = enumerate_sorted(nbar, sh);
        const int64_t nright = (int64_t)right.size() / sh;
        t.rightcol.assign(nright, 0);
        for (int64_t q = 0; q < nright; ++q) {
            const int* jr = &right[q * sh];
            t.rightcol[q] = (int32_t)t.colvar.size();
            const int rm = run_mask(jr, sh);
            for (int64_t a = 0; a < bsh; ++a) {
                if (!keep(rranks, sh, rm, a)) continue;
                int64_t rem = a;
                for (int k = sh - 1; k >= 0; --k) {
                    vars[k] = jr[k] * b + (int)(rem % b);
                    rem /= b;
                }
                t.colvar.push_back(pack_vars(vars.data(), sh));
                t.coloff.push_back(q * bs + a);
            }
        }
        // group m pairs with the columns of the tuples whose first entry is >= m
        for (int m = 0; m < nbar; ++m) {
            const int64_t q = off_first_below(m);
            t.colstart[m] = q < nright ? t.rightcol[q] : (int32_t)t.colvar.size();
        }
    }
    t.wsize = group_bases(t)[nbar];
    return t;
}

// Workspace order of the order-s update: group m is a dense
// rows_m x (ncols - colstart[m]) block, row-major, the groups one after the
// other.  Each GEMM output (r, c) has exactly one slot, so the workspace has
// E_s elements, and a row's outputs are contiguous.
static std::vector<int64_t> group_bases(const UpdateTables& t)
{
    const int nbar = (int)t.colstart.size();
    const int64_t ncols = (int64_t)t.colvar.size();
    std::vector<int64_t> gbase(nbar + 1, 0);
    for (int m = 0; m < nbar; ++m)
        gbase[m + 1] = gbase[m] + (int64_t)(t.rowstart[m + 1] - t.rowstart[m]) * (ncols - t.colstart[m]);
    return gbase;
}

std::vector<int64_t> build_w_rows(const UpdateTables& t)
{
    const int nbar = (int)t.colstart.size();
    const int64_t ncols = (int64_t)t.colvar.size();
    const std::vector<int64_t> gbase = group_bases(t);
    std::vector<int64_t> roww(t.rowvar.size());
    for (int m = 0; m < nbar; ++m) {
        const int64_t width = ncols - t.colstart[m];
        for (int r = t.rowstart[m]; r < t.rowstart[m + 1]; ++r)
            roww[r] = gbase[m] + (int64_t)(r - t.rowstart[m]) * width - t.colstart[m];
    }
    return roww;
}

std::vector<int32_t> build_w_blocks(const UpdateTables& t, int n, int b)
{
    const int nbar = (n + b - 1) / b;
    const int s = t.s, h = t.h, sh = t.sh;
    const int64_t ncols = (int64_t)t.colvar.size();
    const std::vector<int64_t> gbase = group_bases(t);
    const std::vector<int> blocks = enumerate_sorted(nbar, s);
    const int64_t nb = (int64_t)blocks.size() / s;
    std::vector<int32_t> out((size_t)nb * 2);
    for (int64_t q = 0; q < nb; ++q) {
        const int* j = &blocks[q * s];
        const int m = j[h - 1];
        const int64_t r0 = t.leftrow[rank_sorted(j, h, nbar)];
        const int64_t c0 = sh == 0 ? 0 : t.rightcol[rank_sorted(j + h, sh, nbar)];
        const int64_t width = ncols - t.colstart[m];
        out[2 * q] = (int32_t)(gbase[m] + (r0 - t.rowstart[m]) * width + (c0 - t.colstart[m]));
        out[2 * q + 1] = (int32_t)width;
    }
    return out;
}

CumTables build_cum_tables(int n, int b, int s)
{
    CumTables t;
    const int nbar = (n + b - 1) / b;
    t.s = s;
    const unsigned full = (1u << s) - 1u;
    for (unsigned A = 1; A < full; ++A)
        if (A & 1u) t.masks.push_back((uint8_t)A);
    t.nsub = (int)t.masks.size();
    const std::vector<int> blocks = enumerate_sorted(nbar, s);
    const int64_t nb = (int64_t)blocks.size() / s;
    t.subrank.resize((size_t)nb * t.nsub * 2);
    t.mult.resize(nb);
    int ja[kMaxOrder], jc[kMaxOrder];
    for (int64_t q = 0; q < nb; ++q) {
        const int* j = &blocks[q * s];
        t.mult[q] = block_multiplicity(j, s);
        for (int u = 0; u < t.nsub; ++u) {
            int na = 0, nc = 0;
            for (int k = 0; k < s; ++k) {
                if ((t.masks[u] >> k) & 1u) ja[na++] = j[k];
                else jc[nc++] = j[k];
            }
            t.subrank[((size_t)q * t.nsub + u) * 2 + 0] = (int32_t)rank_sorted(ja, na, nbar);
            t.subrank[((size_t)q * t.nsub + u) * 2 + 1] = (int32_t)rank_sorted(jc, nc, nbar);
        }
    }
    return t;
}

void shard_blocks(int nbar, int s, int shard, int nshards, int64_t* begin, int64_t* end)
{
    const int64_t nb = n_sorted(nbar, s);
    *begin = nb * shard / nshards;
    *end = nb * (shard + 1) / nshards;
}

CanonTables build_canon_tables(int n, int b, int s, int slice, int group, int64_t blk0, int64_t blk1)
{
    CanonTables t;
    const int nbar = (n + b - 1) / b;
    const int64_t bs = ipow(b, s);
    t.s = s;
    t.bs = (int)bs;
    const std::vector<int> blocks = enumerate_sorted(nbar, s);
    const int64_t nb = (int64_t)blocks.size() / s;
    // patterns: run-length compositions of s, as bit masks of "same block as the
    // previous position" (bit k set: j[k] == j[k-1])
    std::vector<int> pat_of_mask(1 << kMaxOrder, -1), masks;
    t.blkpat.resize(nb);
    for (int64_t q = 0; q < nb; ++q) {
        const int* j = &blocks[q * s];
        int m = 0;
        for (int k = 1; k < s; ++k)
            if (j[k] == j[k - 1]) m |= 1 << k;
        if (pat_of_mask[m] < 0) {
            pat_of_mask[m] = (int)masks.size();
            masks.push_back(m);
        }
        t.blkpat[q] = pat_of_mask[m];
    }
    t.npat = (int)masks.size();
    t.can_start.assign(t.npat + 1, 0);
    t.map_off.assign((size_t)t.npat * bs, 0);
    if (blk1 < 0 || blk1 > nb) blk1 = nb;
    blk0 = std::max<int64_t>(0, std::min(blk0, blk1));
    auto owned = [&](int64_t q) { return q >= blk0 && q < blk1; };
    std::vector<int64_t> count(t.npat, 0);
    for (int64_t q = 0; q < nb; ++q)
        if (owned(q)) count[t.blkpat[q]]++;
    for (int q = 0; q < t.npat; ++q) {
        const int m = masks[q];
        t.can_start[q] = (int32_t)t.can_off.size();
        int dig[kMaxOrder];
        for (int64_t o = 0; o < bs; ++o) {
            int64_t rem = o;
            for (int k = s - 1; k >= 0; --k) {
                dig[k] = (int)(rem % b);
                rem /= b;
            }
            // sort the digits inside each run (positions k-1, k with bit k set)
            for (int k0 = 0; k0 < s;) {
                int k1 = k0 + 1;
                while (k1 < s && ((m >> k1) & 1)) ++k1;
                std::sort(dig + k0, dig + k1);
                k0 = k1;
            }
            int64_t co = 0;
            for (int k = 0; k < s; ++k) co = co * b + dig[k];
            t.map_off[(size_t)q * bs + o] = (int32_t)co;
            if (co == o) t.can_off.push_back((int32_t)o);
        }
        t.can_start[q + 1] = (int32_t)t.can_off.size();
        // copies per canonical offset, and the non-canonical offsets with their source
        t.dup_start.push_back((int32_t)(t.dup.size() / 2));
        std::vector<int32_t> copies(bs, 0);
        for (int64_t o = 0; o < bs; ++o) {
            const int32_t co = t.map_off[(size_t)q * bs + o];
            copies[co]++;
            if (co != o) {
                t.dup.push_back((int32_t)o);
                t.dup.push_back(co);
            }
        }
        for (int c = t.can_start[q]; c < t.can_start[q + 1]; ++c) t.can_copies.push_back(copies[t.can_off[c]]);
        // ranks of the left / right digits inside the halves' own runs (compressed
        // update tables); a canonical offset is canonical in each half
        const int h = split_rows(s);
        const int64_t bsh = ipow(b, s - h);
        const std::vector<int32_t> lr = half_ranks(b, h, m & ((1 << h) - 1));
        const std::vector<int32_t> rr = half_ranks(b, s - h, (m >> h) & ~1);
        std::vector<int32_t> lr_of(bs, -1);
        for (int c = t.can_start[q]; c < t.can_start[q + 1]; ++c) {
            const int64_t o = t.can_off[c];
            const int32_t rl = lr[o / bsh], rc = rr[o % bsh];
            lr_of[o] = rl < 0 || rc < 0 ? -1 : (rl << 16) | rc;
            t.can_lr.push_back(lr_of[o]);
        }
        t.map_lr.resize((size_t)(q + 1) * bs);
        for (int64_t o = 0; o < bs; ++o) t.map_lr[(size_t)q * bs + o] = lr_of[t.map_off[(size_t)q * bs + o]];
        t.canonical += count[q] * (t.can_start[q + 1] - t.can_start[q]);
    }
    t.dup_start.push_back((int32_t)(t.dup.size() / 2));
    // blocks grouped by pattern, and the work units
    std::vector<int64_t> pstart(t.npat + 1, 0);
    for (int q = 0; q < t.npat; ++q) pstart[q + 1] = pstart[q] + count[q];
    t.pblocks.resize(pstart[t.npat]);
    std::vector<int64_t> fill(pstart.begin(), pstart.end() - 1);
    for (int64_t q = 0; q < nb; ++q)
        if (owned(q)) t.pblocks[fill[t.blkpat[q]]++] = (int32_t)q;
    for (int q = 0; q < t.npat; ++q) {
        const int nc = t.can_start[q + 1] - t.can_start[q];
        for (int sl = 0; sl * slice < nc; ++sl)
            for (int64_t g = pstart[q]; g < pstart[q + 1]; g += group) {
                t.units.push_back(q);
                t.units.push_back(sl);
                t.units.push_back((int32_t)g);
                t.units.push_back((int32_t)std::min<int64_t>(group, pstart[q + 1] - g));
            }
    }
    return t;
}

}  // namespace cw
