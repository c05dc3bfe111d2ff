// Host-side block-layout arithmetic and table generation.
//
// Block structure of Section 2.3 / Algorithm 5: sorted block multi-indices
// j1 <= ... <= js over nbar = ceil(n/b) blocks per mode, lexicographic order,
// each block a dense b^s array (a1 slowest).
#pragma once

#include <cstdint>
#include <vector>

namespace cw {

int64_t binom(int64_t n, int64_t k);
// Number of sorted s-tuples over [0, nbar).
int64_t n_sorted(int nbar, int s);
// Lexicographic rank of a sorted s-tuple over [0, nbar); -1 if invalid.
int64_t rank_sorted(const int* j, int s, int nbar);
// All sorted s-tuples over [0, nbar) in lexicographic order, flattened.
std::vector<int> enumerate_sorted(int nbar, int s);
// Block multiplicity s!/prod r_l! (Algorithm 5), r_l the runs of equal entries.
double block_multiplicity(const int* j, int s);
int64_t ipow(int64_t b, int e);

// Runs of equal entries of a sorted k-tuple as a bit mask: bit i (i >= 1)
// set when j[i] == j[i-1].
int run_mask(const int* j, int k);
// Rank of every k-digit in-block offset (digits base b, the first slowest)
// among the offsets whose digits do not decrease inside the runs of `mask`,
// in increasing order; -1 for the other offsets.
std::vector<int32_t> half_ranks(int b, int k, int mask);

// Tables of the order-s update GEMMs (see UpdateArgs in cw_internal.h).
// compressed: a left tuple jL keeps only the rows whose digits do not
// decrease inside its own runs of equal block indices, a right tuple only
// such columns.  Every canonical element of the order (CanonTables) is still
// produced once, the other elements of diagonal blocks mostly not.
struct UpdateTables {
    int s = 0, h = 0, sh = 0;
    bool compressed = false;
    std::vector<uint32_t> rowvar, colvar;
    std::vector<int64_t> rowoff, coloff;
    std::vector<int32_t> rowstart;  // [nbar + 1] rows of group m
    std::vector<int32_t> colstart;  // [nbar] first column of group m
    std::vector<int32_t> leftrow;   // [sorted h-tuples, lexicographic] first row of the tuple
    std::vector<int32_t> leftcnt;   // [sorted h-tuples] rows of the tuple
    std::vector<int32_t> rightcol;  // [sorted (s-h)-tuples, lexicographic] first column of the tuple
    int64_t wsize = 0;              // workspace slots (GEMM outputs) of the order
};
UpdateTables build_update_tables(int n, int b, int s, bool compressed = false);

// Workspace ("GEMM") order of the order-s update outputs: group m of the
// update is a dense row-major block of rows_m x (ncols - colstart[m]) slots.
// Slot of output (r, c) = roww[r] + c.
std::vector<int64_t> build_w_rows(const UpdateTables& t);
// Per sorted block j of order s (lexicographic rank): {slot of its first row
// and column, row stride}; in-block offset a = aL * b^sh + aR lives at
// slot + rL * stride + rR, with (rL, rR) = (aL, aR) for full tables and the
// ranks of aL and aR (half_ranks of the left and right tuples' runs) for
// compressed ones.
std::vector<int32_t> build_w_blocks(const UpdateTables& t, int n, int b);

// Tables of the order-s cumulant recovery (see CumArgs in cw_internal.h).
struct CumTables {
    int s = 0, nsub = 0;
    std::vector<uint8_t> masks;      // [nsub]
    std::vector<int32_t> subrank;    // [nblocks][nsub][2]
    std::vector<double> mult;        // [nblocks]
};
CumTables build_cum_tables(int n, int b, int s);

// Canonical elements of order s (the recovery computes one element per class
// of entries that super-symmetry makes equal).  A block j whose sorted block
// indices form runs of equal values (lengths r_1..r_k, its "pattern") stores,
// for in-block digits that differ only by a permutation inside a run, the same
// tensor entry several times (Section 2.3 keeps diagonal blocks whole).  The
// canonical offset of a class has its digits non-decreasing inside every run.
struct CanonTables {
    int s = 0, bs = 0, npat = 0;
    std::vector<int32_t> blkpat;     // [nblocks] pattern of each block
    std::vector<int32_t> can_start;  // [npat + 1] canonical offsets of pattern q at can_off[can_start[q]..]
    std::vector<int32_t> can_off;    // canonical in-block offsets, increasing, per pattern
    std::vector<int32_t> map_off;    // [npat][bs] canonical offset of each in-block offset
    std::vector<int32_t> can_copies; // per canonical offset: the offsets of its block holding the same entry
    std::vector<int32_t> dup_start;  // [npat + 1] non-canonical offsets of pattern q at dup[dup_start[q]..]
    std::vector<int32_t> dup;        // pairs {offset, its canonical offset}, per pattern
    std::vector<int32_t> pblocks;    // block ranks grouped by pattern (pattern order, then rank)
    std::vector<int32_t> units;      // [nunits][4] {pattern, slice, first index into pblocks, blocks}
    // workspace position of a canonical offset in the compressed update
    // tables: (rank of its left digits) << 16 | (rank of its right digits)
    std::vector<int32_t> can_lr;     // per canonical offset (as can_off)
    std::vector<int32_t> map_lr;     // [npat][bs]: can_lr of each offset's canonical offset
    int64_t canonical = 0;           // canonical elements of the order (all blocks)
};
// Units of `slice` threads x up to `group` blocks of one pattern, over the
// blocks of lexicographic rank in [blk0, blk1) (blk1 < 0: all blocks).
CanonTables build_canon_tables(int n, int b, int s, int slice, int group, int64_t blk0 = 0, int64_t blk1 = -1);

// Block range [begin, end) of shard `shard` of `nshards` over the sorted blocks
// of order s (contiguous in lexicographic order, balanced by block count).
void shard_blocks(int nbar, int s, int shard, int nshards, int64_t* begin, int64_t* end);

// Split of order s into row factors (h) and column factors (s - h).
inline int split_rows(int s) { return (s + 1) / 2; }

}  // namespace cw
