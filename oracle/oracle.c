/*
 * Oracle for the sliding-window cumulant library: a plain, slow FP64 CPU
 * implementation of the empirical cumulant tensors of a data window.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * What it computes (Section 2.4, Eq. 5: moments carry the 1/t normalisation):
 *   mu_i          = (1/t) sum_l x_{l,i}                     (first cumulant)
 *   y_{l,i}       = x_{l,i} - mu_i                         (two-pass centring)
 *   mu_B[i_B]     = (1/t) sum_l prod_{k in B} y_{l,i_k}    (central moments)
 *   C_s[i]        = sum over set partitions pi of {1..s} whose blocks all
 *                   have size >= 2 of (-1)^{|pi|-1} (|pi|-1)! prod_B mu_B[i_B]
 * This is the recalculation route the paper contrasts its update with
 * (Section 2.6: central moments, partitions whose parts all have size >= 2),
 * i.e. the Moebius inversion of moments over the partition lattice with the
 * singleton parts dropped because central first moments vanish.  It loops
 * over index tuples and over the whole window: there is no sliding, no block
 * structure and no sub-tuple reuse.
 *
 * Raw moments (Eq. 5) are provided for the moment-sum parity tests.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_ORDER 8
#define ORC_MAX_PARTS 4140 /* Bell number B(8) */

/* One set partition of {0..s-1}: its blocks as bitmasks. */
typedef struct {
    int nblocks;
    unsigned masks[ORC_MAX_ORDER];
} orc_partition;

/*
 * Enumerate the set partitions of {0..s-1} through restricted growth strings
 * (a[0] = 0, a[k] <= 1 + max(a[0..k-1])), the enumeration the paper cites
 * for Algorithm 4 (Knuth, TAOCP 7.2.1.4).  Only partitions whose blocks all
 * hold at least `min_block` elements are written.  Returns their count.
 */
static int orc_enumerate_partitions(int s, int min_block, orc_partition* out)
{
    int a[ORC_MAX_ORDER];
    int count = 0;
    for (int k = 0; k < s; ++k) a[k] = 0;
    for (;;) {
        int nb = 0;
        for (int k = 0; k < s; ++k)
            if (a[k] + 1 > nb) nb = a[k] + 1;
        unsigned masks[ORC_MAX_ORDER];
        int sizes[ORC_MAX_ORDER];
        for (int q = 0; q < nb; ++q) { masks[q] = 0u; sizes[q] = 0; }
        for (int k = 0; k < s; ++k) { masks[a[k]] |= 1u << k; sizes[a[k]]++; }
        int ok = 1;
        for (int q = 0; q < nb; ++q)
            if (sizes[q] < min_block) ok = 0;
        if (ok) {
            out[count].nblocks = nb;
            for (int q = 0; q < nb; ++q) out[count].masks[q] = masks[q];
            count++;
        }
        /* next restricted growth string: increment the last position that
         * may still grow, reset everything after it */
        int k = s - 1;
        for (; k >= 1; --k) {
            int mx = 0;
            for (int q = 0; q < k; ++q)
                if (a[q] > mx) mx = a[q];
            if (a[k] <= mx) break;
        }
        if (k < 1) break;
        a[k]++;
        for (int q = k + 1; q < s; ++q) a[q] = 0;
    }
    return count;
}

/* Number of set partitions of {0..s-1} with all blocks of size >= min_block
 * (min_block = 1 gives the Bell numbers of eq. (n1)). */
int orc_count_partitions(int s, int min_block)
{
    if (s < 1 || s > ORC_MAX_ORDER) return -1;
    static orc_partition buf[ORC_MAX_PARTS];
    return orc_enumerate_partitions(s, min_block, buf);
}

/* Number of partitions of {0..s-1} into exactly `sigma` blocks (Stirling
 * numbers of the second kind, eq. (n1)). */
int orc_count_partitions_into(int s, int sigma)
{
    if (s < 1 || s > ORC_MAX_ORDER) return -1;
    static orc_partition buf[ORC_MAX_PARTS];
    int np = orc_enumerate_partitions(s, 1, buf);
    int c = 0;
    for (int q = 0; q < np; ++q)
        if (buf[q].nblocks == sigma) c++;
    return c;
}

/* Column means (Eq. 5 with s = 1) and the centred window, two passes. */
void orc_center(const double* X, int64_t T, int n, double* mu, double* Y)
{
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int64_t l = 0; l < T; ++l) acc += X[l * n + i];
        mu[i] = acc / (double)T;
    }
    for (int64_t l = 0; l < T; ++l)
        for (int i = 0; i < n; ++i) Y[l * n + i] = X[l * n + i] - mu[i];
}

/*
 * Cumulants of order s >= 2 at `ntup` index tuples (each s ints in [0,n),
 * any order), from the centred window Y (T x n, samples are rows, Eq. 1).
 * For each tuple every central moment mu_B, B a subset of the tuple's
 * positions with |B| >= 2, is the plain window mean of the product of the
 * entries of Y; the cumulant is the signed partition sum described above.
 */
void orc_cumulant_tuples(const double* Y, int64_t T, int n, int s,
                         int64_t ntup, const int32_t* tup, double* out)
{
    (void)n;
    static orc_partition parts[ORC_MAX_PARTS];
    int np = orc_enumerate_partitions(s, 2, parts);
    double coef[ORC_MAX_PARTS];
    for (int q = 0; q < np; ++q) {
        /* (-1)^{k-1} (k-1)! */
        int k = parts[q].nblocks;
        double f = 1.0;
        for (int r = 2; r < k; ++r) f *= (double)r;
        coef[q] = (k % 2 == 1) ? f : -f;
    }
    const unsigned nsub = 1u << s;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t u = 0; u < ntup; ++u) {
        const int32_t* idx = tup + u * s;
        double sums[1u << ORC_MAX_ORDER];
        double prod[1u << ORC_MAX_ORDER];
        for (unsigned B = 0; B < nsub; ++B) sums[B] = 0.0;
        prod[0] = 1.0;
        for (int64_t l = 0; l < T; ++l) {
            const double* row = Y + l * (int64_t)n;
            for (unsigned B = 1; B < nsub; ++B) {
                /* product over B = product over B without its lowest
                 * position, times the entry at that position */
                int k = __builtin_ctz(B);
                prod[B] = prod[B & (B - 1u)] * row[idx[k]];
                sums[B] += prod[B];
            }
        }
        double mom[1u << ORC_MAX_ORDER];
        for (unsigned B = 0; B < nsub; ++B) mom[B] = sums[B] / (double)T;
        double c = 0.0;
        for (int q = 0; q < np; ++q) {
            double term = coef[q];
            for (int r = 0; r < parts[q].nblocks; ++r) term *= mom[parts[q].masks[r]];
            c += term;
        }
        out[u] = c;
    }
}

/* Raw moments m_i = (1/t) sum_l prod_k x_{l,i_k} (Eq. 5) at index tuples. */
void orc_moment_tuples(const double* X, int64_t T, int n, int s,
                       int64_t ntup, const int32_t* tup, double* out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t u = 0; u < ntup; ++u) {
        const int32_t* idx = tup + u * s;
        double acc = 0.0;
        for (int64_t l = 0; l < T; ++l) {
            double p = 1.0;
            for (int k = 0; k < s; ++k) p *= X[l * (int64_t)n + idx[k]];
            acc += p;
        }
        out[u] = acc / (double)T;
    }
}

int orc_max_order(void) { return ORC_MAX_ORDER; }
