"""Pins for the CPU oracle: it is checked against things other than itself.

* exact cumulants of tiny integer windows from the cumulant-generating
  function K(u) = log (1/T) sum_t exp(u . x_t), expanded as a truncated power
  series in exact rationals (the textbook definition of cumulants);
* the paper's worked order-3 identity (Section 2.6, beside eq. n1);
* closed forms (mean, biased covariance, third central moment, the fourth
  cumulant through pairings, univariate skewness / kurtosis and kappa5/6);
* exact invariants of empirical cumulants (super-symmetry, translation,
  multilinearity, additivity on product-measure windows);
* partition counts (eq. n1), block multiplicities (Algorithm 5), the norm of
  Eq. me, and statistical behaviour on Gaussian and ICA data;
* the closed-form gradient against central finite differences.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# exact cumulants from the cumulant-generating function
# ----------------------------------------------------------------------------

def _poly_mul(p, q, n, D):
    out = {}
    for a, ca in p.items():
        da = sum(a)
        for b, cb in q.items():
            if da + sum(b) > D:
                continue
            k = tuple(x + y for x, y in zip(a, b))
            out[k] = out.get(k, 0) + ca * cb
    return out


def cgf_cumulants(X_int, D):
    """Exact cumulants kappa_alpha (|alpha| <= D) of the empirical law of the rows."""
    T, n = X_int.shape
    monos = [a for deg in range(D + 1) for a in itertools.product(range(deg + 1), repeat=n)
             if sum(a) == deg]
    monos = sorted(set(monos))
    mgf = {}
    for a in monos:
        fact = 1
        for ai in a:
            fact *= math.factorial(ai)
        acc = Fraction(0)
        for t in range(T):
            v = 1
            for i, ai in enumerate(a):
                v *= int(X_int[t, i]) ** ai
            acc += v
        mgf[a] = acc / (T * fact)
    zero = (0,) * n
    Q = {a: c for a, c in mgf.items() if a != zero}
    K = {}
    Qk = {zero: Fraction(1)}
    for k in range(1, D + 1):
        Qk = _poly_mul(Qk, Q, n, D)
        for a, c in Qk.items():
            K[a] = K.get(a, 0) + Fraction((-1) ** (k + 1), k) * c
    kappa = {}
    for a, c in K.items():
        fact = 1
        for ai in a:
            fact *= math.factorial(ai)
        kappa[a] = c * fact
    return kappa


@pytest.mark.parametrize("seed,n,T,D", [(0, 1, 7, 6), (1, 2, 9, 5), (2, 3, 12, 4), (3, 3, 5, 5),
                                         (4, 2, 12, 6)])
def test_integer_window_matches_cgf_exactly(seed, n, T, D):
    rng = np.random.default_rng(seed)
    X = rng.integers(-3, 4, size=(T, n))
    kappa = cgf_cumulants(X, D)
    for s in range(1, D + 1):
        tup = np.array(list(itertools.combinations_with_replacement(range(n), s)))
        got = oracle.cumulant_tuples(X, tup)
        for t, g in zip(tup, got):
            alpha = tuple(int(np.sum(t == i)) for i in range(n))
            exact = float(kappa.get(alpha, 0))
            assert abs(g - exact) <= 1e-12 * max(1.0, abs(exact)), (s, t, g, exact)


def test_order3_worked_identity():
    """c_123 = m_123 - c_12 c_3 - c_13 c_2 - c_23 c_1 - c_1 c_2 c_3."""
    with open(os.path.join(GOLDEN, "order3_partitions.json")) as f:
        gold = json.load(f)
    assert len(gold["partitions_into"]["2"]) == oracle.stirling2(3, 2)
    assert len(gold["partitions_into"]["3"]) == oracle.stirling2(3, 3)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((500, 3)) + np.array([1.0, -2.0, 0.5])
    X[:, 1] += 0.3 * X[:, 0] ** 2
    c1 = oracle.cumulant_tuples(X, [[0], [1], [2]])
    c12, c13, c23 = oracle.cumulant_tuples(X, [[0, 1], [0, 2], [1, 2]])
    c123 = oracle.cumulant_tuples(X, [[0, 1, 2]])[0]
    m123 = np.mean(X[:, 0] * X[:, 1] * X[:, 2])
    vals = {"m123": m123, "c12": c12, "c13": c13, "c23": c23,
            "c1": c1[0], "c2": c1[1], "c3": c1[2]}
    rhs = sum(term["sign"] * np.prod([vals[k] for k in term["factors"]])
              for term in gold["identity_terms"])
    assert abs(c123 - rhs) < 1e-12 * max(1.0, abs(m123))


# ----------------------------------------------------------------------------
# closed forms
# ----------------------------------------------------------------------------

def test_closed_forms_orders_1_to_4():
    rng = np.random.default_rng(11)
    n, b, T = 5, 2, 400
    X = rng.exponential(size=(T, n)) @ rng.standard_normal((n, n))
    C = oracle.cumulants(X, 4, b)
    full = [oracle.to_full(C[s - 1], n, b, s) for s in range(1, 5)]
    assert np.allclose(full[0], X.mean(axis=0), rtol=1e-13, atol=1e-13)
    assert np.allclose(full[1], np.cov(X.T, bias=True), rtol=1e-12, atol=1e-12)
    Y = X - X.mean(axis=0)
    m3 = np.einsum("ti,tj,tk->ijk", Y, Y, Y) / T
    assert np.allclose(full[2], m3, rtol=1e-11, atol=1e-11)
    m2 = Y.T @ Y / T
    m4 = np.einsum("ti,tj,tk,tl->ijkl", Y, Y, Y, Y) / T
    c4 = m4 - (np.einsum("ij,kl->ijkl", m2, m2) + np.einsum("ik,jl->ijkl", m2, m2)
               + np.einsum("il,jk->ijkl", m2, m2))
    assert np.allclose(full[3], c4, rtol=1e-10, atol=1e-10 * np.abs(m4).max())


def test_univariate_nu_and_kappa5_6():
    rng = np.random.default_rng(3)
    x = rng.gamma(2.0, size=5000)
    X = x[:, None]
    fro, nu = oracle.norms(X, 6)
    assert abs(nu[2] - abs(stats.skew(x, bias=True))) < 1e-10
    assert abs(nu[3] - abs(stats.kurtosis(x, fisher=True, bias=True))) < 1e-10
    m = {k: stats.moment(x, k) for k in range(2, 7)}
    k5 = m[5] - 10 * m[3] * m[2]
    k6 = m[6] - 15 * m[4] * m[2] - 10 * m[3] ** 2 + 30 * m[2] ** 3
    g5 = oracle.cumulant_tuples(X, [[0] * 5])[0]
    g6 = oracle.cumulant_tuples(X, [[0] * 6])[0]
    assert abs(g5 - k5) < 1e-9 * abs(m[5]) and abs(g6 - k6) < 1e-9 * abs(m[6])


def test_raw_moment_order2_is_gram():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((300, 4)) + 2.0
    tup = np.array(list(itertools.product(range(4), repeat=2)))
    got = oracle.moment_tuples(X, tup).reshape(4, 4)
    assert np.allclose(got, X.T @ X / 300, rtol=1e-13)


# ----------------------------------------------------------------------------
# invariants
# ----------------------------------------------------------------------------

def test_super_symmetry_all_permutations():
    rng = np.random.default_rng(2)
    X = rng.standard_t(5, size=(700, 4)) @ rng.standard_normal((4, 4))
    for s in (3, 4, 5):
        base = oracle.sample_sorted_tuples(4, s, 12, seed=s)
        for t in base:
            perms = np.array(sorted(set(itertools.permutations(t))))
            vals = oracle.cumulant_tuples(X, perms)
            assert np.ptp(vals) <= 1e-12 * max(1.0, np.abs(vals).max())


def test_translation_and_multilinearity():
    rng = np.random.default_rng(9)
    n, b, T = 3, 2, 600
    X = rng.gamma(1.5, size=(T, n))
    A = rng.standard_normal((n, n))
    shift = np.array([3.0, -7.0, 0.25])
    CX = oracle.cumulants(X, 5, b)
    CS = oracle.cumulants(X + shift, 5, b)
    CA = oracle.cumulants(X @ A, 5, b)
    assert np.allclose(CS[0], CX[0] + np.concatenate([shift, [0.0]]), atol=1e-12)
    for s in range(2, 6):
        scale = np.abs(CX[s - 1]).max()
        assert np.allclose(CS[s - 1], CX[s - 1], atol=1e-9 * scale)
        full = oracle.to_full(CX[s - 1], n, b, s)
        letters = "abcdefg"[:s]
        upper = "ABCDEFG"[:s]
        spec = letters + "," + ",".join(f"{l}{u}" for l, u in zip(letters, upper)) + "->" + upper
        expect = np.einsum(spec, full, *([A] * s))
        got = oracle.to_full(CA[s - 1], n, b, s)
        assert np.allclose(got, expect, atol=1e-9 * np.abs(expect).max())


def test_exact_additivity_on_product_windows():
    """A window holding every pair (x_i, y_j) is an empirical product measure:
    the cumulants of x + y are exactly the sums of those of x and y."""
    rng = np.random.default_rng(4)
    n = 3
    xs = rng.gamma(2.0, size=(17, n))
    ys = rng.standard_t(6, size=(13, n))
    W = (xs[:, None, :] + ys[None, :, :]).reshape(-1, n)
    for s in range(2, 6):
        tup = np.array(list(itertools.combinations_with_replacement(range(n), s)))
        lhs = oracle.cumulant_tuples(W, tup)
        rhs = oracle.cumulant_tuples(xs, tup) + oracle.cumulant_tuples(ys, tup)
        assert np.allclose(lhs, rhs, atol=1e-10 * np.abs(rhs).max())


def test_padding_when_block_does_not_divide_n():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((100, 5))
    C3 = oracle.cumulants(X, 3, 2)[2]
    idx = oracle.block_elements(5, 2, 3)
    pad = np.any(idx >= 5, axis=1)
    assert pad.any() and np.all(C3[pad] == 0.0)


# ----------------------------------------------------------------------------
# counts, layout, norms
# ----------------------------------------------------------------------------

def test_partition_counts_eq_n1():
    with open(os.path.join(GOLDEN, "eq_n1_counts.json")) as f:
        gold = json.load(f)
    for d, bell in gold["bell"].items():
        assert oracle.count_partitions(int(d)) == bell
    for d, row in gold["stirling2"].items():
        for sig, v in row.items():
            assert oracle.stirling2(int(d), int(sig)) == v
    for d, mults in gold["multiplications"].items():
        d = int(d)
        assert sum(oracle.stirling2(d, sg) * (sg - 1) for sg in range(1, d + 1)) == mults
        assert mults <= (d - 1) * oracle.count_partitions(d)


def test_block_multiplicity_rule():
    with open(os.path.join(GOLDEN, "block_multiplicity.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        assert oracle.block_multiplicity(tuple(case["j"])) == case["multiplicity"]


@pytest.mark.parametrize("n,b,s", [(4, 2, 4), (5, 2, 3), (6, 3, 3), (3, 4, 2)])
def test_block_multiplicities_cover_full_tensor(n, b, s):
    nb = oracle.nbar(n, b)
    tot = sum(oracle.block_multiplicity(j) for j in oracle.sorted_block_tuples(n, b, s))
    assert tot == nb ** s


def test_norm_block_weighted_equals_full_tensor():
    rng = np.random.default_rng(8)
    n, b = 5, 2
    X = rng.standard_t(4, size=(400, n)) @ rng.standard_normal((n, n))
    C = oracle.cumulants(X, 4, b)
    fro, nu = oracle.norms(X, 4)
    for s in range(1, 5):
        full = oracle.to_full(C[s - 1], n, b, s)
        assert abs(np.sqrt(np.sum(full ** 2)) - fro[s - 1]) <= 1e-12 * fro[s - 1]
        blocks = oracle.sorted_block_tuples(n, b, s)
        vals = C[s - 1].reshape(len(blocks), b ** s)
        z = sum(oracle.block_multiplicity(j) * np.sum(v ** 2) for j, v in zip(blocks, vals))
        assert abs(math.sqrt(z) - fro[s - 1]) <= 1e-12 * fro[s - 1]
    assert abs(nu[3] - fro[3] / fro[1] ** 2) < 1e-14 and np.isnan(nu[0])


@pytest.mark.parametrize("k", [1.0, 1.5, 3.0, 4.0])
def test_k_norms_equal_the_full_tensor_sums(k):
    """Eq. me with a general k: the permutation-weighted sum over sorted tuples
    equals the entry-wise sum over the full tensor (expanded from the blocks),
    k = 2 is the Frobenius norm, and a single variable gives |kappa_s|."""
    rng = np.random.default_rng(81)
    n, b = 4, 3
    X = rng.gamma(2.0, size=(300, n)) @ rng.standard_normal((n, n))
    C = oracle.cumulants(X, 4, b)
    got = oracle.norms_k(X, 4, k)
    for s in range(1, 5):
        full = oracle.to_full(C[s - 1], n, b, s)
        want = float(np.sum(np.abs(full) ** k)) ** (1.0 / k)
        assert abs(got[s - 1] - want) <= 1e-12 * want
    fro, _ = oracle.norms(X, 4)
    np.testing.assert_allclose(oracle.norms_k(X, 4, 2.0), fro, rtol=1e-13)
    x = rng.exponential(size=(500, 1))
    cum = [float(oracle.cumulants(x, 4, 1)[s - 1][0]) for s in range(1, 5)]
    np.testing.assert_allclose(oracle.norms_k(x, 4, k), np.abs(cum), rtol=1e-13)


# ----------------------------------------------------------------------------
# statistical behaviour
# ----------------------------------------------------------------------------

def test_gaussian_high_orders_vanish_like_root_T():
    n = 3
    for seed in range(3):
        rng = np.random.default_rng(100 + seed)
        for T in (2000, 32000):
            X = rng.standard_normal((T, n))
            fro, _ = oracle.norms(X, 5)
            for s in (3, 4, 5):
                # standard error of an order-s moment of N(0,1) is sqrt(m_2s / T)
                m2s = math.prod(range(1, 2 * s, 2))
                assert fro[s - 1] < 4.0 * n ** (s / 2) * math.sqrt(m2s / T)


def test_ica_population_fourth_cumulant_norm():
    n = 8
    rng = np.random.default_rng(5)
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    U = rng.uniform(-math.sqrt(3), math.sqrt(3), size=(1 << 17, n))
    X = U @ Q.T
    fro, _ = oracle.norms(X, 4)
    # orthogonal mixing keeps ||C4||_F^2 = sum_k kappa4^2 = n (6/5)^2
    assert abs(fro[3] ** 2 - n * 1.44) < 0.05 * n * 1.44
    # C3 = 0 in population; each empirical entry has standard error ~ 1/sqrt(T)
    assert fro[2] < 3.0 * n ** 1.5 / math.sqrt(X.shape[0])


# ----------------------------------------------------------------------------
# gradient
# ----------------------------------------------------------------------------

def test_grad_closed_form_vs_finite_differences():
    rng = np.random.default_rng(12)
    T, n = 60, 3
    X = rng.uniform(-1.7, 1.7, size=(T, n)) @ rng.standard_normal((n, n))
    w = [0.0, 0.3, 0.7, 1.0, 1.0]
    g = oracle.grad(X, w)
    h = 1e-4
    for (t, a) in [(0, 0), (5, 1), (17, 2), (59, 0), (33, 1)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[t, a] += h
        Xm[t, a] -= h
        fd = (oracle.loss(Xp, w) - oracle.loss(Xm, w)) / (2 * h)
        assert abs(fd - g[t, a]) < 1e-6 * max(1.0, abs(fd))


def test_grad_invariants():
    rng = np.random.default_rng(13)
    X = rng.uniform(-1.7, 1.7, size=(200, 4)) @ rng.standard_normal((4, 4))
    w = [0.0, 0.0, 0.0, 1.0, 1.0]
    g = oracle.grad(X, w)
    assert np.allclose(g.sum(axis=0), 0.0, atol=1e-12 * np.abs(g).max() * 200)
    fro, _ = oracle.norms(X, 4)
    euler = sum(2 * s * w[s] * fro[s - 1] ** 2 for s in range(1, 5))
    assert abs(np.sum(X * g) - euler) < 1e-9 * euler


def test_storage_index_agrees_with_enumerated_layout():
    for n, b, s in [(7, 3, 4), (5, 2, 3), (4, 4, 5), (6, 1, 3)]:
        idx = oracle.block_elements(n, b, s)
        keep = np.all(idx < n, axis=1)
        for e in np.nonzero(keep)[0]:
            g = oracle.storage_index(n, b, idx[e])
            assert np.array_equal(np.sort(idx[g]), np.sort(idx[e]))


# ----------------------------------------------------------------------------
# moments -> cumulants (Algorithms 3-4)
# ----------------------------------------------------------------------------

def test_set_partitions_are_the_bell_numbers_of_eq_n1():
    with open(os.path.join(GOLDEN, "eq_n1_counts.json")) as f:
        gold = json.load(f)
    for d, bell in gold["bell"].items():
        parts = list(oracle.set_partitions(range(int(d))))
        assert len(parts) == bell
        seen = set()
        for p in parts:  # each a partition of 0..d-1, no duplicates
            assert sorted(x for blk in p for x in blk) == list(range(int(d)))
            key = frozenset(frozenset(blk) for blk in p)
            assert key not in seen
            seen.add(key)


@pytest.mark.parametrize("seed,n,T,D", [(5, 2, 9, 5), (6, 3, 11, 4), (7, 1, 8, 6)])
def test_moms2cums_matches_cgf_on_integer_windows(seed, n, T, D):
    """Algorithms 3-4 on the window's raw moments give the exact cumulants of
    the cumulant-generating function."""
    rng = np.random.default_rng(seed)
    X = rng.integers(-3, 4, size=(T, n)).astype(np.float64)
    kappa = cgf_cumulants(X.astype(np.int64), D)
    b = 2
    M = oracle.moments(X, D, b)
    for s in range(1, D + 1):
        tup = np.array(list(itertools.combinations_with_replacement(range(n), s)), dtype=np.int32)
        got = oracle.moms2cums_tuples(M, n, b, tup)
        want = np.array([float(kappa[tuple(int(np.sum(t == i)) for i in range(n))]) for t in tup])
        assert np.allclose(got, want, rtol=1e-9, atol=1e-9 * max(1.0, np.abs(want).max()))
