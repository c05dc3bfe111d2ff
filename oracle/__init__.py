"""Oracle: plain FP64 CPU reference for sliding-window cumulant tensors.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path: its block layout, its
partition enumeration and its arithmetic are written here independently.

Every quantity is recomputed from the whole window, in FP64:

* ``C_1`` is the column mean (Eq. 5 with s = 1, normalisation 1/t);
* ``C_s`` for s >= 2 is the signed sum over set partitions with all parts of
  size >= 2 of products of central moments, the recalculation route of
  Section 2.6, evaluated per index tuple by ``oracle.c``;
* the block layout is the one of Section 2.3 / Algorithm 5: only blocks
  ``j1 <= ... <= js`` are stored, in lexicographic order, each a dense
  ``b^s`` block, row-major with the first in-block index slowest; variables
  past ``n`` (when ``b`` does not divide ``n``) are zero padding;
* norms (Eq. me, k = 2) are the plain sum of squares over the full ``n^s``
  tensor, each sorted tuple counted once per distinct permutation, and
  ``nu_s`` follows Eq. mef;
* the gradient of ``sum_s w_s ||C_s||_F^2`` (orders 1..4) is the closed form
  through the centred data, derived by hand from ``C_2 = mu_2``,
  ``C_3 = mu_3`` and ``C_4 = mu_4 - (3 pairings of mu_2 x mu_2)``.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(brute-force cumulant-generating-function expansion in exact rationals,
closed forms, invariants, finite differences).
"""
from __future__ import annotations

import ctypes
import itertools
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_handle = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` (plain C, OpenMP) into ``liboracle.so``."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _handle
    with _lock:
        if _handle is None:
            build()
            lib = ctypes.CDLL(_SO)
            i64, i32, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            lib.orc_center.argtypes = [dp, i64, i32, dp, dp]
            lib.orc_cumulant_tuples.argtypes = [dp, i64, i32, i32, i64, dp, dp]
            lib.orc_moment_tuples.argtypes = [dp, i64, i32, i32, i64, dp, dp]
            lib.orc_count_partitions.argtypes = [i32, i32]
            lib.orc_count_partitions_into.argtypes = [i32, i32]
            _handle = lib
    return _handle


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ----------------------------------------------------------------------------
# partition counts (eq. n1)
# ----------------------------------------------------------------------------

def count_partitions(s: int, min_block: int = 1) -> int:
    """Set partitions of an s-set with every part of size >= min_block."""
    return int(_lib().orc_count_partitions(s, min_block))


def stirling2(s: int, sigma: int) -> int:
    """Partitions of an s-set into exactly sigma parts, by enumeration."""
    return int(_lib().orc_count_partitions_into(s, sigma))


# ----------------------------------------------------------------------------
# block layout (Section 2.3, Algorithm 5)
# ----------------------------------------------------------------------------

def nbar(n: int, b: int) -> int:
    return -(-n // b)


def sorted_block_tuples(n: int, b: int, s: int) -> list[tuple[int, ...]]:
    """All sorted block multi-indices j1 <= ... <= js, lexicographic order."""
    return list(itertools.combinations_with_replacement(range(nbar(n, b)), s))


def layout_size(n: int, b: int, s: int) -> int:
    return len(sorted_block_tuples(n, b, s)) * b ** s


def block_elements(n: int, b: int, s: int) -> np.ndarray:
    """Variable multi-index of every stored element of order s, shape (E_s, s).

    Element e = block_rank * b^s + offset, offset row-major over (a1..as) with
    a1 slowest; the variable index of position k is j_k * b + a_k.
    """
    blocks = np.array(sorted_block_tuples(n, b, s), dtype=np.int64).reshape(-1, s)
    inner = np.array(list(itertools.product(range(b), repeat=s)), dtype=np.int64).reshape(-1, s)
    idx = blocks[:, None, :] * b + inner[None, :, :]
    return idx.reshape(-1, s)


def storage_index(n: int, b: int, i) -> int:
    """Storage index of the tensor entry at variable multi-index i (its sorted form).

    The sorted block tuple j maps to strictly increasing c_k = j_k + k over
    [0, nbar + s - 1) (stars and bars); its lexicographic rank counts the
    combinations that first differ from c at some position k with a smaller
    value there.
    """
    v = sorted(int(x) for x in i)
    s = len(v)
    N = nbar(n, b) + s - 1
    c = [v[k] // b + k for k in range(s)]
    rank = 0
    lo = 0
    for k in range(s):
        for u in range(lo, c[k]):
            rank += math.comb(N - 1 - u, s - 1 - k)
        lo = c[k] + 1
    off = 0
    for k in range(s):
        off = off * b + v[k] % b
    return rank * b ** s + off


def block_multiplicity(j: tuple[int, ...]) -> int:
    """d! / prod_l r_l! with r_l the run lengths of equal indices (Algorithm 5)."""
    r = math.factorial(len(j))
    for _, grp in itertools.groupby(j):
        r //= math.factorial(len(list(grp)))
    return r


def tuple_permutations(i) -> int:
    """Number of distinct orderings of an index tuple (same rule, element level)."""
    return block_multiplicity(tuple(sorted(i)))


def to_full(block_vals: np.ndarray, n: int, b: int, s: int) -> np.ndarray:
    """Expand a block-layout super-symmetric tensor to its full n^s form."""
    idx = block_elements(n, b, s)
    full = np.full((n,) * s, np.nan)
    keep = np.all(idx < n, axis=1)
    for perm in itertools.permutations(range(s)):
        full[tuple(idx[keep][:, list(perm)].T)] = block_vals[keep]
    return full


def from_full(full: np.ndarray, n: int, b: int, s: int) -> np.ndarray:
    """Block layout of a full tensor (padding entries are zero)."""
    idx = block_elements(n, b, s)
    keep = np.all(idx < n, axis=1)
    out = np.zeros(idx.shape[0])
    out[keep] = full[tuple(idx[keep].T)]
    return out


# ----------------------------------------------------------------------------
# cumulants and moments
# ----------------------------------------------------------------------------

def _as_f64(X) -> np.ndarray:
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    if X.ndim != 2:
        raise ValueError("window must be T x n")
    return X


def center(X) -> tuple[np.ndarray, np.ndarray]:
    X = _as_f64(X)
    T, n = X.shape
    mu = np.empty(n)
    Y = np.empty_like(X)
    _lib().orc_center(_ptr(X), T, n, _ptr(mu), _ptr(Y))
    return mu, Y


def cumulant_tuples(X, tuples, *, centred=None) -> np.ndarray:
    """C_s at the given index tuples (shape (m, s)), all of one order s."""
    X = _as_f64(X)
    tup = np.ascontiguousarray(np.asarray(tuples, dtype=np.int32))
    if tup.ndim != 2:
        raise ValueError("tuples must be (m, s)")
    m, s = tup.shape
    T, n = X.shape
    mu, Y = centred if centred is not None else center(X)
    if s == 1:
        return mu[tup[:, 0]].copy()
    out = np.empty(m)
    if m:
        _lib().orc_cumulant_tuples(_ptr(Y), T, n, s, m, _ptr(tup), _ptr(out))
    return out


def moment_tuples(X, tuples) -> np.ndarray:
    """Raw moments (Eq. 5) at index tuples."""
    X = _as_f64(X)
    tup = np.ascontiguousarray(np.asarray(tuples, dtype=np.int32))
    m, s = tup.shape
    T, n = X.shape
    out = np.empty(m)
    if m:
        _lib().orc_moment_tuples(_ptr(X), T, n, s, m, _ptr(tup), _ptr(out))
    return out


def _block_eval(fn, X, n, b, s):
    idx = block_elements(n, b, s)
    keep = np.all(idx < n, axis=1)
    srt = np.sort(idx[keep], axis=1)
    uniq, inv = np.unique(srt, axis=0, return_inverse=True)
    vals = fn(uniq)
    out = np.zeros(idx.shape[0])
    out[keep] = vals[inv.reshape(-1)]
    return out


def cumulants(X, d: int, b: int) -> list[np.ndarray]:
    """[C_1, ..., C_d] of the window, each in block layout (FP64)."""
    X = _as_f64(X)
    n = X.shape[1]
    cen = center(X)
    return [_block_eval(lambda u: cumulant_tuples(X, u, centred=cen), X, n, b, s)
            for s in range(1, d + 1)]


def moments(X, d: int, b: int) -> list[np.ndarray]:
    """[M_1, ..., M_d] raw moments of the window in block layout (Eq. 5)."""
    X = _as_f64(X)
    n = X.shape[1]
    return [_block_eval(lambda u: moment_tuples(X, u), X, n, b, s) for s in range(1, d + 1)]


def sample_sorted_tuples(n: int, s: int, count: int, seed: int) -> np.ndarray:
    """`count` seeded random sorted index tuples of order s (with repetition)."""
    rng = np.random.default_rng(seed)
    t = np.sort(rng.integers(0, n, size=(count, s)), axis=1)
    return t.astype(np.int32)


# ----------------------------------------------------------------------------
# moments -> cumulants (Algorithms 3-4), from given moment tensors
# ----------------------------------------------------------------------------

def set_partitions(items):
    """All set partitions of the list `items` (each a list of blocks): the
    first item either forms a block of its own or joins one block of a
    partition of the rest."""
    items = list(items)
    if not items:
        yield []
        return
    first, rest = items[0], items[1:]
    for part in set_partitions(rest):
        yield [[first]] + part
        for k in range(len(part)):
            yield part[:k] + [[first] + part[k]] + part[k + 1:]


def moms2cums_tuples(M, n: int, b: int, tuples) -> np.ndarray:
    """Cumulants at index tuples (all of one order s) from moment tensors, by
    Algorithms 3-4: C_s(i) = M_s(i) - A(i), A(i) the sum over the set
    partitions of the s positions into at least two parts of the product of
    the lower-order cumulants at the parts' sub-tuples, those computed the
    same way (memoised).  M[k-1] is M_k in the block layout.  Orders >= 2 do
    not depend on the point the moments are taken about; C_1 = M_1 does."""
    memo = {}

    def cum(t):
        if t in memo:
            return memo[t]
        s = len(t)
        val = float(M[s - 1][storage_index(n, b, t)])
        for part in set_partitions(range(s)):
            if len(part) < 2:
                continue
            prod = 1.0
            for blk in part:
                prod *= cum(tuple(sorted(t[k] for k in blk)))
            val -= prod
        memo[t] = val
        return val

    return np.array([cum(tuple(sorted(int(x) for x in row))) for row in np.asarray(tuples)])


# ----------------------------------------------------------------------------
# norms and the non-Gaussianity estimator (Eqs. me, mef)
# ----------------------------------------------------------------------------

def norms(X, d: int) -> tuple[np.ndarray, np.ndarray]:
    """(||C_1||, ..., ||C_d||) Frobenius norms and (nu_1..nu_d), NaN below 3.

    The squared norm sums C[i]^2 over all n^s index tuples; each sorted tuple
    is evaluated once and counted once per distinct permutation.
    """
    X = _as_f64(X)
    n = X.shape[1]
    cen = center(X)
    fro = np.zeros(d)
    for s in range(1, d + 1):
        tup = np.array(list(itertools.combinations_with_replacement(range(n), s)), dtype=np.int32)
        vals = cumulant_tuples(X, tup, centred=cen)
        cnt = np.array([tuple_permutations(t) for t in tup], dtype=np.float64)
        fro[s - 1] = math.sqrt(float(np.sum(cnt * vals * vals)))
    nu = np.full(d, np.nan)
    for s in range(3, d + 1):
        with np.errstate(divide="ignore", invalid="ignore"):
            nu[s - 1] = fro[s - 1] / fro[1] ** (s / 2.0)
    return fro, nu


def norms_k(X, d: int, k: float) -> np.ndarray:
    """Entry-wise k-norms (sum over all n^s index tuples of |C[i]|^k)^(1/k), s = 1..d
    (Eq. me with a general k, Algorithm 5); each sorted tuple is evaluated once and
    counted once per distinct permutation."""
    X = _as_f64(X)
    n = X.shape[1]
    cen = center(X)
    out = np.zeros(d)
    for s in range(1, d + 1):
        tup = np.array(list(itertools.combinations_with_replacement(range(n), s)), dtype=np.int32)
        vals = cumulant_tuples(X, tup, centred=cen)
        cnt = np.array([tuple_permutations(t) for t in tup], dtype=np.float64)
        out[s - 1] = float(np.sum(cnt * np.abs(vals) ** k)) ** (1.0 / k)
    return out


# ----------------------------------------------------------------------------
# gradient of L = sum_s w_s ||C_s||_F^2 (orders 1..4), closed form
# ----------------------------------------------------------------------------

def _kr(Y: np.ndarray, k: int) -> np.ndarray:
    """Row-wise Kronecker power: row t holds y_t (x) ... (x) y_t (k factors), first slowest."""
    out = np.ones((Y.shape[0], 1))
    for _ in range(k):
        out = (out[:, :, None] * Y[:, None, :]).reshape(Y.shape[0], -1)
    return out


def full_central_moments(Y: np.ndarray, s: int, chunk: int = 512) -> np.ndarray:
    """Full central-moment tensor mu_s = (1/T) sum_t y_t^{(x)s}, as the product of
    the Kronecker powers of orders floor(s/2) and ceil(s/2), summed over row chunks."""
    T, n = Y.shape
    s1 = s // 2
    acc = np.zeros((n ** s1, n ** (s - s1)))
    for t0 in range(0, T, chunk):
        Yc = Y[t0:t0 + chunk]
        acc += _kr(Yc, s1).T @ _kr(Yc, s - s1)
    return (acc / T).reshape((n,) * s)


def _contract_rows(Y: np.ndarray, Cfull: np.ndarray, chunk: int = 512) -> np.ndarray:
    """out[t, a] = sum_{i2..is} C[a, i2..is] y_{t,i2} ... y_{t,is} (row chunks)."""
    T, n = Y.shape
    k = Cfull.ndim - 1
    Cm = Cfull.reshape(n, n ** k)
    out = np.empty((T, n))
    for t0 in range(0, T, chunk):
        out[t0:t0 + chunk] = _kr(Y[t0:t0 + chunk], k) @ Cm.T
    return out


def full_cumulants_closed_form(X, d: int) -> list[np.ndarray]:
    """Full C_1..C_d for d <= 4 by the closed forms in central moments."""
    if d > 4:
        raise ValueError("closed forms are written for orders <= 4")
    mu, Y = center(X)
    out = [mu]
    if d >= 2:
        out.append(full_central_moments(Y, 2))
    if d >= 3:
        out.append(full_central_moments(Y, 3))
    if d >= 4:
        m2 = out[1]
        m4 = full_central_moments(Y, 4)
        pair = (m2[:, :, None, None] * m2[None, None, :, :] + m2[:, None, :, None] * m2[None, :, None, :]
                + m2[:, None, None, :] * m2[None, :, :, None])
        out.append(m4 - pair)
    return out


def loss(X, w) -> float:
    """L = sum_s w[s] ||C_s||_F^2 from the tuple-evaluated cumulants."""
    d = len(w) - 1
    fro, _ = norms(X, d)
    return float(sum(w[s] * fro[s - 1] ** 2 for s in range(1, d + 1)))


def grad(X, w) -> np.ndarray:
    """dL/dX for L = sum_{s=1..4} w[s] ||C_s||_F^2, w indexed by order (w[0] unused).

    L depends on X through the mean (order 1) and the centred data Y = X - mean
    (orders >= 2), so dL/dX = g1 + P g with P the centring projector and
      g2[t,a] = 2 w2 (2/T) sum_j C2[a,j] y[t,j]
      g3[t,a] = 2 w3 (3/T) sum_jk C3[a,j,k] y[t,j] y[t,k]
      g4[t,a] = 2 w4 ((4/T) sum_jkl C4[a,j,k,l] y_j y_k y_l - (12/T) sum_j D[a,j] y_j),
                D[i,j] = sum_kl C4[i,j,k,l] C2[k,l]
      g1[t,a] = 2 w1 mu_a / T.
    """
    X = _as_f64(X)
    T, n = X.shape
    d = len(w) - 1
    if d > 4:
        raise ValueError("closed-form gradient is written for orders <= 4")
    C = full_cumulants_closed_form(X, max(d, 2))
    mu, Y = center(X)
    g = np.zeros_like(Y)
    if d >= 2 and w[2]:
        g += 2.0 * w[2] * (2.0 / T) * (Y @ C[1])
    if d >= 3 and w[3]:
        g += 2.0 * w[3] * (3.0 / T) * _contract_rows(Y, C[2])
    if d >= 4 and w[4]:
        D = (C[3].reshape(n * n, n * n) @ C[1].reshape(n * n)).reshape(n, n)
        g += 2.0 * w[4] * ((4.0 / T) * _contract_rows(Y, C[3]) - (12.0 / T) * (Y @ D))
    g = g - g.mean(axis=0, keepdims=True)
    if d >= 1 and w[1]:
        g += 2.0 * w[1] * mu[None, :] / T
    return g
