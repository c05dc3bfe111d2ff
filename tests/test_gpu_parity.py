"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Bar (FP64 form): relative Frobenius error <= 1e-10 per order against the FP64
oracle, element by element on windows the oracle recomputes in seconds, and on
seeded samples of sorted tuples at the full workload sizes.  Integer-valued
windows (exact products and sums) must match to 1e-12.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle
from paper_1701_06446_gb300 import CumWin, CumwinError
from paper_1701_06446_gb300.streams import WORKLOADS, Stream

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def gpu_cumulants(h):
    return [h.cumulants(s).cpu().numpy() for s in range(1, h.d + 1)]


def rel_fro(got, ref):
    den = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) / (den if den > 0 else 1.0)


def assert_window_parity(h, X, tol=TOL_FP64):
    ref = oracle.cumulants(X, h.d, h.b)
    got = gpu_cumulants(h)
    for s in range(1, h.d + 1):
        assert got[s - 1].shape == ref[s - 1].shape
        err = rel_fro(got[s - 1], ref[s - 1])
        assert err <= tol, (s, err)
    fro, nu = h.norms()
    ofro, onu = oracle.norms(X, h.d)
    assert np.allclose(fro, ofro, rtol=tol, atol=0), (fro, ofro)
    for s in range(3, h.d + 1):
        assert abs(nu[s - 1] - onu[s - 1]) <= tol * abs(onu[s - 1])


def test_small_gauss_then_t_every_shift():
    """n=4, d=4, b=2, T=1000, p=100: every one of the 190 shifts vs the oracle."""
    W = WORKLOADS["n4_d4_b2_T1000_p100"]
    X = W.stream().rows(0, W.length)
    Xd = dev(X)
    with CumWin(W.n, W.d, W.b, W.T, W.p, "fp64") as h:
        h.fill(Xd[: W.T])
        assert_window_parity(h, X[: W.T])
        for w in range(W.shifts):
            h.push(Xd[W.T + w * W.p: W.T + (w + 1) * W.p])
            if w % 10 == 9 or w == W.shifts - 1:
                assert_window_parity(h, X[(w + 1) * W.p: (w + 1) * W.p + W.T])
            else:
                ref = oracle.cumulants(X[(w + 1) * W.p: (w + 1) * W.p + W.T], W.d, W.b)
                got = gpu_cumulants(h)
                for s in range(1, W.d + 1):
                    assert rel_fro(got[s - 1], ref[s - 1]) <= TOL_FP64


@pytest.mark.parametrize("n,d,b,T,p", [(3, 4, 2, 12, 4), (2, 6, 1, 9, 3), (5, 5, 2, 16, 5),
                                       (3, 3, 4, 10, 10), (1, 6, 1, 11, 1)])
def test_integer_windows_exact(n, d, b, T, p):
    rng = np.random.default_rng(n * 100 + d)
    X = rng.integers(-3, 4, size=(T + 3 * p, n)).astype(np.float32)
    Xd = dev(X)
    with CumWin(n, d, b, T, p, "fp64") as h:
        h.fill(Xd[:T])
        assert_window_parity(h, X[:T], tol=1e-12)
        for w in range(3):
            h.push(Xd[T + w * p: T + (w + 1) * p])
        assert_window_parity(h, X[3 * p: 3 * p + T], tol=1e-12)


@pytest.mark.parametrize("n,d,b,T,p", [(7, 4, 3, 64, 7), (5, 5, 2, 50, 7), (9, 3, 4, 33, 33),
                                       (6, 4, 1, 40, 1), (10, 6, 3, 80, 16), (33, 3, 4, 300, 64),
                                       (2, 8, 1, 30, 4), (5, 7, 3, 60, 7), (4, 7, 4, 64, 16)])
def test_ragged_shapes_and_shift_sizes(n, d, b, T, p):
    """Padding (b does not divide n), p not dividing T, p = 1, p = T, high orders
    (d = 7 with canonical orders 5-6 below a top order without the canonical
    recovery, whose subset terms read their sums at every element)."""
    rng = np.random.default_rng(7 * n + d)
    steps = 5
    X = (rng.standard_t(5, size=(T + steps * p, n)) @ rng.standard_normal((n, n))).astype(np.float32)
    Xd = dev(X)
    with CumWin(n, d, b, T, p, "fp64") as h:
        h.fill(Xd[:T])
        for w in range(steps):
            h.push(Xd[T + w * p: T + (w + 1) * p])
        assert_window_parity(h, X[steps * p: steps * p + T])
        win = h.window().cpu().numpy()
        assert np.array_equal(win, X[steps * p: steps * p + T])


def test_padding_entries_are_exact_zero():
    rng = np.random.default_rng(3)
    n, b, d, T = 7, 3, 4, 100
    X = rng.standard_normal((T, n)).astype(np.float32)
    with CumWin(n, d, b, T, 10, "fp64") as h:
        h.fill(dev(X))
        for s in range(1, d + 1):
            C = h.cumulants(s).cpu().numpy()
            pad = np.any(oracle.block_elements(n, b, s) >= n, axis=1)
            assert np.all(C[pad] == 0.0)


def test_explicit_outgoing_rows_match_ring():
    """push(x_in, x_out = the oldest rows) is bitwise the ring-buffer shift when
    both recompute X_(-) (a window that is not a whole number of batches has no
    batch-sum FIFO)."""
    W = WORKLOADS["n4_d4_b2_T1000_p100"]
    X = W.stream().rows(0, 3000)
    Xd = dev(X)
    T, p = 1000, 96
    with CumWin(4, 4, 2, T, p) as a, CumWin(4, 4, 2, T, p) as b:
        a.fill(Xd[:T])
        b.fill(Xd[:T])
        assert not a.fifo and not b.fifo
        for w in range(20):
            a.push(Xd[T + w * p: T + (w + 1) * p])
            b.push(Xd[T + w * p: T + (w + 1) * p], Xd[w * p: (w + 1) * p].clone())
        for s in range(1, 5):
            assert torch.equal(a.cumulants(s), b.cumulants(s))


def test_fp64_fifo_matches_recomputing_form():
    """FP64 batch-sum FIFO (Section 2.4's alternative): a regular shift subtracts the
    leaving batch's stored FP64 sums.  The recomputing form (caller-supplied X_(-))
    forms the same products and adds them in another order, so the two agree to the
    rounding of FP64 additions, and both match the oracle."""
    W = WORKLOADS["n4_d4_b2_T1000_p100"]
    X = W.stream().rows(0, 4000)
    Xd = dev(X)
    T, p = 1000, 100
    with CumWin(4, 4, 2, T, p) as a, CumWin(4, 4, 2, T, p) as b:
        a.fill(Xd[:T])
        b.fill(Xd[:T])
        assert a.fifo and b.fifo
        for w in range(25):
            a.push(Xd[T + w * p: T + (w + 1) * p])
            b.push(Xd[T + w * p: T + (w + 1) * p], Xd[w * p: (w + 1) * p].clone())
        assert a.fifo and not b.fifo
        for s in range(1, 5):
            assert rel_fro(a.moments(s).cpu().numpy(), b.moments(s).cpu().numpy()) <= 1e-14, s
        assert_window_parity(a, X[25 * p: 25 * p + T])
        assert_window_parity(b, X[25 * p: 25 * p + T])


@pytest.mark.parametrize("n,d,b,T,p", [(6, 4, 2, 600, 50), (5, 6, 4, 256, 32)])
def test_fp64_fifo_retired_by_short_shift_and_restored_by_recompute(n, d, b, T, p):
    """An irregular shift retires the FP64 FIFO; recompute refills it batch by batch
    from the ring's head, which is then no longer a multiple of p, so the slots
    follow the head; two full turns of the window later the sums still match the
    oracle and a fresh recomputation."""
    rng = np.random.default_rng(31)
    X = (rng.standard_t(5, size=(T + 40 * p, n)) + 0.5).astype(np.float32)
    Xd = dev(X)
    with CumWin(n, d, b, T, p) as h:
        h.fill(Xd[:T])
        assert h.fifo
        pos = T
        for w in range(3):
            h.push(Xd[pos: pos + p])
            pos += p
        assert_window_parity(h, X[pos - T: pos])
        h.push(Xd[pos: pos + 7])  # fewer rows than p: X_(-) recomputed, FIFO retired
        pos += 7
        assert not h.fifo
        for w in range(3):
            h.push(Xd[pos: pos + p])
            pos += p
        assert not h.fifo
        assert_window_parity(h, X[pos - T: pos])
        h.recompute()
        assert h.fifo
        for w in range(2 * T // p + 3):
            h.push(Xd[pos: pos + p])
            pos += p
        assert h.fifo
        assert_window_parity(h, X[pos - T: pos])
        slide = [h.moments(s).cpu().numpy() for s in range(1, d + 1)]
        h.recompute()
        for s in range(1, d + 1):
            assert rel_fro(slide[s - 1], h.moments(s).cpu().numpy()) <= 1e-13, s


def test_sliding_equals_fresh_after_1e4_shifts():
    """10^4 shifts of the n=4 workload, extended with the same generator."""
    W = WORKLOADS["n4_d4_b2_T1000_p100"]
    shifts = 10_000
    X = W.stream().rows(0, W.T + shifts * W.p)
    Xd = dev(X)
    with CumWin(W.n, W.d, W.b, W.T, W.p, "fp64") as h:
        h.fill(Xd[: W.T])
        for w in range(shifts):
            h.push(Xd[W.T + w * W.p: W.T + (w + 1) * W.p])
        slide = gpu_cumulants(h)
        assert_window_parity(h, X[shifts * W.p:])
        h.recompute()
        fresh = gpu_cumulants(h)
        for s in range(1, W.d + 1):
            assert rel_fro(slide[s - 1], fresh[s - 1]) <= TOL_FP64


def test_ica_mix_forward_all_elements():
    """n=32, d=4, b=4, T=4096: every stored element of every order."""
    W = WORKLOADS["n32_d4_b4_T4096_ica"]
    X = W.stream().rows(0, W.T)
    with CumWin(W.n, W.d, W.b, W.T, W.p, "fp64") as h:
        h.fill(dev(X))
        assert_window_parity(h, X)


def _sampled_parity(h, X, per_order, seed, tol=TOL_FP64):
    n, b = h.n, h.b
    cen = oracle.center(X)
    for s in range(1, h.d + 1):
        C = h.cumulants(s).cpu().numpy()
        tup = oracle.sample_sorted_tuples(n, s, per_order, seed=seed + s)
        idx = np.array([oracle.storage_index(n, b, t) for t in tup])
        ref = oracle.cumulant_tuples(X, tup, centred=cen)
        err = rel_fro(C[idx], ref)
        assert err <= tol, (s, err)


def test_n60_workload_sampled():
    """n=60, d=4, b=3, T=2^15, p=2^10: fill and 3 shifts, sampled tuples per order."""
    W = WORKLOADS["n60_d4_b3_T32768_p1024"]
    start = (1 << 19) - W.T - W.p  # straddle the Gaussian -> copula switch
    X = W.stream().rows(start, start + W.T + 3 * W.p)
    Xd = dev(X)
    with CumWin(W.n, W.d, W.b, W.T, W.p, "fp64") as h:
        h.fill(Xd[: W.T])
        for w in range(3):
            h.push(Xd[W.T + w * W.p: W.T + (w + 1) * W.p])
        _sampled_parity(h, X[3 * W.p:], 1500, seed=60)


def test_n48_order6_workload_sampled():
    """n=48, d=6, b=4, T=2^16, p=2^12: fill and one shift, sampled tuples per order."""
    W = WORKLOADS["n48_d6_b4_T65536_p4096"]
    X = W.stream().rows(0, W.T + W.p)
    Xd = dev(X)
    with CumWin(W.n, W.d, W.b, W.T, W.p, "fp64") as h:
        h.fill(Xd[: W.T])
        h.push(Xd[W.T:])
        _sampled_parity(h, X[W.p:], 300, seed=48)


def test_cuda_graph_replay_matches_eager():
    W = WORKLOADS["n4_d4_b2_T1000_p100"]
    X = W.stream().rows(0, 4000)
    Xd = dev(X)
    with CumWin(4, 4, 2, 1000, 100) as eager, CumWin(4, 4, 2, 1000, 100) as cap:
        eager.fill(Xd[:1000])
        cap.fill(Xd[:1000])
        buf = torch.empty(100, 4, device="cuda")
        buf.copy_(Xd[1000:1100])
        torch.cuda.synchronize()
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                cap.push(buf)
        torch.cuda.synchronize()
        # capture does not execute: replay the captured shift 20 times with fresh data
        for w in range(20):
            buf.copy_(Xd[1000 + w * 100: 1100 + w * 100])
            g.replay()
            eager.push(Xd[1000 + w * 100: 1100 + w * 100])
        torch.cuda.synchronize()
        for k in range(1, 5):
            assert torch.equal(eager.cumulants(k), cap.cumulants(k))


def test_nonfinite_sample_sets_status():
    X = np.random.default_rng(0).standard_normal((60, 3)).astype(np.float32)
    with CumWin(3, 3, 2, 50, 5) as h:
        h.fill(dev(X[:50]))
        assert h.status() == 0
        bad = X[50:55].copy()
        bad[2, 1] = np.nan
        h.push(dev(bad))
        assert h.status() == -5
        with pytest.raises(CumwinError) as ei:
            h.norms()
        assert ei.value.code == -5


def test_call_sequence_and_argument_errors():
    with CumWin(3, 3, 2, 50, 5) as h:
        x = torch.zeros(5, 3, device="cuda")
        with pytest.raises(CumwinError) as ei:
            h.push(x)
        assert ei.value.code == -4  # push before fill
        h.fill(torch.zeros(50, 3, device="cuda"))
        with pytest.raises(ValueError):
            h.cumulants(4)
        out = torch.empty(100, dtype=torch.float64, device="cuda")
        assert h.lib.cumwin_cumulants(h._h, 4, out.data_ptr()) == -1  # EINVAL from the ABI
        with pytest.raises(CumwinError):
            h.push(torch.zeros(51, 3, device="cuda"))
        fro, nu = h.norms()
        assert fro[1] == 0.0 and np.isnan(nu[2])  # constant window: nu is 0/0


@pytest.mark.parametrize("k", [1.0, 2.0, 3.5])
def test_k_norms_and_marginals(k):
    """Algorithm 5 with a general k against the oracle's k-norms; the per-variable
    skewness and excess kurtosis against scipy's biased estimators."""
    from scipy import stats
    n, d, b, T, p = 7, 4, 3, 300, 50
    rng = np.random.default_rng(17)
    X = (rng.gamma(2.0, size=(T + 2 * p, n)) @ rng.standard_normal((n, n)) + 1.0).astype(np.float32)
    Xd = dev(X)
    Xw = X[2 * p:].astype(np.float64)
    want = oracle.norms_k(Xw, d, k)
    for precision, tol in (("fp64", 1e-10), ("bf16", 5e-3)):
        with CumWin(n, d, b, T, p, precision) as h:
            h.fill(Xd[:T])
            h.push(Xd[T:T + p])
            h.push(Xd[T + p:])
            got = h.norms_k(k)
            np.testing.assert_allclose(got, want, rtol=tol)
            if k == 2.0:
                np.testing.assert_allclose(got, h.norms()[0], rtol=1e-12)
            sk, ku = h.marginals()
            np.testing.assert_allclose(sk, stats.skew(Xw, axis=0, bias=True), rtol=tol, atol=tol)
            np.testing.assert_allclose(ku, stats.kurtosis(Xw, axis=0, fisher=True, bias=True), rtol=tol, atol=tol)
    with CumWin(n, 2, b, T, p, "fp64") as h2:
        h2.fill(Xd[:T])
        sk, ku = h2.marginals()
        assert np.all(np.isnan(sk)) and np.all(np.isnan(ku))
        with pytest.raises(CumwinError):
            h2.norms_k(0.5)


@pytest.mark.parametrize("n,precision", [(256, "fp64"), (255, "bf16"), (256, "bf16")])
def test_maximum_number_of_variables(n, precision):
    """n at the largest the layout takes (256 variables, padded or not), orders
    1-3 with b = 8 (order 3: 3.06 M stored elements), FP64 and split forms,
    sampled tuples against the oracle after shifts through the ring."""
    d, b, T, p = 3, 8, 512, 64
    rng = np.random.default_rng(61 + n)
    A = rng.standard_normal((n, n)) / np.sqrt(n)
    X = (rng.gamma(2.0, size=(T + 4 * p, n)) @ A).astype(np.float32)
    Xd = dev(X)
    with CumWin(n, d, b, T, p, precision) as h:
        h.fill(Xd[:T])
        for w in range(4):
            h.push(Xd[T + w * p: T + (w + 1) * p])
        Xw = X[4 * p: 4 * p + T]
        cen = oracle.center(Xw)
        tol = TOL_FP64 if precision == "fp64" else {1: 2e-5, 2: 5e-5, 3: 5e-4}
        for s in range(1, d + 1):
            tup = oracle.sample_sorted_tuples(n, s, 300, seed=7 * s + n)
            idx = np.array([oracle.storage_index(n, b, t) for t in tup])
            ref = oracle.cumulant_tuples(Xw, tup, centred=cen)
            err = rel_fro(h.cumulants(s).cpu().numpy()[idx], ref)
            assert err <= (tol if precision == "fp64" else tol[s]), (s, err)
        assert np.array_equal(h.window().cpu().numpy(), Xw)


@pytest.mark.parametrize("d,precision", [(1, "fp64"), (1, "bf16"), (2, "fp64"), (2, "bf16")])
def test_lowest_orders(d, precision):
    """d = 1 (means only) and d = 2 (covariance): no order above the split and no
    nu; the recovery, norms and ring still follow the window."""
    n, b, T, p = 11, 3, 96, 16
    rng = np.random.default_rng(71 + d)
    X = (rng.standard_normal((T + 5 * p, n)) * 2.0 + 1.0).astype(np.float32)
    Xd = dev(X)
    with CumWin(n, d, b, T, p, precision) as h:
        h.fill(Xd[:T])
        for w in range(5):
            h.push(Xd[T + w * p: T + (w + 1) * p])
        Xw = X[5 * p: 5 * p + T]
        ref = oracle.cumulants(Xw, d, b)
        tol = [TOL_FP64] * d if precision == "fp64" else [2e-5, 5e-5][:d]
        for s in range(1, d + 1):
            assert rel_fro(h.cumulants(s).cpu().numpy(), ref[s - 1]) <= tol[s - 1], s
        fro, nu = h.norms()
        ofro, _ = oracle.norms(Xw, d)
        assert np.allclose(fro, ofro, rtol=max(tol), atol=0)
        assert np.all(np.isnan(nu))
        assert np.array_equal(h.window().cpu().numpy(), Xw)


@pytest.mark.parametrize("n,d,b,precision", [(7, 4, 3, "fp64"), (9, 3, 4, "bf16"), (5, 5, 2, "fp64")])
def test_full_tensor_expansion(n, d, b, precision):
    """cumwin_full expands the block layout into the full super-symmetric n^s
    tensor: equal to the oracle's expansion of the same stored values, and to
    the oracle's cumulants within the form's tolerance."""
    T, p = 80, 10
    rng = np.random.default_rng(101 + n)
    X = (rng.standard_normal((T + 3 * p, n)) + 0.5).astype(np.float32)
    Xd = dev(X)
    with CumWin(n, d, b, T, p, precision) as h:
        h.fill(Xd[:T])
        for w in range(3):
            h.push(Xd[T + w * p: T + (w + 1) * p])
        Xw = X[3 * p: 3 * p + T]
        ref = oracle.cumulants(Xw, d, b)
        for s in range(1, d + 1):
            full = h.full(s).cpu().numpy()
            assert full.shape == (n,) * s
            # every full index reads the stored element of its sorted tuple (a diagonal block
            # also stores the unsorted in-block orders, which agree up to rounding)
            blk = h.cumulants(s).cpu().numpy()
            tup = list(itertools.product(range(n), repeat=s))
            want = np.array([blk[oracle.storage_index(n, b, tuple(sorted(t)))] for t in tup]).reshape((n,) * s)
            assert np.array_equal(full, want), s
            tol = TOL_FP64 if precision == "fp64" else 5e-4
            assert rel_fro(full, oracle.to_full(ref[s - 1], n, b, s)) <= tol, s


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_estimators_enqueue_match_norms(precision):
    """||C_s|| and nu_s formed on the device (cumwin_estimators_enqueue), into host
    and device memory, equal what cumwin_norms returns, and nu matches the oracle."""
    W = WORKLOADS["n4_d4_b2_T1000_p100"]
    X = W.stream().rows(0, W.T + 3 * W.p)
    Xd = dev(X)
    with CumWin(W.n, W.d, W.b, W.T, W.p, precision) as h:
        h.fill(Xd[: W.T])
        fro_h = torch.zeros(W.d, dtype=torch.float64).pin_memory()
        nu_h = torch.zeros(W.d, dtype=torch.float64).pin_memory()
        st_h = torch.full((1,), -1, dtype=torch.int32).pin_memory()
        nu_d = torch.zeros(W.d, dtype=torch.float64, device="cuda")
        for k in range(3):
            h.push(Xd[W.T + k * W.p: W.T + (k + 1) * W.p])
            h.estimators_enqueue(fro_h, nu_h, st_h)
            h.estimators_enqueue(nu_out=nu_d)
        h.join()
        torch.cuda.synchronize()
        fro, nu = h.norms()
    assert int(st_h.item()) == 0
    np.testing.assert_allclose(fro_h.numpy(), fro, rtol=1e-14)
    np.testing.assert_allclose(nu_h.numpy()[2:], nu[2:], rtol=1e-14)
    np.testing.assert_allclose(nu_d.cpu().numpy()[2:], nu[2:], rtol=1e-14)
    assert np.all(np.isnan(nu_h.numpy()[:2]))
    ofro, onu = oracle.norms(X[3 * W.p:], W.d)
    tol = 1e-10 if precision == "fp64" else 1e-3
    np.testing.assert_allclose(nu_h.numpy()[2:], onu[2:], rtol=tol)


@pytest.mark.parametrize("n,d,b", [(10, 6, 4), (9, 5, 4), (7, 6, 3)])
def test_moments_of_canonical_orders_at_every_stored_element(n, d, b):
    """The update of a canonical order (orders 5-6, b^s >= 256) forms only the rows
    and columns of its compressed tables, so its sums exist at canonical elements
    only; cumwin_moments returns every stored element from its canonical one.  FP64
    form (moments about zero): every stored element of every order against the
    oracle's raw moments, after shifts and after a recompute."""
    T, p = 300, 40
    rng = np.random.default_rng(11 * n + d + b)
    X = (rng.standard_t(6, size=(T + 3 * p, n)) @ rng.standard_normal((n, n)) / np.sqrt(n) + 0.3)
    X = X.astype(np.float32)
    Xd = dev(X)
    ref = oracle.moments(X[3 * p:], d, b)
    with CumWin(n, d, b, T, p, "fp64") as h:
        h.fill(Xd[:T])
        for w in range(3):
            h.push(Xd[T + w * p: T + (w + 1) * p])
        for s in range(1, d + 1):
            assert rel_fro(h.moments(s).cpu().numpy(), ref[s - 1]) <= TOL_FP64, s
        h.recompute()
        for s in range(1, d + 1):
            assert rel_fro(h.moments(s).cpu().numpy(), ref[s - 1]) <= TOL_FP64, s


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
@pytest.mark.parametrize("n,d,b", [(10, 6, 4), (9, 5, 4), (7, 6, 3)])
def test_canonical_orders_are_exactly_symmetric(n, d, b, precision):
    """Orders 5-6 with blocks of >= 256 elements are recovered once per class of
    entries that super-symmetry makes equal and copied to the permuted offsets of
    diagonal blocks: the full tensor is then bitwise invariant under every
    permutation of its indices, and matches the oracle."""
    import itertools
    T, p = 400, 50
    rng = np.random.default_rng(7 * n + d + b)
    X = (rng.standard_t(6, size=(T + 3 * p, n)) @ rng.standard_normal((n, n)) / np.sqrt(n) + 0.2)
    X = X.astype(np.float32)
    Xd = dev(X)
    with CumWin(n, d, b, T, p, precision) as h:
        h.fill(Xd[:T])
        for w in range(3):
            h.push(Xd[T + w * p: T + (w + 1) * p])
        ref = oracle.cumulants(X[3 * p:], d, b)
        tol = TOL_FP64 if precision == "fp64" else 1e-3
        for s in (5, 6):
            if s > d:
                continue
            full = h.full(s).cpu().numpy()
            for perm in itertools.permutations(range(s)):
                assert np.array_equal(full, full.transpose(perm)), (s, perm)
            assert rel_fro(h.cumulants(s).cpu().numpy(), ref[s - 1]) <= tol, s
