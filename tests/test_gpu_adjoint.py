"""GPU adjoint of L = sum_s w_s ||C_s||_F^2 (full-tensor norms) with respect to
the window, through the C ABI (cumwin_grad) and the autograd Function.

Checked against the oracle's closed-form gradient, against central finite
differences of the FP64 GPU loss (h = 1e-3), and against two exact
invariants: translation invariance of orders >= 2 (column sums vanish) and
homogeneity (sum x . grad = sum_s 2 s w_s ||C_s||^2).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_06446_gb300 import CumWin, CumulantNormLoss
from paper_1701_06446_gb300.streams import WORKLOADS

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel_fro(got, ref):
    return np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)


def gpu_loss(h, X, w):
    h.fill(dev(X))
    fro, _ = h.norms()
    return sum(w[s] * fro[s - 1] ** 2 for s in range(1, h.d + 1))


@pytest.mark.parametrize("w", [[0, 0, 0, 1, 1], [0, 0.5, 0.3, 1.0, 2.0]])
def test_grad_matches_oracle_on_ica_mix(w):
    W = WORKLOADS["n32_d4_b4_T4096_ica"]
    X = W.stream().rows(0, W.T)
    with CumWin(W.n, W.d, W.b, W.T, W.p, "fp64") as h:
        h.fill(dev(X))
        g = h.grad(w).cpu().numpy()
    ref = oracle.grad(X.astype(np.float64), w)
    assert rel_fro(g, ref) <= 1e-5, rel_fro(g, ref)


@pytest.mark.parametrize("n,d,b,T", [(7, 4, 3, 300), (5, 3, 2, 200), (9, 4, 1, 256), (1, 4, 1, 100)])
def test_grad_small_shapes_vs_oracle(n, d, b, T):
    rng = np.random.default_rng(n * 10 + d)
    X = (rng.gamma(2.0, size=(T, n)) @ rng.standard_normal((n, n)) / np.sqrt(n) + 1.0).astype(np.float32)
    w = [0.0, 0.7, 0.4, 1.0, 1.5][: d + 1]
    with CumWin(n, d, b, T, T // 4, "fp64") as h:
        h.fill(dev(X))
        g = h.grad(w).cpu().numpy()
    ref = oracle.grad(X.astype(np.float64), w)
    assert rel_fro(g, ref) <= 1e-5, rel_fro(g, ref)


def test_grad_vs_central_finite_differences():
    n, d, b, T = 32, 4, 4, 4096
    W = WORKLOADS["n32_d4_b4_T4096_ica"]
    X = W.stream(np.float64).rows(0, T)
    # perturbations of h = 1e-3 must survive the FP32 window: scale the data so
    # that FP32 rounding of x + h stays far below h
    w = [0, 0, 0, 1, 1]
    hstep = 1e-3
    rng = np.random.default_rng(17)
    picks = [(int(rng.integers(T)), int(rng.integers(n))) for _ in range(256)]
    with CumWin(n, d, b, T, T, "fp64") as h:
        h.fill(dev(X))
        g = h.grad(w).cpu().numpy()
        Xf = X.astype(np.float32).astype(np.float64)
        fd = []
        for t, a in picks:
            Xp, Xm = Xf.copy(), Xf.copy()
            Xp[t, a] += hstep
            Xm[t, a] -= hstep
            # the values the GPU sees are the FP32-rounded ones: divide by the actual step
            step = np.float32(Xp[t, a]) - np.float32(Xm[t, a])
            fd.append((gpu_loss(h, Xp, w) - gpu_loss(h, Xm, w)) / float(step))
    fd = np.array(fd)
    got = np.array([g[t, a] for t, a in picks])
    scale = np.abs(g).max()
    assert np.max(np.abs(fd - got)) <= 2e-4 * scale, (np.max(np.abs(fd - got)), scale)


def test_grad_invariants():
    W = WORKLOADS["n32_d4_b4_T4096_ica"]
    X = W.stream().rows(0, W.T)
    w = [0, 0, 0.5, 1, 1]
    with CumWin(W.n, W.d, W.b, W.T, W.p, "fp64") as h:
        h.fill(dev(X))
        g = h.grad(w).cpu().numpy().astype(np.float64)
        fro, _ = h.norms()
    assert np.abs(g.sum(axis=0)).max() <= 1e-4 * np.abs(g).max() * np.sqrt(W.T)
    euler = sum(2 * s * w[s] * fro[s - 1] ** 2 for s in range(1, 5))
    assert abs(np.sum(X.astype(np.float64) * g) - euler) <= 1e-5 * euler


def test_grad_after_shifts_uses_window_order():
    """After shifts the ring is rotated; the gradient rows follow the window (oldest first)."""
    n, d, b, T, p = 6, 4, 2, 400, 50
    rng = np.random.default_rng(2)
    X = rng.standard_t(6, size=(T + 5 * p, n)).astype(np.float32)
    w = [0, 0.2, 0.3, 1, 1]
    with CumWin(n, d, b, T, p, "fp64") as h:
        h.fill(dev(X[:T]))
        for k in range(5):
            h.push(dev(X[T + k * p: T + (k + 1) * p]))
        g = h.grad(w).cpu().numpy()
    ref = oracle.grad(X[5 * p:].astype(np.float64), w)
    assert rel_fro(g, ref) <= 1e-5


def test_autograd_function_backward():
    W = WORKLOADS["n32_d4_b4_T4096_ica"]
    X = dev(W.stream().rows(0, W.T)).requires_grad_(True)
    w = [0, 0, 0, 1, 1]
    L = CumulantNormLoss.apply(X, w, W.b)
    L.backward()
    ref = oracle.grad(X.detach().cpu().numpy().astype(np.float64), w)
    assert rel_fro(X.grad.cpu().numpy(), ref) <= 1e-5
    fro, _ = oracle.norms(X.detach().cpu().numpy(), 4)
    assert abs(L.item() - (fro[2] ** 2 + fro[3] ** 2)) <= 1e-9 * L.item()


@pytest.mark.parametrize("w", [[0, 0, 0, 1, 1], [0, 0.5, 0.3, 1.0, 2.0]])
def test_library_loss_matches_oracle(w):
    """cumwin_loss forms L = sum_s w_s ||C_s||^2 on the device; the oracle's loss is
    the full-tensor sum over its own cumulants."""
    W = WORKLOADS["n32_d4_b4_T4096_ica"]
    X = W.stream().rows(0, W.T)
    with CumWin(W.n, W.d, W.b, W.T, W.p, "fp64") as h:
        h.fill(dev(X))
        L = float(h.loss(w).item())
    ref = oracle.loss(X.astype(np.float64), w)
    assert abs(L - ref) <= 1e-10 * abs(ref), (L, ref)


def test_mixed_form_grad_close_to_fp64_form():
    W = WORKLOADS["n32_d4_b4_T4096_ica"]
    X = dev(W.stream().rows(0, W.T))
    w = [0, 0, 0, 1, 1]
    with CumWin(W.n, W.d, W.b, W.T, W.p, "fp64") as a, CumWin(W.n, W.d, W.b, W.T, W.p, "bf16") as m:
        a.fill(X)
        m.fill(X)
        ga = a.grad(w).cpu().numpy()
        gm = m.grad(w).cpu().numpy()
    assert rel_fro(gm, ga) <= 1e-3


@pytest.mark.parametrize("form", ["fp64", "bf16"])
def test_grad_order6_canonical_orders_vs_oracle_loss_differences(form):
    """d = 6, b = 4: orders 5 and 6 run the canonical recovery, and the sums of
    order 5 are kept at its canonical elements only (in workspace order in the
    mixed forms); the adjoint gathers them back to the block layout before it
    expands the moments.  The gradient at 24 seeded entries against central
    differences of the oracle's FP64 loss on the same (FP32-representable)
    window, h = 1e-3 (the oracle's closed form stops at order 4)."""
    n, d, b, T = 6, 6, 4, 256
    rng = np.random.default_rng(66)
    X = (rng.gamma(2.0, size=(T, n)) @ rng.standard_normal((n, n)) / np.sqrt(n)).astype(np.float32)
    Xd = X.astype(np.float64)
    w = [0.0, 0.3, 0.5, 1.0, 1.5, 0.8, 0.6]
    with CumWin(n, d, b, T, T // 4, form) as h:
        h.fill(dev(X))
        g = h.grad(w).cpu().numpy()
    hstep = 1e-3
    picks = [(int(rng.integers(T)), int(rng.integers(n))) for _ in range(24)]
    fd = []
    for t, a in picks:
        Xp, Xm = Xd.copy(), Xd.copy()
        Xp[t, a] += hstep
        Xm[t, a] -= hstep
        fd.append((oracle.loss(Xp, w) - oracle.loss(Xm, w)) / (2 * hstep))
    fd = np.array(fd)
    got = np.array([g[t, a] for t, a in picks])
    tol = 1e-4 if form == "fp64" else 2e-3
    assert np.linalg.norm(got - fd) <= tol * np.linalg.norm(fd), (got, fd)
