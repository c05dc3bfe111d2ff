"""Seeded synthetic data streams shaped like the workloads of the paper.

This module only draws random numbers; it holds none of the method's
arithmetic, and both the CUDA path and the CPU oracle take its output as
input.  Every stream is split into fixed chunks of ``CHUNK`` rows, each drawn
from its own ``SeedSequence`` child, so any row range is reproducible no
matter how the stream is consumed.

Workloads (samples are rows, Eq. 1):

* ``gauss_then_t``      n=4: N(0, S), S = A A^T / n, then a multivariate
                        Student-t(nu=4) with scale S (nu-2)/nu, so that the
                        covariance stays S.
* ``gauss_then_expcop`` n=60: N(0, S) then a Gaussian copula with the
                        correlation of S and exponential(1) marginals.
* ``mvt``               n=48: multivariate t(nu=5) with a random correlation
                        matrix as scale.
* ``ica_mix``           n=32: X = U Q^T, U uniform(-sqrt3, sqrt3) sources,
                        Q a random orthogonal matrix.
* ``gauss_then_tcop``   the paper's own illustration (Section 4.2): Gaussian
                        then a t-copula (nu=10) with Gaussian marginals.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy import special

CHUNK = 4096


def _spd(rng: np.random.Generator, n: int) -> np.ndarray:
    A = rng.standard_normal((n, n))
    return A @ A.T / n


def _corr(S: np.ndarray) -> np.ndarray:
    d = np.sqrt(np.diag(S))
    return S / d[:, None] / d[None, :]


def _orthogonal(rng: np.random.Generator, n: int) -> np.ndarray:
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


@dataclass
class Stream:
    """A reproducible, randomly addressable stream of n-variate samples."""

    kind: str
    n: int
    seed: int
    switch_at: int = 0          # first sample index of the second regime
    dtype: type = np.float32

    def __post_init__(self):
        root = np.random.SeedSequence(self.seed)
        self._param_seed, self._chunk_root = root.spawn(2)
        rng = np.random.default_rng(self._param_seed)
        n = self.n
        if self.kind in ("gauss_then_t", "gauss_then_expcop", "gauss_then_tcop"):
            self.S = _spd(rng, n)
            self.L = np.linalg.cholesky(self.S)
            self.R = _corr(self.S)
            self.LR = np.linalg.cholesky(self.R)
        elif self.kind == "mvt":
            self.R = _corr(_spd(rng, n))
            self.LR = np.linalg.cholesky(self.R)
        elif self.kind == "ica_mix":
            self.Q = _orthogonal(rng, n)
        elif self.kind == "gauss":
            self.S = _spd(rng, n)
            self.L = np.linalg.cholesky(self.S)
        elif self.kind == "t4":
            self.S = _spd(rng, n)
            self.L = np.linalg.cholesky(self.S * 0.5)
        else:
            raise ValueError(f"unknown stream kind {self.kind!r}")

    def _chunk(self, c: int) -> np.ndarray:
        rng = np.random.default_rng(np.random.SeedSequence(
            entropy=self._chunk_root.entropy, spawn_key=self._chunk_root.spawn_key + (c,)))
        n = self.n
        first = np.arange(c * CHUNK, (c + 1) * CHUNK)
        second = first >= self.switch_at if self.switch_at else np.zeros(CHUNK, bool)
        z = rng.standard_normal((CHUNK, n))
        k = self.kind
        if k == "gauss_then_t":
            g = rng.chisquare(4.0, size=CHUNK)
            a = z @ self.L.T
            b = (z @ self.L.T) * math.sqrt(0.5) / np.sqrt(g / 4.0)[:, None]
            x = np.where(second[:, None], b, a)
        elif k == "gauss_then_expcop":
            a = z @ self.L.T
            u = special.ndtr(z @ self.LR.T)
            b = -np.log1p(-u)
            x = np.where(second[:, None], b, a)
        elif k == "gauss_then_tcop":
            g = rng.chisquare(10.0, size=CHUNK)
            a = z @ self.L.T
            w = (z @ self.LR.T) / np.sqrt(g / 10.0)[:, None]
            u = special.stdtr(10.0, w)
            b = special.ndtri(u) * np.sqrt(np.diag(self.S))[None, :]
            x = np.where(second[:, None], b, a)
        elif k == "mvt":
            g = rng.chisquare(5.0, size=CHUNK)
            x = (z @ self.LR.T) / np.sqrt(g / 5.0)[:, None]
        elif k == "ica_mix":
            u = rng.uniform(-math.sqrt(3.0), math.sqrt(3.0), size=(CHUNK, n))
            x = u @ self.Q.T
        elif k == "gauss":
            x = z @ self.L.T
        elif k == "t4":
            g = rng.chisquare(4.0, size=CHUNK)
            x = (z @ self.L.T) / np.sqrt(g / 4.0)[:, None]
        return x.astype(self.dtype)

    def rows(self, start: int, stop: int) -> np.ndarray:
        """Samples start..stop-1 as a (stop-start) x n array."""
        if stop <= start:
            return np.zeros((0, self.n), self.dtype)
        c0, c1 = start // CHUNK, (stop - 1) // CHUNK
        parts = [self._chunk(c) for c in range(c0, c1 + 1)]
        block = np.concatenate(parts, axis=0)
        off = start - c0 * CHUNK
        return np.ascontiguousarray(block[off:off + (stop - start)])


# ----------------------------------------------------------------------------
# the workloads of the benchmark configurations
# ----------------------------------------------------------------------------

@dataclass(frozen=True)
class Workload:
    name: str
    n: int
    d: int
    b: int
    T: int
    p: int
    length: int
    kind: str
    seed: int
    switch_at: int = 0

    def stream(self, dtype=np.float32) -> Stream:
        return Stream(self.kind, self.n, self.seed, self.switch_at, dtype)

    @property
    def shifts(self) -> int:
        return (self.length - self.T) // self.p


WORKLOADS = {
    # n=4, d=2..4, b=2, T=1000, p=100: Gaussian then multivariate t(4), 20000 samples
    "n4_d4_b2_T1000_p100": Workload("n4_d4_b2_T1000_p100", 4, 4, 2, 1000, 100, 20000,
                                    "gauss_then_t", 1, 10000),
    # n=60, d=2..4, b=3, T=2^15, p=2^10: Gaussian then exponential-marginal copula, 2^20 samples
    "n60_d4_b3_T32768_p1024": Workload("n60_d4_b3_T32768_p1024", 60, 4, 3, 1 << 15, 1 << 10,
                                       1 << 20, "gauss_then_expcop", 2, 1 << 19),
    # n=48, d=2..6, b=4, T=2^16, p=2^12: multivariate t(5), 2^20 samples
    "n48_d6_b4_T65536_p4096": Workload("n48_d6_b4_T65536_p4096", 48, 6, 4, 1 << 16, 1 << 12,
                                       1 << 20, "mvt", 3),
    # n=32, d=4, b=4, T=4096: orthogonal mix of uniform sources (gradient workload)
    "n32_d4_b4_T4096_ica": Workload("n32_d4_b4_T4096_ica", 32, 4, 4, 4096, 256, 4096,
                                    "ica_mix", 5),
}


def batched_streams(seed: int = 4, count: int = 512):
    """Parameters of the many-stream workload: n~U{8..64}, d~U{3,4},
    T~U{2^12, 2^14}, Gaussian or t(4) per stream, b=4, p=256."""
    rng = np.random.default_rng(seed)
    n = rng.integers(8, 65, size=count)
    d = rng.integers(3, 5, size=count)
    T = np.where(rng.integers(0, 2, size=count) == 0, 1 << 12, 1 << 14)
    kind = np.where(rng.integers(0, 2, size=count) == 0, "gauss", "t4")
    return [dict(n=int(n[i]), d=int(d[i]), T=int(T[i]), b=4, p=256, kind=str(kind[i]),
                 seed=seed * 100003 + i) for i in range(count)]


# ----------------------------------------------------------------------------
# the paper's illustration stream (Section 4.2) at full scale, drawn on the GPU
# ----------------------------------------------------------------------------

def student_t_cdf_even(x, nu: int):
    """CDF of Student's t with an even number of degrees of freedom nu, in
    closed form: with s = x / sqrt(nu + x^2),
    F(x) = 1/2 + (s/2) * sum_{k < nu/2} C(2k, k) / 4^k * (1 - s^2)^k.
    Works on numpy arrays and torch tensors alike (elementwise)."""
    if nu <= 0 or nu % 2:
        raise ValueError("nu must be a positive even integer")
    s = x / (nu + x * x) ** 0.5
    c = 1.0 - s * s
    term = s * 0.0 + 1.0
    acc = term
    for k in range(1, nu // 2):
        term = term * c * (2 * k - 1) / (2 * k)
        acc = acc + term
    return 0.5 + 0.5 * s * acc


class GaussThenTCopulaGPU:
    """The stream of Section 4.2 drawn on a CUDA device with torch: the first
    `first` samples are N(0, S); every later sample comes from a t-copula with
    nu degrees of freedom and the correlation of S, with the Gaussian marginals
    N(0, S_ii) of the first part (x_i = sqrt(S_ii) * Phi^{-1}(F_nu(w_i)),
    w = z / sqrt(g / nu), z ~ N(0, corr(S)), g ~ chi^2_nu).  S = A A^T / n with
    A ~ N(0, 1)^{n x n}.  Seeded with torch.Generator; rows are produced in
    order, `take(k)` returns the next k rows (k x n, float32, on the device)."""

    def __init__(self, n: int, first: int, seed: int, nu: int = 10, device="cuda"):
        import torch
        self.torch = torch
        self.n, self.first, self.nu, self.pos = n, first, nu, 0
        self.dev = torch.device(device)
        self.gen = torch.Generator(device=self.dev)
        self.gen.manual_seed(seed)
        A = torch.randn(n, n, generator=self.gen, device=self.dev, dtype=torch.float64)
        S = A @ A.T / n
        self.sd = torch.sqrt(torch.diag(S))
        R = S / self.sd[:, None] / self.sd[None, :]
        self.L = torch.linalg.cholesky(S)
        self.LR = torch.linalg.cholesky(R)

    def take(self, k: int):
        torch = self.torch
        out = torch.empty(k, self.n, device=self.dev, dtype=torch.float32)
        done = 0
        while done < k:
            m = min(k - done, 1 << 18)
            z = torch.randn(m, self.n, generator=self.gen, device=self.dev, dtype=torch.float64)
            gauss = self.pos + done < self.first
            if gauss:
                m = min(m, self.first - (self.pos + done))
                x = z[:m] @ self.L.T
            else:
                # chi^2_nu as a sum of nu squared standard normals (one seeded generator)
                c = torch.randn(m, self.nu, generator=self.gen, device=self.dev, dtype=torch.float64)
                chi = (c * c).sum(dim=1)
                w = (z[:m] @ self.LR.T) / torch.sqrt(chi / self.nu)[:, None]
                u = student_t_cdf_even(w, self.nu).clamp(1e-300, 1.0 - 1e-16)
                x = torch.special.ndtri(u) * self.sd[None, :]
            out[done:done + m] = x.to(torch.float32)
            done += m
        self.pos += k
        return out
