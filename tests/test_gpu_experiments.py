"""The paper's experiments at reduced size on the GPU: the stream of Section
4.2 (Gaussian window, then t-copula updates with Gaussian marginals) drives
nu_4 up until the last Gaussian batch has left the window while ||C_2|| and
the marginals stay put; the sliding update is faster than a recalculation."""
import numpy as np
import pytest
import torch

from paper_1701_06446_gb300.experiments import detection, speedup
from paper_1701_06446_gb300.streams import GaussThenTCopulaGPU

pytestmark = pytest.mark.gpu


def test_tcopula_stream_keeps_gaussian_marginals():
    n, first = 6, 1 << 16
    gen = GaussThenTCopulaGPU(n, first=first, seed=3)
    a = gen.take(first).double()
    c = gen.take(1 << 17).double()
    sd = gen.sd
    for x in (a, c):
        z = x / sd[None, :]
        assert torch.allclose(z.mean(0), torch.zeros(n, dtype=z.dtype, device=z.device), atol=0.03)
        assert torch.allclose(z.var(0), torch.ones(n, dtype=z.dtype, device=z.device), atol=0.05)
        k = ((z - z.mean(0)) ** 4).mean(0) / z.var(0) ** 2 - 3.0  # marginal excess kurtosis ~ 0
        assert float(k.abs().max()) < 0.15


def test_detection_small():
    out = detection(seeds=1, n=16, T=1 << 16, p=1 << 12, wmax=20, b=4)
    nu4 = out["curves_seed0"]["nu4"]
    c2 = out["curves_seed0"]["c2"]
    sat = (1 << 16) // (1 << 12) + 1
    assert nu4[sat - 1] > 2.5 * nu4[0], nu4
    assert np.all(np.diff(nu4[: sat]) > -0.1 * nu4[sat - 1])  # rises (up to noise) until saturation
    assert max(c2) / min(c2) < 1.2


def test_speedup_small():
    out = speedup(n=12, configs=((1 << 15, 4, 4),), fractions=(16,), reps=3)
    row = out["rows"][0]
    assert row["speedup"] > 2.0, row
