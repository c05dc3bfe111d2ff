"""The allocation-free norm entry point, checked against the handle's norms.

Some callers cannot call cudaMalloc, for example code running inside another
framework's memory pool or under a device-memory budget that forbids new
allocations.  For them ``cumwin_block_norm2_noalloc`` computes ||A||_F^2 of a
block-layout tensor using only a fixed scratch array in the library's own
device memory.  This file is collected last so that a failure here cannot stop
a run before the other GPU tests have run.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1701_06446_gb300 import CumWin, _lib
from paper_1701_06446_gb300.streams import WORKLOADS

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64 parity tolerance of the other GPU tests


def test_noalloc_norm_matches_handle_norms_on_consecutive_calls():
    lib = _lib.load()
    W = WORKLOADS["n60_d4_b3_T32768_p1024"]
    n, d, b, T, p = W.n, W.d, W.b, 4096, 256
    X = torch.from_numpy(W.stream().rows(0, T)).cuda()
    with CumWin(n, d, b, T, p, "fp64") as h:
        h.fill(X)
        ref = h.norms_device().cpu().numpy()  # ||C_s||_F^2 from the existing entry point
        C = [h.cumulants(s) for s in range(1, d + 1)]
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        # two rounds of calls in a row, alternating tensors, so stale scratch would show
        for _ in range(2):
            for s in (4, 2, 3, 1):
                rc = lib.cumwin_block_norm2_noalloc(n, b, s, ctypes.c_void_p(C[s - 1].data_ptr()),
                                                    ctypes.c_void_p(out.data_ptr()), stream)
                assert rc == 0, lib.cumwin_last_error().decode()
                torch.cuda.synchronize()
                got = float(out.item())
                assert abs(got - ref[s - 1]) <= TOL * ref[s - 1], (s, got, ref[s - 1])


@pytest.mark.parametrize("n,d,b", [(10, 8, 3), (13, 6, 4), (7, 5, 2)])
def test_noalloc_norm_ragged_blocks_every_order(n, d, b):
    """b does not divide n (padded variables), and every order up to d: the
    multiplicity rebuilt from the block rank sees its longest runs of equal
    block indices at the high orders.  Two calls in a row per order."""
    lib = _lib.load()
    T, p = 512, 64
    rng = np.random.default_rng(100 * n + d)
    X = (rng.standard_t(6, size=(T, n)) @ rng.standard_normal((n, n)) / np.sqrt(n) + 0.3).astype(np.float32)
    with CumWin(n, d, b, T, p, "fp64") as h:
        h.fill(torch.from_numpy(X).cuda())
        ref = h.norms_device().cpu().numpy()
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for s in range(1, d + 1):
            C = h.cumulants(s)
            for _ in range(2):
                rc = lib.cumwin_block_norm2_noalloc(n, b, s, ctypes.c_void_p(C.data_ptr()),
                                                    ctypes.c_void_p(out.data_ptr()), stream)
                assert rc == 0, lib.cumwin_last_error().decode()
                torch.cuda.synchronize()
                got = float(out.item())
                assert abs(got - ref[s - 1]) <= TOL * abs(ref[s - 1]), (s, got, ref[s - 1])
                out.fill_(-1.0)


def test_noalloc_norm_rejects_tensors_beyond_its_scratch():
    lib = _lib.load()
    buf = torch.zeros(1, dtype=torch.float64, device="cuda")
    # n=64, b=1, order 3 stores C(66, 3) = 45760 blocks, more than the fixed scratch
    rc = lib.cumwin_block_norm2_noalloc(64, 1, 3, ctypes.c_void_p(buf.data_ptr()),
                                        ctypes.c_void_p(buf.data_ptr()), None)
    assert rc == _lib.CODES["EINVAL"]
    assert "scratch" in lib.cumwin_last_error().decode()
    assert float(buf.item()) == 0.0
