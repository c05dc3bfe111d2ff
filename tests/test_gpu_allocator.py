"""Every byte of device state comes from the allocator of cumwin_set_allocator.

A counting allocator (ctypes callbacks around PyTorch's caching allocator)
is installed, handles of both forms are created and driven through every
call that needs scratch (fill, pushes, k-norms, marginals, the adjoint), and
the test checks that the bytes the allocator handed out equal what the
handle reports holding, that nothing is allocated after creation (except the
adjoint's workspace at its first call), and that destroy gives every block
back.  The library's own default (cudaMallocAsync) is exercised too.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1701_06446_gb300 import CumWin, CumWinBatch, _lib

pytestmark = pytest.mark.gpu


class CountingAllocator:
    def __init__(self):
        self.live = {}
        self.allocs = 0
        self.frees = 0
        self.bytes = 0
        self.streams = set()
        self.alloc_cb = _lib.ALLOC_FN(self._alloc)
        self.free_cb = _lib.FREE_FN(self._free)

    def _alloc(self, ctx, nbytes, stream, out):
        try:
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
        except Exception:
            return 1
        self.live[ptr] = int(nbytes)
        self.allocs += 1
        self.bytes += int(nbytes)
        self.streams.add(int(stream or 0))
        out[0] = ptr
        return 0

    def _free(self, ctx, ptr, nbytes, stream):
        assert self.live.pop(int(ptr)) == int(nbytes)
        self.frees += 1
        torch.cuda.caching_allocator_delete(int(ptr))

    def __enter__(self):
        _lib.set_allocator(self.alloc_cb, self.free_cb)
        return self

    def __exit__(self, *exc):
        _lib.set_allocator()  # back to the binding's default (the caching allocator)


def _data(n, T, extra, seed):
    rng = np.random.default_rng(seed)
    X = (rng.standard_t(6, size=(T + extra, n)) @ rng.standard_normal((n, n)) / np.sqrt(n) + 0.4)
    return torch.from_numpy(X.astype(np.float32)).cuda()


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_every_byte_goes_through_the_allocator(precision):
    lib = _lib.load()
    n, d, b, T, p = 11, 4, 3, 512, 64
    X = _data(n, T, 4 * p, 3)
    with CountingAllocator() as ca:
        h = CumWin(n, d, b, T, p, precision)
        held = int(lib.cumwin_device_bytes(h._h))
        assert ca.allocs > 0 and ca.bytes == held == sum(ca.live.values())
        h.fill(X[:T])
        for w in range(4):
            h.push(X[T + w * p: T + (w + 1) * p])
        h.norms()
        h.norms_k(3.0)
        h.marginals()
        h.recompute()
        torch.cuda.synchronize()
        assert ca.bytes == held, "a call after create allocated device memory"
        h.grad([0, 0, 1, 1, 1])  # the adjoint's workspace: allocated once, at the first call
        grad_bytes = ca.bytes - held
        assert grad_bytes > 0 and int(lib.cumwin_device_bytes(h._h)) == ca.bytes
        h.grad([0, 0, 1, 1, 1])
        assert ca.bytes == held + grad_bytes
        h.close()
        assert ca.live == {} and ca.frees == ca.allocs


def test_batch_memory_goes_through_the_allocator():
    ns, ds, Ts = [9, 13, 6], [3, 4, 4], [256, 512, 256]
    b, p = 4, 64
    with CountingAllocator() as ca:
        B = CumWinBatch(ns, ds, Ts, b, p, "bf16")
        created = ca.bytes
        assert created > 0
        B.fill([_data(n, T, 0, i) for i, (n, T) in enumerate(zip(ns, Ts))])
        rows = [_data(n, p, 0, 10 + i)[:p] for i, n in enumerate(ns)]
        B.push(B.pack(rows))
        B.norms()
        torch.cuda.synchronize()
        assert ca.bytes == created
        B.close()
        assert ca.live == {}


def test_default_allocator_when_none_is_installed():
    """Both callbacks NULL: the library's default (stream-ordered allocation on
    the handle's stream, synchronised) gives a working handle."""
    lib = _lib.load()
    n, d, b, T, p = 7, 4, 2, 256, 32
    X = _data(n, T, p, 5)
    assert lib.cumwin_set_allocator(None, None, None) == 0
    try:
        with CumWin(n, d, b, T, p, "bf16") as h:
            h.fill(X[:T])
            h.push(X[T:])
            fro, _ = h.norms()
            assert np.all(np.isfinite(fro)) and int(lib.cumwin_device_bytes(h._h)) > 0
    finally:
        _lib.set_allocator()
    # one callback without the other is rejected
    assert lib.cumwin_set_allocator(ctypes.cast(_lib._TORCH_ALLOC, ctypes.c_void_p), None, None) == \
        _lib.CODES["EINVAL"]
