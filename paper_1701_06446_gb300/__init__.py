"""Sliding-window cumulant tensors on one GB300 GPU.

Python binding of ``libcumwin.so`` (C ABI in ``include/cumwin.h``).  Every
step of the path runs in the library's CUDA kernels; this module only
marshals arguments.  PyTorch supplies device memory and streams.

    cw = CumWin(n=60, d=4, b=3, T=32768, p=1024, precision="bf16")
    cw.fill(X0)             # first window, (T, n) float32 on the GPU
    cw.push(x_in)           # one window shift, (p, n) float32 on the GPU
    C4 = cw.cumulants(4)    # block layout, float64
    fro, nu = cw.norms()    # ||C_s||_F and nu_s (Eqs. me, mef)
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import CumwinError, check

__all__ = ["CumWin", "CumWinBatch", "CumwinError", "CumulantNormLoss", "layout_size", "block_rank",
           "element_index", "selftest_tables", "library_path", "shard_blocks", "estimators_from_fro2"]


def library_path() -> str:
    return _lib.path()


def layout_size(n: int, b: int, order: int) -> int:
    r = _lib.load().cumwin_layout_size(n, b, order)
    if r < 0:
        raise ValueError("bad layout arguments")
    return int(r)


def block_rank(n: int, b: int, order: int, j) -> int:
    arr = (ctypes.c_int * order)(*[int(x) for x in j])
    return int(_lib.load().cumwin_block_rank(n, b, order, arr))


def element_index(n: int, b: int, order: int, i) -> int:
    arr = (ctypes.c_int * order)(*[int(x) for x in i])
    return int(_lib.load().cumwin_element_index(n, b, order, arr))


def selftest_tables(n: int, b: int, order: int) -> int:
    return int(_lib.load().cumwin_selftest_tables(n, b, order))


def shard_blocks(n: int, b: int, d: int, shard: int, nshards: int) -> tuple[int, int]:
    """Block range [begin, end) of order d owned by shard `shard` of `nshards` (cumwin_shard_blocks)."""
    lo, hi = ctypes.c_int64(), ctypes.c_int64()
    check(_lib.load().cumwin_shard_blocks(n, b, d, shard, nshards, ctypes.byref(lo), ctypes.byref(hi)),
          "cumwin_shard_blocks")
    return lo.value, hi.value


def estimators_from_fro2(fro2) -> tuple[np.ndarray, np.ndarray]:
    """(||C_s||, nu_s) from squared norms of orders 1..d (cumwin_estimators_from_fro2)."""
    z = np.ascontiguousarray(np.asarray(fro2, dtype=np.float64))
    fro, nu = np.zeros(len(z)), np.zeros(len(z))
    check(_lib.load().cumwin_estimators_from_fro2(len(z), z.ctypes.data, fro.ctypes.data, nu.ctypes.data),
          "cumwin_estimators_from_fro2")
    return fro, nu


def _dev_ptr(t: torch.Tensor, dtype: torch.dtype, name: str) -> int:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    return t.data_ptr()


class CumWin:
    """One sliding window of an n-variate stream with cumulants of orders 1..d."""

    def __init__(self, n: int, d: int, b: int, T: int, p: int, precision: str = "fp64",
                 device=None, shard: int = 0, nshards: int = 1):
        self.lib = _lib.load()
        if precision not in _lib.PRECISION:
            raise ValueError(f"precision must be one of {list(_lib.PRECISION)}")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.n, self.d, self.b, self.T, self.p = n, d, b, T, p
        self.precision = precision
        self.shard, self.nshards = shard, nshards
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            self._stream = torch.cuda.current_stream(self.device).cuda_stream
            check(self.lib.cumwin_create_shard(n, d, b, T, p, _lib.PRECISION[precision],
                                               ctypes.c_void_p(self._stream), shard, nshards,
                                               ctypes.byref(self._h)),
                  "cumwin_create_shard")
        self.sizes = [layout_size(n, b, s) for s in range(1, d + 1)]

    # -- stream management ---------------------------------------------------
    def _sync_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        if s != self._stream:
            check(self.lib.cumwin_set_stream(self._h, ctypes.c_void_p(s)), "cumwin_set_stream")
            self._stream = s

    def close(self):
        if self._h:
            self.lib.cumwin_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- the path --------------------------------------------------------------
    def fill(self, X: torch.Tensor):
        if X.dim() != 2 or X.shape[0] != self.T or X.shape[1] < self.n or X.stride(1) != 1:
            raise ValueError("fill expects a (T, n) float32 tensor with unit column stride")
        self._sync_stream()
        check(self.lib.cumwin_fill(self._h, _dev_ptr(X, torch.float32, "X"), X.stride(0)),
              "cumwin_fill")

    def push(self, x_in: torch.Tensor, x_out: torch.Tensor | None = None):
        if x_in.dim() != 2 or x_in.shape[1] < self.n or x_in.stride(1) != 1:
            raise ValueError("push expects (p, n) float32 tensors with unit column stride")
        p = x_in.shape[0]
        out_ptr = None
        if x_out is not None:
            if x_out.shape != x_in.shape or x_out.stride() != x_in.stride():
                raise ValueError("x_out must match x_in in shape and strides")
            out_ptr = ctypes.c_void_p(_dev_ptr(x_out, torch.float32, "x_out"))
        self._sync_stream()
        check(self.lib.cumwin_push(self._h, _dev_ptr(x_in, torch.float32, "x_in"), out_ptr, p,
                                   x_in.stride(0)), "cumwin_push")

    def join(self):
        """Make the current stream wait (on the device) for the last pipelined push."""
        self._sync_stream()
        check(self.lib.cumwin_join(self._h), "cumwin_join")

    def set_pipeline(self, enable: bool):
        """Overlap each push's recovery with the next push's update (the default) or not."""
        self._sync_stream()
        check(self.lib.cumwin_set_pipeline(self._h, int(bool(enable))), "cumwin_set_pipeline")

    def push_host(self, x_in):
        """Shift with X_(+) in host memory (numpy array or CPU tensor, pinned if possible)."""
        if isinstance(x_in, torch.Tensor):
            if x_in.is_cuda or x_in.dtype != torch.float32:
                raise ValueError("push_host expects a CPU float32 tensor")
            ptr, p, ld = x_in.data_ptr(), x_in.shape[0], x_in.stride(0)
        else:
            x_in = np.ascontiguousarray(x_in, dtype=np.float32)
            ptr, p, ld = x_in.ctypes.data, x_in.shape[0], x_in.shape[1]
        self._sync_stream()
        check(self.lib.cumwin_push_host(self._h, ctypes.c_void_p(ptr), p, ld), "cumwin_push_host")

    def _order(self, order: int):
        if not 1 <= order <= self.d:
            raise ValueError(f"order must be in 1..{self.d}")

    def cumulants(self, order: int, out: torch.Tensor | None = None) -> torch.Tensor:
        self._order(order)
        if out is None:
            out = torch.empty(self.sizes[order - 1], dtype=torch.float64, device=self.device)
        self._sync_stream()
        check(self.lib.cumwin_cumulants(self._h, order, _dev_ptr(out, torch.float64, "out")),
              "cumwin_cumulants")
        return out

    def full(self, order: int) -> torch.Tensor:
        """C_order as the full super-symmetric n^order tensor (cumwin_full)."""
        self._order(order)
        out = torch.empty((self.n,) * order, dtype=torch.float64, device=self.device)
        self._sync_stream()
        check(self.lib.cumwin_full(self._h, order, _dev_ptr(out, torch.float64, "out")), "cumwin_full")
        return out

    def moments(self, order: int) -> torch.Tensor:
        self._order(order)
        out = torch.empty(self.sizes[order - 1], dtype=torch.float64, device=self.device)
        self._sync_stream()
        check(self.lib.cumwin_moments(self._h, order, out.data_ptr()), "cumwin_moments")
        return out

    def shift(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.float32)
        self._sync_stream()
        check(self.lib.cumwin_shift(self._h, out.ctypes.data), "cumwin_shift")
        return out

    def norms(self) -> tuple[np.ndarray, np.ndarray]:
        fro = np.zeros(self.d)
        nu = np.zeros(self.d)
        self._sync_stream()
        check(self.lib.cumwin_norms(self._h, fro.ctypes.data, nu.ctypes.data), "cumwin_norms")
        return fro, nu

    def norms_device(self, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.d, dtype=torch.float64, device=self.device)
        self._sync_stream()
        check(self.lib.cumwin_norms_device(self._h, _dev_ptr(out, torch.float64, "out")),
              "cumwin_norms_device")
        return out

    def norms_enqueue(self, fro2_out: torch.Tensor, status_out: torch.Tensor | None = None):
        """Enqueue copies of ||C_s||^2 (d float64) and of the device status (int32)
        into the given tensors (CUDA, or host memory: pinned for an asynchronous
        copy, pageable makes the copy synchronous), behind the last push's
        recovery; valid after ``join()`` and a synchronisation (see cumwin_norms_enqueue)."""
        def ptr(t, dtype, count, what):
            if t.dtype != dtype or not t.is_contiguous() or t.numel() < count:
                raise ValueError(f"{what} must be a contiguous {dtype} tensor of at least {count} elements")
            return ctypes.c_void_p(t.data_ptr())
        sp = ptr(status_out, torch.int32, 1, "status_out") if status_out is not None else None
        self._sync_stream()
        check(self.lib.cumwin_norms_enqueue(self._h, ptr(fro2_out, torch.float64, self.d, "fro2_out"), sp),
              "cumwin_norms_enqueue")

    def estimators_enqueue(self, fro_out: torch.Tensor | None = None, nu_out: torch.Tensor | None = None,
                           status_out: torch.Tensor | None = None):
        """Enqueue ||C_s||_F and nu_s (d float64 each, formed on the device) and the
        device status (int32) into the given tensors (CUDA or host memory), behind
        the last push's recovery; valid after ``join()`` and a synchronisation
        (see cumwin_estimators_enqueue)."""
        def ptr(t, dtype, count, what):
            if t is None:
                return None
            if t.dtype != dtype or not t.is_contiguous() or t.numel() < count:
                raise ValueError(f"{what} must be a contiguous {dtype} tensor of at least {count} elements")
            return ctypes.c_void_p(t.data_ptr())
        args = (ptr(fro_out, torch.float64, self.d, "fro_out"), ptr(nu_out, torch.float64, self.d, "nu_out"),
                ptr(status_out, torch.int32, 1, "status_out"))
        if all(a is None for a in args):
            raise ValueError("give at least one output")
        self._sync_stream()
        check(self.lib.cumwin_estimators_enqueue(self._h, *args), "cumwin_estimators_enqueue")

    def loss(self, w, out: torch.Tensor | None = None) -> torch.Tensor:
        """L = sum_s w[s] ||C_s||_F^2 of the current window as a 0-d float64 CUDA tensor
        (cumwin_loss; w[0] ignored)."""
        wa = np.zeros(self.d + 1)
        wv = np.asarray(w, dtype=np.float64)[: self.d + 1]
        wa[:len(wv)] = wv
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=self.device)
        self._sync_stream()
        check(self.lib.cumwin_loss(self._h, wa.ctypes.data, _dev_ptr(out, torch.float64, "out")), "cumwin_loss")
        return out

    def recompute(self):
        self._sync_stream()
        check(self.lib.cumwin_recompute(self._h), "cumwin_recompute")

    def recenter(self):
        """Re-fix the shift at the window's column means and recompute about it (cumwin_recenter)."""
        self._sync_stream()
        check(self.lib.cumwin_recenter(self._h), "cumwin_recenter")

    def set_auto_recenter(self, limit: float):
        """Re-centre automatically when the mean drifts more than `limit` standard
        deviations from the shift (cumwin_set_auto_recenter; 0 turns it off)."""
        self._sync_stream()
        check(self.lib.cumwin_set_auto_recenter(self._h, ctypes.c_double(limit)), "cumwin_set_auto_recenter")

    def drift(self) -> tuple[float, int]:
        """(last measured drift ratio, automatic re-centrings so far) (cumwin_drift)."""
        r, k = ctypes.c_double(), ctypes.c_int64()
        self._sync_stream()
        check(self.lib.cumwin_drift(self._h, ctypes.byref(r), ctypes.byref(k)), "cumwin_drift")
        return r.value, k.value

    def window(self) -> torch.Tensor:
        out = torch.empty(self.T, self.n, dtype=torch.float32, device=self.device)
        self._sync_stream()
        check(self.lib.cumwin_window(self._h, out.data_ptr()), "cumwin_window")
        return out

    def grad(self, w) -> torch.Tensor:
        """d(sum_s w[s] ||C_s||_F^2)/d window (T x n, oldest sample first)."""
        wa = np.zeros(self.d + 1)
        wa[:len(w)] = np.asarray(w, dtype=np.float64)[: self.d + 1]
        out = torch.empty(self.T, self.n, dtype=torch.float32, device=self.device)
        self._sync_stream()
        check(self.lib.cumwin_grad(self._h, wa.ctypes.data, out.data_ptr()), "cumwin_grad")
        return out

    def set_timing(self, enable=True):
        """Phase timing of later shifts (see cumwin_set_timing): True / 1 splits each
        shift into staging, update and recovery; 2 leaves the staging inside the
        update (no event between the operand build and the GEMM)."""
        level = int(enable) if not isinstance(enable, bool) else int(enable)
        check(self.lib.cumwin_set_timing(self._h, level), "cumwin_set_timing")

    def get_timing(self) -> dict:
        a, u, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        k, L = ctypes.c_int64(), ctypes.c_int64()
        check(self.lib.cumwin_get_timing(self._h, ctypes.byref(a), ctypes.byref(u), ctypes.byref(c),
                                         ctypes.byref(k), ctypes.byref(L)), "cumwin_get_timing")
        return {"stage_ms": a.value, "update_ms": u.value, "cumulant_ms": c.value,
                "shifts": k.value, "launches": L.value}

    def tune(self, reps: int = 5) -> int:
        """Autotune the tensor-core update (K-split) on the last shift's data."""
        ks = ctypes.c_int()
        self._sync_stream()
        check(self.lib.cumwin_tune(self._h, reps, ctypes.byref(ks)), "cumwin_tune")
        return ks.value

    def tiles(self) -> dict:
        """The update's tile choice (cumwin_get_tiles): K-split, rows per item, super-block height."""
        a, b_, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(self.lib.cumwin_get_tiles(self._h, ctypes.byref(a), ctypes.byref(b_), ctypes.byref(c)),
              "cumwin_get_tiles")
        return {"ksplit": a.value, "rows_per_item": b_.value, "group": c.value}

    def set_tiles(self, ksplit: int, rows_per_item: int, group: int):
        """Pin the update's tile choice (cumwin_set_tiles)."""
        self._sync_stream()
        check(self.lib.cumwin_set_tiles(self._h, ksplit, rows_per_item, group), "cumwin_set_tiles")

    def norms_k(self, k: float) -> np.ndarray:
        """Entry-wise k-norms ||C_s||_k, s = 1..d (Algorithm 5 with a general k >= 1)."""
        out = np.zeros(self.d)
        self._sync_stream()
        check(self.lib.cumwin_norms_k(self._h, ctypes.c_double(k), out.ctypes.data), "cumwin_norms_k")
        return out

    def marginals(self):
        """Per-variable skewness and excess kurtosis of the window (NaN above order d)."""
        sk = np.zeros(self.n)
        ku = np.zeros(self.n)
        self._sync_stream()
        check(self.lib.cumwin_marginals(self._h, sk.ctypes.data, ku.ctypes.data), "cumwin_marginals")
        return sk, ku

    @property
    def fifo(self) -> bool:
        """True when the next nominal shift uses the batch-sum FIFO (see cumwin_push)."""
        r = int(self.lib.cumwin_fifo(self._h))
        check(min(r, 0), "cumwin_fifo")
        return r == 1

    def status(self) -> int:
        self._sync_stream()
        return int(self.lib.cumwin_status(self._h))


class CumWinBatch:
    """Many independent windows (uneven n, d, T; shared b, p, precision) advanced together."""

    def __init__(self, ns, ds, Ts, b: int, p: int, precision: str = "bf16", device=None):
        self.lib = _lib.load()
        if precision not in _lib.PRECISION:
            raise ValueError(f"precision must be one of {list(_lib.PRECISION)}")
        self.ns, self.ds, self.Ts = list(map(int, ns)), list(map(int, ds)), list(map(int, Ts))
        if not (len(self.ns) == len(self.ds) == len(self.Ts)) or not self.ns:
            raise ValueError("ns, ds and Ts must be non-empty and of equal length")
        self.nwin, self.b, self.p = len(self.ns), b, p
        self.dmax = max(self.ds)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self._h = ctypes.c_void_p()
        na = (ctypes.c_int * self.nwin)(*self.ns)
        da = (ctypes.c_int * self.nwin)(*self.ds)
        ta = (ctypes.c_int64 * self.nwin)(*self.Ts)
        with torch.cuda.device(self.device):
            self._stream = torch.cuda.current_stream(self.device).cuda_stream
            check(self.lib.cumwin_batch_create(self.nwin, na, da, ta, b, p, _lib.PRECISION[precision],
                                               ctypes.c_void_p(self._stream), ctypes.byref(self._h)),
                  "cumwin_batch_create")
        self.offsets = [int(self.lib.cumwin_batch_offset(self._h, i)) for i in range(self.nwin + 1)]

    def close(self):
        if self._h:
            self.lib.cumwin_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check_stream(self):
        if torch.cuda.current_stream(self.device).cuda_stream != self._stream:
            raise RuntimeError("a batch issues its work on the stream current at creation")

    def fill(self, Xs):
        if len(Xs) != self.nwin:
            raise ValueError("one first window per stream")
        ptrs = []
        for X, n, T in zip(Xs, self.ns, self.Ts):
            if X.shape != (T, n) or not X.is_contiguous():
                raise ValueError("window i must be a contiguous (T_i, n_i) float32 tensor")
            ptrs.append(_dev_ptr(X, torch.float32, "X"))
        self._check_stream()
        arr = (ctypes.c_void_p * self.nwin)(*ptrs)
        check(self.lib.cumwin_batch_fill(self._h, arr), "cumwin_batch_fill")

    def pack(self, rows) -> torch.Tensor:
        """Concatenate the p new rows of every window into the packed push layout."""
        return torch.cat([r.reshape(-1) for r in rows]).contiguous()

    def push(self, x_packed: torch.Tensor):
        if x_packed.dim() != 1 or x_packed.numel() < self.offsets[-1]:
            raise ValueError("push expects the packed rows of all windows")
        self._check_stream()
        check(self.lib.cumwin_batch_push(self._h, _dev_ptr(x_packed, torch.float32, "x")),
              "cumwin_batch_push")

    def cumulants(self, window: int, order: int) -> torch.Tensor:
        if not 0 <= window < self.nwin or not 1 <= order <= self.ds[window]:
            raise ValueError("bad window or order")
        out = torch.empty(layout_size(self.ns[window], self.b, order), dtype=torch.float64,
                          device=self.device)
        check(self.lib.cumwin_batch_cumulants(self._h, window, order, out.data_ptr()),
              "cumwin_batch_cumulants")
        return out

    def norms(self):
        fro = np.zeros((self.nwin, self.dmax))
        nu = np.zeros((self.nwin, self.dmax))
        check(self.lib.cumwin_batch_norms(self._h, fro.ctypes.data, nu.ctypes.data), "cumwin_batch_norms")
        return fro, nu

    def tune(self, reps: int = 5) -> int:
        ks = ctypes.c_int()
        check(self.lib.cumwin_batch_tune(self._h, reps, ctypes.byref(ks)), "cumwin_batch_tune")
        return ks.value

    def tiles(self) -> dict:
        """The update's tile choice (cumwin_batch_get_tiles)."""
        a, b_, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(self.lib.cumwin_batch_get_tiles(self._h, ctypes.byref(a), ctypes.byref(b_), ctypes.byref(c)),
              "cumwin_batch_get_tiles")
        return {"ksplit": a.value, "rows_per_item": b_.value, "group": c.value}

    @property
    def fifo(self) -> bool:
        """True when the batch's shifts use the batch-sum FIFO."""
        r = int(self.lib.cumwin_batch_fifo(self._h))
        check(min(r, 0), "cumwin_batch_fifo")
        return r == 1

    def status(self) -> int:
        return int(self.lib.cumwin_batch_status(self._h))

    def set_single_launch(self, enable: bool) -> bool:
        """Run each shift as one cooperative launch (the default where available) or
        phase by phase; returns whether single-launch shifts are available."""
        r = int(self.lib.cumwin_batch_set_single_launch(self._h, int(bool(enable))))
        check(min(r, 0), "cumwin_batch_set_single_launch")
        return r == 1

    def launches(self) -> int:
        """Kernels launched by the last push."""
        r = int(self.lib.cumwin_batch_launches(self._h))
        check(min(r, 0), "cumwin_batch_launches")
        return r


class CumulantNormLoss(torch.autograd.Function):
    """L(X) = sum_s w[s] ||C_s(X)||_F^2 for a window X (T x n), with a hand-written adjoint.

    Forward loads X as a fresh window into a handle and has the library form L
    on the device (``cumwin_loss``); backward calls ``cumwin_grad`` on the same
    handle.
    """

    @staticmethod
    def forward(ctx, X: torch.Tensor, w, b: int = 4):
        T, n = X.shape
        d = len(w) - 1
        cw = CumWin(n, d, b, T, T, "fp64", device=X.device)
        cw.fill(X.detach().contiguous())
        ctx.cw = cw
        ctx.w = list(w)
        return cw.loss(w)  # formed by the library on the device (cumwin_loss)

    @staticmethod
    def backward(ctx, gout):
        g = ctx.cw.grad(ctx.w)
        ctx.cw.close()
        return (g * gout.to(g.dtype)).to(torch.float32), None, None
