"""ctypes loader of ``libcumwin.so``: declares the C ABI of ``include/cumwin.h``.

There is no fallback: if the library cannot be built or loaded, importing the
binding raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_int, c_i64, c_vp, c_dp, c_fp = (ctypes.c_int, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float))
c_double = ctypes.c_double
_handle_p = ctypes.POINTER(c_vp)

# name -> (restype, argtypes)
SIGNATURES = {
    "cumwin_create": (c_int, [c_int, c_int, c_int, c_i64, c_int, c_int, c_vp, _handle_p]),
    "cumwin_destroy": (c_int, [c_vp]),
    "cumwin_set_stream": (c_int, [c_vp, c_vp]),
    "cumwin_fill": (c_int, [c_vp, c_vp, c_i64]),
    "cumwin_push": (c_int, [c_vp, c_vp, c_vp, c_int, c_i64]),
    "cumwin_push_host": (c_int, [c_vp, c_vp, c_int, c_i64]),
    "cumwin_cumulants": (c_int, [c_vp, c_int, c_vp]),
    "cumwin_moments": (c_int, [c_vp, c_int, c_vp]),
    "cumwin_full": (c_int, [c_vp, c_int, c_vp]),
    "cumwin_shift": (c_int, [c_vp, c_vp]),
    "cumwin_norms": (c_int, [c_vp, c_vp, c_vp]),
    "cumwin_norms_device": (c_int, [c_vp, c_vp]),
    "cumwin_recompute": (c_int, [c_vp]),
    "cumwin_recenter": (c_int, [c_vp]),
    "cumwin_window": (c_int, [c_vp, c_vp]),
    "cumwin_grad": (c_int, [c_vp, c_vp, c_vp]),
    "cumwin_status": (c_int, [c_vp]),
    "cumwin_set_timing": (c_int, [c_vp, c_int]),
    "cumwin_get_timing": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "cumwin_block_norm2_noalloc": (c_int, [c_int, c_int, c_int, c_vp, c_vp, c_vp]),
    "cumwin_tune": (c_int, [c_vp, c_int, c_vp]),
    "cumwin_fifo": (c_int, [c_vp]),
    "cumwin_join": (c_int, [c_vp]),
    "cumwin_norms_enqueue": (c_int, [c_vp, c_vp, c_vp]),
    "cumwin_set_pipeline": (c_int, [c_vp, c_int]),
    "cumwin_norms_k": (c_int, [c_vp, c_double, c_vp]),
    "cumwin_marginals": (c_int, [c_vp, c_vp, c_vp]),
    "cumwin_batch_create": (c_int, [c_int, c_vp, c_vp, c_vp, c_int, c_int, c_int, c_vp, _handle_p]),
    "cumwin_batch_destroy": (c_int, [c_vp]),
    "cumwin_batch_fill": (c_int, [c_vp, c_vp]),
    "cumwin_batch_offset": (c_i64, [c_vp, c_int]),
    "cumwin_batch_push": (c_int, [c_vp, c_vp]),
    "cumwin_batch_cumulants": (c_int, [c_vp, c_int, c_int, c_vp]),
    "cumwin_batch_norms": (c_int, [c_vp, c_vp, c_vp]),
    "cumwin_batch_tune": (c_int, [c_vp, c_int, c_vp]),
    "cumwin_batch_fifo": (c_int, [c_vp]),
    "cumwin_batch_status": (c_int, [c_vp]),
    "cumwin_batch_launches": (c_i64, [c_vp]),
    "cumwin_layout_size": (c_i64, [c_int, c_int, c_int]),
    "cumwin_block_rank": (c_i64, [c_int, c_int, c_int, c_vp]),
    "cumwin_element_index": (c_i64, [c_int, c_int, c_int, c_vp]),
    "cumwin_selftest_tables": (c_int, [c_int, c_int, c_int]),
    "cumwin_strerror": (ctypes.c_char_p, [c_int]),
    "cumwin_last_error": (ctypes.c_char_p, []),
    "cumwin_version": (c_int, []),
    "cumwin_set_allocator": (c_int, [c_vp, c_vp, c_vp]),
    "cumwin_estimators_enqueue": (c_int, [c_vp, c_vp, c_vp, c_vp]),
    "cumwin_loss": (c_int, [c_vp, c_vp, c_vp]),
    "cumwin_set_auto_recenter": (c_int, [c_vp, c_double]),
    "cumwin_drift": (c_int, [c_vp, c_vp, c_vp]),
    "cumwin_create_shard": (c_int, [c_int, c_int, c_int, c_i64, c_int, c_int, c_vp, c_int, c_int, _handle_p]),
    "cumwin_shard_blocks": (c_int, [c_int, c_int, c_int, c_int, c_int, c_vp, c_vp]),
    "cumwin_estimators_from_fro2": (c_int, [c_int, c_vp, c_vp, c_vp]),
    "cumwin_get_tiles": (c_int, [c_vp, c_vp, c_vp, c_vp]),
    "cumwin_set_tiles": (c_int, [c_vp, c_int, c_int, c_int]),
    "cumwin_batch_get_tiles": (c_int, [c_vp, c_vp, c_vp, c_vp]),
    "cumwin_batch_set_single_launch": (c_int, [c_vp, c_int]),
    "cumwin_device_bytes": (c_i64, [c_vp]),
}

# allocator callbacks of cumwin_set_allocator
ALLOC_FN = ctypes.CFUNCTYPE(c_int, c_vp, ctypes.c_size_t, c_vp, ctypes.POINTER(c_vp))
FREE_FN = ctypes.CFUNCTYPE(None, c_vp, c_vp, ctypes.c_size_t, c_vp)


def _torch_alloc(ctx, nbytes, stream, out):
    """Device memory for the library from PyTorch's caching allocator."""
    try:
        import torch
        dev = torch.cuda.current_device()
        out[0] = torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
        return 0
    except Exception:  # reported by the library as ENOMEM
        return 1


def _torch_free(ctx, ptr, nbytes, stream):
    try:
        import torch
        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:  # interpreter shutdown: the process gives the memory back
        pass


_TORCH_ALLOC = ALLOC_FN(_torch_alloc)
_TORCH_FREE = FREE_FN(_torch_free)
_installed = []  # callbacks currently installed (kept alive while the library may call them)


def set_allocator(alloc=None, free=None) -> None:
    """Install ctypes callbacks (ALLOC_FN / FREE_FN) as the library's allocator
    for handles created from now on; no arguments restores PyTorch's caching
    allocator, which the binding installs when it loads the library."""
    lib = load()
    if alloc is None and free is None:
        alloc, free = _TORCH_ALLOC, _TORCH_FREE
    _installed.append((alloc, free))
    check(lib.cumwin_set_allocator(ctypes.cast(alloc, c_vp), ctypes.cast(free, c_vp), None),
          "cumwin_set_allocator")


def path() -> str:
    return _build.OUT


def load():
    """Build (if stale) and load ``libcumwin.so``; raises on any failure."""
    global _lib
    with _lock:
        if _lib is None:
            so = _build.build()
            lib = ctypes.CDLL(so)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            # handles take their device memory from PyTorch's caching allocator
            if lib.cumwin_set_allocator(ctypes.cast(_TORCH_ALLOC, c_vp), ctypes.cast(_TORCH_FREE, c_vp),
                                        None) != 0:
                raise RuntimeError("cumwin_set_allocator failed")
            _lib = lib
    return _lib


class CumwinError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load()
        msg = lib.cumwin_strerror(code).decode()
        detail = lib.cumwin_last_error().decode()
        super().__init__(f"{where}: {msg} ({code})" + (f": {detail}" if detail else ""))
        self.code = code


def check(code: int, where: str) -> int:
    if code != 0:
        raise CumwinError(code, where)
    return code


CODES = dict(OK=0, EINVAL=-1, ENOMEM=-2, ECUDA=-3, ESTATE=-4, ENONFINITE=-5, ETIMEOUT=-6,
             ENOTSUP=-7)
PRECISION = {"fp64": 0, "bf16": 1, "fp16": 2}
