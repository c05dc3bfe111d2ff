"""CPU-only checks of the C ABI: the library builds, loads and exports every
symbol declared in include/*.h; its host-side layout helpers agree with the
oracle's independently written block layout (Section 2.3, Algorithm 5); the
update and cumulant tables pass their enumeration self-test.  No GPU calls."""
import ctypes
import glob
import itertools
import os
import re

import numpy as np
import pytest

import oracle
import paper_1701_06446_gb300 as cw
from paper_1701_06446_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(cumwin_\w+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_lib.load()._name)
    names = declared_functions()
    assert "cumwin_create" in names and "cumwin_push" in names
    for name in names:
        assert hasattr(lib, name), name
    # the binding declares exactly the header's functions
    assert set(_lib.SIGNATURES) == set(names)


def test_version_and_errors():
    lib = _lib.load()
    assert lib.cumwin_version() >= 100
    for code in range(0, -8, -1):
        assert lib.cumwin_strerror(code)
    assert lib.cumwin_batch_launches(None) == -1  # EINVAL, no device call
    with pytest.raises(ValueError):
        cw.layout_size(4, 2, 9)
    with pytest.raises(ValueError):
        cw.layout_size(0, 2, 3)


@pytest.mark.parametrize("n,b,s", [(4, 2, 4), (60, 3, 2), (60, 3, 3), (48, 4, 3), (7, 3, 4),
                                   (5, 2, 5), (3, 4, 6)])
def test_layout_size_and_rank_match_oracle(n, b, s):
    blocks = oracle.sorted_block_tuples(n, b, s)
    assert cw.layout_size(n, b, s) == len(blocks) * b ** s == oracle.layout_size(n, b, s)
    step = max(1, len(blocks) // 300)
    for r in range(0, len(blocks), step):
        assert cw.block_rank(n, b, s, blocks[r]) == r


@pytest.mark.parametrize("n,b,s", [(4, 2, 4), (7, 3, 3), (5, 2, 5), (6, 4, 2)])
def test_element_index_matches_oracle_layout(n, b, s):
    idx = oracle.block_elements(n, b, s)
    keep = np.all(idx < n, axis=1)
    for e in np.nonzero(keep)[0]:
        t = idx[e]
        got = cw.element_index(n, b, s, t)
        # storage index of the canonical (sorted) tuple holds the same multiset
        srt = np.sort(t)
        assert np.array_equal(np.sort(idx[got]), srt)
        for perm in itertools.permutations(t):
            assert cw.element_index(n, b, s, perm) == got


@pytest.mark.parametrize("n,b,s", [(4, 2, 1), (4, 2, 4), (60, 3, 2), (20, 3, 4), (7, 3, 5),
                                   (12, 4, 6), (9, 2, 6), (6, 2, 8), (5, 5, 3), (1, 1, 4),
                                   (24, 4, 5), (16, 4, 6), (13, 3, 6)])
def test_update_and_cumulant_tables_selftest(n, b, s):
    assert cw.selftest_tables(n, b, s) == 0


def test_bad_arguments_rejected_without_gpu():
    lib = _lib.load()
    h = ctypes.c_void_p()
    # argument checks run before any CUDA call
    for args in [(0, 4, 2, 100, 10), (4, 0, 2, 100, 10), (4, 9, 2, 100, 10), (4, 4, 0, 100, 10),
                 (4, 4, 2, 0, 1), (4, 4, 2, 100, 0), (4, 4, 2, 100, 101), (300, 2, 1, 10, 1),
                 (257, 2, 8, 10, 1), (250, 2, 43, 10, 1)]:  # above 256 variables, also once padded
        assert lib.cumwin_create(*args, 0, None, ctypes.byref(h)) == _lib.CODES["EINVAL"]
    assert lib.cumwin_create(4, 4, 2, 100, 10, 7, None, ctypes.byref(h)) == _lib.CODES["EINVAL"]
    assert lib.cumwin_push(None, None, None, 1, 4) == _lib.CODES["EINVAL"]
    assert lib.cumwin_norms(None, None, None) == _lib.CODES["EINVAL"]


def test_noalloc_norm_rejects_oversized_blocks_without_gpu():
    """The allocation-free norm bounds the block size as cumwin_create does (the
    padded variable count at most 256, b^order below 2^31) and returns EINVAL
    before any CUDA call; a non-null dummy pointer is never dereferenced."""
    lib = _lib.load()
    dummy = ctypes.c_void_p(16)
    # n=10, b=16, order 8: one block of 16^8 = 2^32 elements (would wrap to 0 in 32 bits)
    # n=200, b=150: 300 padded variables; n=256, b=256, order 4: 2^32 elements in one block
    for n, b, s in [(10, 16, 8), (200, 150, 2), (256, 256, 4), (9, 40, 6)]:
        rc = lib.cumwin_block_norm2_noalloc(n, b, s, dummy, dummy, None)
        assert rc == _lib.CODES["EINVAL"], (n, b, s, rc)
        assert "block size" in lib.cumwin_last_error().decode()
    for args in [(0, 2, 2), (4, 0, 2), (4, 2, 0), (4, 2, 9)]:
        assert lib.cumwin_block_norm2_noalloc(*args, dummy, dummy, None) == _lib.CODES["EINVAL"]
    assert lib.cumwin_block_norm2_noalloc(4, 2, 2, None, dummy, None) == _lib.CODES["EINVAL"]


@pytest.mark.parametrize("n,b,d,k", [(48, 4, 6, 2), (48, 4, 6, 8), (7, 3, 5, 3), (4, 2, 4, 2), (60, 3, 4, 5)])
def test_shard_blocks_partition_the_top_order(n, b, d, k):
    """The shards' block ranges are contiguous, cover every sorted block of order d
    once, and hold nearly equal block counts."""
    nb = len(oracle.sorted_block_tuples(n, b, d))
    ranges = [cw.shard_blocks(n, b, d, r, k) for r in range(k)]
    assert ranges[0][0] == 0 and ranges[-1][1] == nb
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0
    sizes = [e - s for s, e in ranges]
    assert max(sizes) - min(sizes) <= 1
    with pytest.raises(cw.CumwinError):
        cw.shard_blocks(n, b, d, k, k)


def test_estimators_from_squared_norms():
    fro2 = np.array([4.0, 9.0, 8.0, 3.0])
    fro, nu = cw.estimators_from_fro2(fro2)
    assert np.allclose(fro, np.sqrt(fro2))
    assert np.isnan(nu[:2]).all()
    assert np.allclose(nu[2:], [np.sqrt(8.0) / 3.0 ** 1.5, np.sqrt(3.0) / 3.0 ** 2])
