"""The benchmark's work counts, on the CPU: every roofline fraction that bench.py
reports divides one of these numbers by a measured time, so each is checked
here against an independent derivation (brute-force enumeration or a closed
form), not against itself.
"""
import itertools
import math
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from paper_1701_06446_gb300 import layout_size  # noqa: E402
from paper_1701_06446_gb300.streams import WORKLOADS  # noqa: E402


def canonical_digits(J, b):
    """Brute force: the in-block digit tuples of block tuple J whose digits do not
    decrease inside each run of equal block indices."""
    s = len(J)
    n = 0
    for a in itertools.product(range(b), repeat=s):
        if all(not (J[k] == J[k + 1] and a[k] > a[k + 1]) for k in range(s - 1)):
            n += 1
    return n


@pytest.mark.parametrize("nb,b,s", [(3, 2, 3), (2, 3, 4), (4, 2, 4), (3, 4, 3)])
def test_canonical_elements_are_the_multisets_of_variables(nb, b, s):
    """One canonical element per distinct entry of a super-symmetric tensor: the
    brute-force count over all sorted block tuples equals both the bench's
    per-block product formula summed and C(nb*b + s - 1, s)."""
    blocks = list(itertools.combinations_with_replacement(range(nb), s))
    brute = sum(canonical_digits(J, b) for J in blocks)
    formula = sum(bench._run_mask_count(J, b) for J in blocks)
    assert brute == formula == math.comb(nb * b + s - 1, s)


@pytest.mark.parametrize("n,b,s", [(8, 4, 5), (12, 4, 5), (8, 4, 6), (12, 4, 6)])
def test_gemm_outputs_brute_force(n, b, s):
    """Outputs of a canonical order's compressed update GEMM: for every sorted block
    tuple, (left-half digit rows canonical inside the left half) x (right-half
    columns canonical inside the right half), enumerated digit by digit."""
    assert bench.canonical_order(b, s)
    nb = -(-n // b)
    h = (s + 1) // 2
    brute = 0
    for J in itertools.combinations_with_replacement(range(nb), s):
        brute += canonical_digits(J[:h], b) * canonical_digits(J[h:], b)
    got = bench.gemm_outputs(n, b, s)
    assert got == brute
    assert math.comb(nb * b + s - 1, s) <= got <= layout_size(n, b, s)


def test_gemm_outputs_of_other_orders_are_every_stored_element():
    for n, b, s in [(48, 4, 4), (60, 3, 4), (10, 3, 5), (10, 2, 6)]:
        assert not bench.canonical_order(b, s)
        assert bench.gemm_outputs(n, b, s) == layout_size(n, b, s)


def test_n48_work_closed_forms():
    """n=48, b=4, d=6, p=2^12: the update needs every stored element of orders 1-4
    (E_s = C(12 + s - 1, s) 4^s) and the canonical elements of orders 5-6
    (C(48 + s - 1, s)); the recovery's two-word arithmetic is 12 FP32 operations
    per subset term (2^(s-1) - 1 terms) of those canonical elements."""
    W = WORKLOADS["n48_d6_b4_T65536_p4096"]
    E = {s: math.comb(12 + s - 1, s) * 4 ** s for s in range(1, 7)}
    assert [layout_size(48, 4, s) for s in range(1, 7)] == [E[s] for s in range(1, 7)]
    need = sum(E[s] for s in range(1, 5)) + math.comb(52, 5) + math.comb(53, 6)
    fifo = bench.algorithmic_work(W, True)
    full = bench.algorithmic_work(W, False)
    assert fifo["update"] == 2 * 4096 * need
    assert full["update"] == 2 * fifo["update"]
    assert fifo["recovery_fp32_ops"] == 12 * (15 * math.comb(52, 5) + 31 * math.comb(53, 6))
    assert fifo["computed_elements"][6] == math.comb(53, 6) == 22957480
    assert fifo["update_issued"] >= fifo["update"]
