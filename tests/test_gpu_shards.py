"""Block shards of the top order (cumwin_create_shard) on one GPU.

Each shard handle updates and recovers only its range of the top order's
blocks; run one after the other on the same samples (no shard waits on
another), their block ranges put together must equal the unsharded handle's
top-order cumulants, bitwise (the same kernels produce every element), the
orders below d must equal the unsharded ones on every shard, and the shards'
squared norms of the top order must add up to the unsharded one.  The
collectives that join shards on several GPUs are checked on CPU
(test_shard_gloo.py).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1701_06446_gb300 import CumWin, CumwinError, shard_blocks

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,d,b,nshards,form", [(24, 5, 4, 2, "bf16"), (20, 6, 4, 3, "fp16"), (13, 6, 3, 2, "bf16")])
def test_shards_put_together_equal_the_whole(n, d, b, nshards, form):
    T, p, steps = 512, 64, 6
    rng = np.random.default_rng(n * 10 + d)
    X = (rng.standard_t(6, size=(T + steps * p, n)) @ rng.standard_normal((n, n)) / np.sqrt(n) + 0.5)
    Xd = torch.from_numpy(X.astype(np.float32)).cuda()
    bs = b ** d
    with CumWin(n, d, b, T, p, form) as whole:
        whole.fill(Xd[:T])
        for w in range(steps):
            whole.push(Xd[T + w * p: T + (w + 1) * p])
        ref = [whole.cumulants(s) for s in range(1, d + 1)]
        ref_fro2 = whole.norms_device().cpu().numpy()
    top = torch.full_like(ref[d - 1], float("nan"))
    fro2_top = 0.0
    for k in range(nshards):
        lo, hi = shard_blocks(n, b, d, k, nshards)
        with CumWin(n, d, b, T, p, form, shard=k, nshards=nshards) as h:
            h.fill(Xd[:T])
            for w in range(steps):
                h.push(Xd[T + w * p: T + (w + 1) * p])
            for s in range(1, d):
                assert torch.equal(h.cumulants(s), ref[s - 1]), (k, s)
            top[lo * bs: hi * bs] = h.cumulants(d)[lo * bs: hi * bs]
            f2 = h.norms_device().cpu().numpy()
            assert np.array_equal(f2[: d - 1], ref_fro2[: d - 1])
            fro2_top += f2[d - 1]
    assert torch.equal(top, ref[d - 1])
    assert abs(fro2_top - ref_fro2[d - 1]) <= 1e-12 * ref_fro2[d - 1]
    # and against the oracle on sampled tuples of the top order
    Xw = X[steps * p:]
    tup = oracle.sample_sorted_tuples(n, d, 300, seed=d)
    idx = np.array([oracle.storage_index(n, b, t) for t in tup])
    want = oracle.cumulant_tuples(Xw, tup)
    got = top.cpu().numpy()[idx]
    assert np.linalg.norm(got - want) <= 1e-4 * np.linalg.norm(want)


def test_shard_arguments():
    for args, code in [((8, 4, 4, 256, 32, "bf16", 0, 2), -7),   # top order 4: not sharded
                       ((8, 5, 4, 256, 32, "fp64", 0, 2), -7),   # FP64 form
                       ((8, 5, 2, 256, 32, "bf16", 0, 2), -7),   # b^d = 32 < 256
                       ((8, 5, 4, 256, 32, "bf16", 2, 2), -1),   # shard out of range
                       ((8, 5, 4, 256, 32, "bf16", 0, 0), -1)]:
        n, d, b, T, p, form, k, m = args
        with pytest.raises(CumwinError) as ei:
            CumWin(n, d, b, T, p, form, shard=k, nshards=m)
        assert ei.value.code == code, args
    with CumWin(8, 5, 4, 256, 32, "bf16", shard=1, nshards=2) as h:
        h.fill(torch.randn(256, 8, device="cuda"))
        with pytest.raises(CumwinError) as ei:
            h.grad([0, 0, 0, 0, 1, 1])
        assert ei.value.code == -7
