"""Sharded batches on the GPU: races planned in shares (here three shares
planned one after the other on the one GPU of this process, as three ranks
would on three GPUs: nothing in a share waits for another) reassemble to the
one-GPU batch bit for bit, because every race keeps its global index as its
noise counter's race word."""
import numpy as np
import pytest

from paper_2607_25388_b300 import scenario as S
from paper_2607_25388_b300 import shard as SH

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_shares_reassemble_the_one_gpu_batch():
    p = S.params_fullscale()
    K, L = 1024, 2
    races = S.batched_races(n_races=24, K=K, L=L, seed0=3000, n_points=800)
    shapes = [(sc.X0.shape[0], sc.T) for sc in races]
    whole, _ = SH.plan_share(races, list(range(len(races))), K, L, p, seed=8)
    ref = SH.reassemble(whole, shapes, L)
    parts = {}
    for ids in SH.partition(shapes, 3, L):
        got, ms = SH.plan_share(races, ids, K, L, p, seed=8)
        assert ms > 0 and set(got) == set(ids)
        parts.update(got)
    out = SH.reassemble(parts, shapes, L)
    for a, b in zip(out, ref):
        np.testing.assert_array_equal(a, b)
