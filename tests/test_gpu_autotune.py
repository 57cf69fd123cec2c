"""The autotuner on a small problem: it measures every launch shape, checks
that each gives the identical plan, stores the fastest, and the stored shape
plans exactly like the default."""
import numpy as np
import pytest

from paper_2607_25388_b300 import scenario as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_tune_store_lookup_and_invariance(tmp_path):
    from paper_2607_25388_b300 import autotune as A, planner as P
    path = str(tmp_path / "tune.json")
    best = A.tune(3, 24, 512, 1, reps=2, warmup=1, path=path)
    assert ((best["block"], best["samples_per_thread"]) in A.SHAPES or best["block"] == 0) and best["ms"] > 0
    o = A.lookup(3, 24, 512, 1, path)
    assert o is not None and o.block == best["block"]
    sc = S.grid_race(S.fourier_track(778), 3, 24, 512, 1, 779)
    p = S.params_fullscale()
    trk = P.Track.from_data(sc.track)
    res = []
    for opts in (None, o):
        U = torch.as_tensor(sc.U0.copy()).cuda()
        out = P.ibr_plan(trk, p, torch.as_tensor(sc.X0).cuda(), U, torch.as_tensor(sc.vref_scale).cuda(), 24, 512, 1,
                         seed=9, opts=opts)
        torch.cuda.synchronize()
        res.append((out["xi"].cpu().numpy(), out["k_star"].cpu().numpy()))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    np.testing.assert_array_equal(res[0][1], res[1][1])
