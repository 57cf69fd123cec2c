"""The autotuner on a small problem: it measures every launch shape and
schedule, checks that each gives the identical plan, stores the fastest,
and the stored shape plans exactly like the default."""
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
    assert o is not None and o.block == best["block"] and o.schedule == best["schedule"]
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


def test_tune_batch_and_auto_shape_plan_identically(tmp_path):
    from paper_2607_25388_b300 import autotune as A, planner as P
    p = S.params_fullscale()
    races = S.batched_races(n_races=6, K=512, L=1, seed0=4000, n_points=600)
    trk = P.Track.from_many([sc.track for sc in races])
    b = P.Batch(trk, [dict(track_id=r, n_v=sc.X0.shape[0], T=sc.T, ego=sc.ego, race_tag=r)
                      for r, sc in enumerate(races)], K=512, L=1)
    X0 = torch.as_tensor(np.concatenate([sc.X0 for sc in races])).cuda()
    U0 = torch.as_tensor(np.concatenate([sc.U0.reshape(-1) for sc in races])).cuda()
    vs = torch.as_tensor(np.concatenate([sc.vref_scale for sc in races])).cuda()
    path = str(tmp_path / "tune.json")
    best = A.tune_batch(b, p, X0, U0, vs, reps=1, warmup=1, path=path)
    assert best["ms"] > 0 and A.lookup_batch(b, path) is not None
    import os
    os.environ["SGTP_AUTOTUNE_CACHE"] = path
    try:
        res = []
        for opts in (None, "auto"):
            U = U0.clone()
            out = b.plan(p, X0, U, vs, seed=3, opts=opts)
            torch.cuda.synchronize()
            res.append((out["xi"].cpu().numpy(), out["k_star"].cpu().numpy(), U.cpu().numpy()))
    finally:
        del os.environ["SGTP_AUTOTUNE_CACHE"]
    for x, y in zip(*res):
        np.testing.assert_array_equal(x, y)
