"""Closed-loop robustness: a ten-car race advanced through 25 consecutive
plans (each vehicle applies the first 10 steps of its plan, the warm start
shifts), as a receding-horizon controller would run it.  Every plan must
report a clean device status (no timed-out wait, no Frenet search that gave
up), finite trajectories and in-range selections."""
import numpy as np
import pytest

from paper_2607_25388_b300 import scenario as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_twenty_five_closed_loop_plans_stay_clean():
    from paper_2607_25388_b300 import learned as LR, planner as P
    p = S.params_fullscale()
    race = LR.Race(S.ten_car_race(205, K=4096, T=60, L=3))
    statuses = []
    for q in range(25):
        out = P.ibr_plan(race.track, p, race.X, race.U, race.vs, 60, 4096, 3, ego=0, seed=q)
        statuses.append(P.sync_status(out["status"]))
        xi = out["xi"].cpu().numpy()
        ks = out["k_star"].cpu().numpy()
        assert np.isfinite(xi).all(), f"plan {q}"
        assert ((ks >= 0) & (ks < 4096)).all(), f"plan {q}"
        race.advance(out["xi"], 10)
    assert statuses == [0] * 25, statuses
