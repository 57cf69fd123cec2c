"""The trial metrics of the library (sim.trial_metrics, host logic) against
the paper's definitions worked by hand (Sec. IV-C, Evaluation Metrics):
Wins, CFW among the wins, FPR from the final unwrapped progress, durations,
CSD, mean ego speed and MCS."""
import numpy as np
import pytest


def test_trial_metrics_by_hand():
    from paper_2607_25388_b300.sim import trial_metrics
    base = dict(n_v=3, ego=0, alive=0, close_segments=0, close_steps=0, d=np.zeros(3))
    rs = [
        # ego gains 10 m vs 5 and 7; started 3 m and 6 m behind them: ahead of opponent 1 only at the end
        dict(base, steps=100, ego_collision=0, ego_speed_sum=100 * 40.0, ego_du2_sum=0.99,
             progress=np.array([10.0, 5.0, 7.0]), rel0=np.array([0.0, 3.0, 6.0]), close_segments=2, close_steps=30),
        # ego gains less than opponent 2: no win, ahead of nobody; contact with a vehicle at step 50
        dict(base, steps=50, ego_collision=1, ego_speed_sum=50 * 30.0, ego_du2_sum=4.9,
             progress=np.array([6.0, 5.0, 7.0]), rel0=np.array([0.0, 3.0, 6.0]), close_segments=1, close_steps=10),
        # a win ended by a wall contact, ahead of both
        dict(base, steps=20, ego_collision=2, ego_speed_sum=20 * 50.0, ego_du2_sum=0.0,
             progress=np.array([30.0, 5.0, 7.0]), rel0=np.array([0.0, 3.0, 6.0])),
    ]
    m = trial_metrics(rs, dt=0.05, limit_s=50.0, eps_s=0.025)
    assert m["wins"] == pytest.approx(2 / 3)
    assert m["cfw"] == pytest.approx(1 / 2)
    assert m["fpr"] == pytest.approx((0.5 + 0.0 + 1.0) / 3)
    assert m["d_mean"] == pytest.approx((5.0 + 2.5 + 1.0) / 3)
    assert m["d_max"] == pytest.approx(5.0)
    assert m["d_ratio"] == pytest.approx((5.0 + 2.5 + 1.0) / 3 / 50.0)
    assert m["csd"] == pytest.approx(40 * 0.05 / 3)
    assert m["v_ego"] == pytest.approx((4000 + 1500 + 1000) / 170)
    assert m["mcs"] == pytest.approx((0.99 / 99 + 4.9 / 49 + 0.0) / 3)
    assert m["contacts"] == pytest.approx(2 / 3)
