"""Edge cases of the planning call against the oracle: a single vehicle (no
opponents), no Jacobi rounds (L = 0), one sample per response (K = 1), the
largest race (16 vehicles, 15 opponents) and the longest horizon
(T = 128).  Every best response is recomputed by the oracle from the GPU's
own inputs (teacher-forced, the rules of tests/parity_util.py)."""
import numpy as np
import pytest

from paper_2607_25388_b300 import scenario as S
from tests.test_gpu_plan_parity import gpu_plan, teacher_forced_check

pytestmark = pytest.mark.gpu


def _race(n_v, T, K, L, seed):
    return S.grid_race(S.fourier_track(seed, n_points=800), n_v, T, K, L, seed + 1)


@pytest.mark.parametrize("n_v,T,K,L,seed,n_check", [
    (1, 30, 64, 2, 701, None),        # a single vehicle: no opponents in any response
    (2, 20, 128, 0, 702, None),       # L = 0: round 0 and the extra ego response only
    (2, 25, 1, 1, 703, None),         # K = 1: the only sample is selected, feasible or not
    (16, 20, 256, 1, 704, 20),        # 16 vehicles: 15 opponents per response
    (2, 128, 96, 1, 705, None),       # the longest horizon, ragged K
])
def test_plan_edge_cases_teacher_forced(n_v, T, K, L, seed, n_check):
    sc = _race(n_v, T, K, L, seed)
    p = S.params_fullscale()
    g = gpu_plan(sc, p, K, L, seed=seed)
    assert g["status"][0] == 0
    assert ((g["k_star"] >= 0) & (g["k_star"] < K)).all()
    if K == 1:
        assert (g["k_star"] == 0).all()
    teacher_forced_check(sc, p, g, K, L, seed=seed, n_check=n_check)
    np.testing.assert_array_equal(g["U"], g["u_hist"][L + 1])


def test_plan_with_a_vehicle_facing_backwards():
    """One vehicle of a three-car race faces against the track direction at
    50 m/s, so its nominal and selected trajectories run about 95 segments
    backwards: the plan must report a clean status and every response must
    match the oracle's (teacher-forced)."""
    T, K, L = 60, 256, 1
    sc = S.grid_race(S.fourier_track(708), 3, T, K, L, 709)
    sc.X0[1, 2] += np.float32(np.pi)
    sc.X0[1, 3] = np.float32(50.0)
    p = S.params_fullscale()
    g = gpu_plan(sc, p, K, L, seed=4)
    assert g["status"][0] == 0
    teacher_forced_check(sc, p, g, K, L, seed=4)
