"""The GA-IBR-MPPI and perturbed-prediction planning calls at the full
ten-car size (n_v = 10, K = 16384, T = 60, L = 5, the benchmark's launch
shape), checked against the FP64 oracle on sampled best responses.

* GA-IBR-MPPI (lambda = 1e4): two responses recomputed in full by the
  oracle from the GPU's own inputs (all 16384 samples), under the
  tolerance of tests/test_gpu_mppi.py.
* Perturbed predictions (severe setting, (0.4, 0.2) m): for two responses,
  the oracle perturbs the GPU's previous-round predictions itself and
  evaluates the GPU's pick and 160 random candidates; the pick's
  trajectory must match and no sampled feasible candidate may beat it
  beyond the selection tolerance (as the SGTP full-size test)."""
import numpy as np
import pytest

import oracle as O
from paper_2607_25388_b300 import scenario as S
from tests.parity_util import STATE_RTOL, assert_rel_close
from tests.test_gpu_mppi import check_mppi_response, nominal_predictions
from tests.test_gpu_perturb import gpu_plan as gpu_plan_perturbed

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_full_size_mppi_plan_sampled_responses():
    from paper_2607_25388_b300 import planner as P
    from tests.test_gpu_mppi import gpu_plan
    sc = S.ten_car_race(200)
    p = S.params_fullscale()
    K, L, lam = sc.K, sc.L, 1.0e4
    g = gpu_plan(sc, p, K, L, seed=21, lam=lam)
    assert g["status"][0] == 0
    assert ((g["k_star"] >= 0) & (g["k_star"] < K)).all()
    trk = P.Track.from_data(sc.track)
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    nominal = nominal_predictions(sc, p)
    for rnd, i in ((2, 4), (L + 1, sc.ego)):
        check_mppi_response(sc, p, g, K, L, 21, lam, 0, rnd, i, trk, ot, nominal)


def test_full_size_perturbed_plan_sampled_responses():
    sc = S.ten_car_race(200)
    p = S.params_fullscale()
    K, L, T, sigma = sc.K, sc.L, sc.T, (0.4, 0.2)
    g = gpu_plan_perturbed(sc, p, K, L, seed=33, sigma=sigma)
    assert g["status"][0] == 0
    assert ((g["k_star"] >= 0) & (g["k_star"] < K)).all()
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    n_tail = O.tail_count(p["mu_tail"], T)
    rng = np.random.default_rng(2)
    for rnd, i in ((1, 0), (4, 7)):
        prev = g["xi_hist"][rnd - 1]
        u_nom = g["u_hist"][rnd - 1][i]
        others = [j for j in range(10) if j != i]
        opp = np.stack([prev[j] for j in others])
        pert = [O.perturb_prediction(ot, prev[j], T, 33, 0, i, rnd, j, sigma[0], sigma[1], n_tail) for j in others]
        opp_pos = np.stack([q[0] for q in pert])
        delta = np.stack([q[1] for q in pert])
        kg = int(g["k_star"][rnd * 10 + i])
        kl = np.unique(np.concatenate([[kg], rng.integers(0, K, 160)]))
        o = O.rollout_costs_perturbed(p, ot, sc.X0[i], u_nom, sc.vref_scale[i], opp, opp_pos, delta, T, k_list=kl,
                                      seed=33, agent=i, rnd=rnd, want_states=True)
        pos = int(np.nonzero(kl == kg)[0][0])
        assert_rel_close(g["xi_hist"][rnd][i], o["states"][pos], STATE_RTOL, f"round {rnd} agent {i} xi")
        feas, cost = o["feasible"].astype(bool), o["cost"]
        if feas[pos]:
            better = feas & (cost < cost[pos] - 1e-5 * max(1.0, abs(cost[pos])))
            assert not better.any(), f"round {rnd} agent {i}: a sampled candidate beats the GPU pick"
