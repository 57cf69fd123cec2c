"""Pins of the oracle's GA-IBR-MPPI update (Sec. IV-A, second ablation):
the path-integral mean U_new = sum_k w_k U^(k) / sum_k w_k with
w_k = exp(-(c_k - c_min) / lambda), checked against what the mathematics
fixes rather than against a retyped formula:

* lambda -> 0: all weight on the lowest-cost sample, so U_new is that
  sample's controls (the SGTP argmin without the feasibility filter);
* lambda -> infinity: equal weights, so U_new is the plain mean of the
  sampled (clipped) controls;
* zero noise: every sample is the clipped nominal, so U_new is too;
* K = 1: the only sample;
* costs of order 1e6 at a small temperature: the shift by c_min keeps the
  weights finite, and a weighted mean stays inside the samples' range;
* the planning loop: with every sample feasible, the lambda -> 0 plan is
  exactly the SGTP plan (same responses, Jacobi order and extra ego round).
"""
import numpy as np

import oracle as O
from paper_2607_25388_b300 import scenario as S


def _oval_problem(K=96, T=30):
    sc = S.single_br_oval(K=K, T=T)
    p = S.params_fullscale()
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    return sc, p, ot


def _samples(sc, p, ot, K, T, **kw):
    return O.rollout_costs(p, ot, sc.X0[0], sc.U0[0], 1.0, sc.opp, T, K=K, seed=4, agent=1, rnd=1,
                           want_controls=True, **kw)


def test_small_temperature_gives_the_lowest_cost_sample():
    K, T = 96, 30
    sc, p, ot = _oval_problem(K, T)
    o = _samples(sc, p, ot, K, T)
    r = O.best_response_mppi(p, ot, sc.X0[0], sc.U0[0], 1.0, sc.opp, T, K, 1e-300, seed=4, agent=1, rnd=1)
    kb = int(np.argmin(o["cost"]))
    assert r["k_min"] == kb
    np.testing.assert_array_equal(r["u_new"], o["controls"][kb])
    np.testing.assert_allclose(r["xi_new"], O.rollout(p, sc.X0[0], o["controls"][kb], T), rtol=0, atol=1e-9)


def test_large_temperature_gives_the_sample_mean():
    K, T = 96, 30
    sc, p, ot = _oval_problem(K, T)
    o = _samples(sc, p, ot, K, T)
    r = O.best_response_mppi(p, ot, sc.X0[0], sc.U0[0], 1.0, sc.opp, T, K, 1e300, seed=4, agent=1, rnd=1)
    np.testing.assert_allclose(r["u_new"], o["controls"].mean(axis=0), rtol=1e-12, atol=1e-14)


def test_zero_noise_keeps_the_clipped_nominal():
    K, T = 40, 25
    sc, p, ot = _oval_problem(K, T)
    p = dict(p, sigma_a=0.0, sigma_delta=0.0)
    u_nom = sc.U0[0].astype(np.float64).copy()
    u_nom[::3, 0] = 50.0          # outside [a_min, a_max]
    u_nom[1::4, 1] = -2.0         # outside [-delta_max, delta_max]
    r = O.best_response_mppi(p, ot, sc.X0[0], u_nom, 1.0, sc.opp, T, K, 3.0e3, seed=2)
    f = {k: float(np.float32(p[k])) for k in ("a_min", "a_max", "delta_max")}   # the values the oracle receives
    want = np.stack([np.clip(u_nom[:, 0], f["a_min"], f["a_max"]),
                     np.clip(u_nom[:, 1], -f["delta_max"], f["delta_max"])], 1)
    np.testing.assert_allclose(r["u_new"], want, rtol=1e-15, atol=0)
    np.testing.assert_allclose(r["xi_new"], O.rollout(p, sc.X0[0], want, T), rtol=0, atol=1e-9)


def test_single_sample_is_returned_unchanged():
    T = 30
    sc, p, ot = _oval_problem(1, T)
    o = _samples(sc, p, ot, 1, T)
    r = O.best_response_mppi(p, ot, sc.X0[0], sc.U0[0], 1.0, sc.opp, T, 1, 7.0, seed=4, agent=1, rnd=1)
    assert r["k_min"] == 0
    np.testing.assert_allclose(r["u_new"], o["controls"][0], rtol=1e-15, atol=0)


def test_small_temperature_on_large_costs_stays_finite_and_in_range():
    K, T = 128, 60
    sc = S.ten_car_race(200, K=K, T=T, L=1)
    p = S.params_fullscale()
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    nominal = np.stack([O.rollout(p, sc.X0[i], sc.U0[i], T) for i in range(10)])
    opp = nominal[1:]
    o = O.rollout_costs(p, ot, sc.X0[0], sc.U0[0], sc.vref_scale[0], opp, T, K=K, seed=9, rnd=1,
                        want_controls=True)
    assert o["cost"].min() > 1e5                 # exp(-c / lambda) alone would underflow to 0 / 0
    lam = 50.0
    r = O.best_response_mppi(p, ot, sc.X0[0], sc.U0[0], sc.vref_scale[0], opp, T, K, lam, seed=9, rnd=1,
                             want_costs=True)
    np.testing.assert_array_equal(r["costs"], o["cost"])
    assert np.isfinite(r["u_new"]).all() and np.isfinite(r["xi_new"]).all()
    lo, hi = o["controls"].min(axis=0), o["controls"].max(axis=0)
    assert (r["u_new"] >= lo - 1e-12).all() and (r["u_new"] <= hi + 1e-12).all()
    # a weight of 1 on the best sample, under 1 on the rest: U_new moves toward it
    kb = int(np.argmin(o["cost"]))
    mean = o["controls"].mean(axis=0)
    assert np.abs(r["u_new"] - o["controls"][kb]).sum() < np.abs(mean - o["controls"][kb]).sum()


def test_plan_at_zero_temperature_equals_the_sgtp_plan_when_every_sample_is_feasible():
    """Feasibility thresholds set so that every sample passes: SGTP's
    selection is then the plain lowest-cost sample, which is the lambda -> 0
    limit of the path-integral update, in every response of the loop."""
    T, K, L = 20, 48, 2
    sc = S.grid_race(S.fourier_track(611, n_points=900), 3, T, K, L, 612)
    p = dict(S.params_fullscale(), m_bd=-1e9, d_col=-1e9)
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    a = O.ibr_plan(p, ot, sc.X0, sc.U0, sc.vref_scale, T, K, L, sc.ego, seed=6, want_hist=True)
    b = O.ibr_plan_mppi(p, ot, sc.X0, sc.U0, sc.vref_scale, T, K, L, sc.ego, 1e-300, seed=6, want_hist=True)
    np.testing.assert_array_equal(a["k_star"], b["k_star"])
    np.testing.assert_array_equal(a["u_hist"], b["u_hist"])
    np.testing.assert_allclose(b["xi_hist"], a["xi_hist"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(b["xi"], a["xi"], rtol=0, atol=1e-9)
