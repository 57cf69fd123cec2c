"""Pins of the oracle's perturbed opponent predictions (robustness study of
Sec. IV, Table II; plain Gaussian noise in Frenet coordinates, first order):

* on a straight the raceline direction is +x, so the longitudinal noise
  moves points along x only and the lateral noise along y only;
* the displacements have zero mean and standard deviations sigma_lon and
  sigma_lat (statistics over thousands of steps), uncorrelated;
* on a circular arc a purely longitudinal displacement is tangent to the
  arc (up to the half-segment chord angle);
* the summary shifts equal the last step's longitudinal displacement and
  the tail mean of the lateral ones;
* the noise is not the samples' noise (its counter carries the 2^30 tag)
  and differs between observers;
* with zero sigma the perturbed plan is the SGTP plan.
"""
import math

import numpy as np

import oracle as O
from paper_2607_25388_b300 import scenario as S


def _oval():
    td = S.oval_track()
    return td, O.Track(td.xr, td.wl, td.wr)


def _straight_traj(T, x0=10.0, y0=1.0, v=1.4):
    st = np.zeros((T + 1, 4))
    st[:, 0] = x0 + v * np.arange(T + 1)
    st[:, 1] = y0
    st[:, 3] = 28.0
    return st


def test_straight_frame_and_statistics():
    td, ot = _oval()
    T = 120
    st = _straight_traj(T)
    dx, dy = [], []
    for obs in range(4):
        for rnd in range(4):
            for jv in range(4):
                out, _ = O.perturb_prediction(ot, st, T, 77, 5, obs, rnd, jv, 0.4, 0.2, 36)
                assert np.array_equal(out[0], st[0]) and np.array_equal(out[:, 2:], st[:, 2:])
                dx.append(out[1:, 0] - st[1:, 0])
                dy.append(out[1:, 1] - st[1:, 1])
    dx, dy = np.concatenate(dx), np.concatenate(dy)
    n = dx.size
    assert abs(dx.mean()) < 4 * 0.4 / math.sqrt(n) and abs(dy.mean()) < 4 * 0.2 / math.sqrt(n)
    assert abs(dx.std() / 0.4 - 1) < 0.05 and abs(dy.std() / 0.2 - 1) < 0.05
    assert abs(np.corrcoef(dx, dy)[0, 1]) < 4 / math.sqrt(n)
    # longitudinal noise alone moves points along x only, lateral alone along y only
    a, _ = O.perturb_prediction(ot, st, T, 77, 5, 1, 2, 3, 0.4, 0.0, 36)
    b, _ = O.perturb_prediction(ot, st, T, 77, 5, 1, 2, 3, 0.0, 0.2, 36)
    np.testing.assert_allclose(a[:, 1], st[:, 1], atol=1e-12)
    np.testing.assert_allclose(b[:, 0], st[:, 0], atol=1e-12)


def test_arc_longitudinal_noise_is_tangent():
    td, ot = _oval()
    R, cx, cy = 50.0, 200.0, 50.0          # first semicircle of the oval
    T = 30
    th = np.linspace(0.2, 2.9, T + 1)       # the semicircle spans theta in [0, pi]
    st = np.zeros((T + 1, 4))
    st[:, 0] = cx + (R - 1.0) * np.sin(th)
    st[:, 1] = cy - (R - 1.0) * np.cos(th)
    out, _ = O.perturb_prediction(ot, st, T, 3, 0, 0, 1, 1, 0.5, 0.0, 9)
    disp = out[1:, :2] - st[1:, :2]
    radial = np.stack([np.sin(th[1:]), -np.cos(th[1:])], 1)
    cosang = np.abs((disp * radial).sum(1)) / np.maximum(np.hypot(disp[:, 0], disp[:, 1]), 1e-12)
    assert cosang.max() < 0.03          # half the chord angle of 1.785 m segments on R = 50 m is 0.018 rad


def test_summary_shifts_follow_the_displacements():
    td, ot = _oval()
    T, n_tail = 40, 12
    st = _straight_traj(T)
    out, delta = O.perturb_prediction(ot, st, T, 11, 2, 3, 1, 4, 0.3, 0.15, n_tail)
    assert abs(delta[0] - (out[T, 0] - st[T, 0])) < 1e-12
    assert abs(delta[1] - (out[T - n_tail + 1:, 1] - st[T - n_tail + 1:, 1]).mean()) < 1e-12


def test_noise_is_not_the_samples_and_differs_by_observer():
    td, ot = _oval()
    T = 20
    st = _straight_traj(T)
    out, _ = O.perturb_prediction(ot, st, T, 9, 1, 2, 3, 4, 1.0, 1.0, 6)
    z = np.stack([out[1:, 0] - st[1:, 0], out[1:, 1] - st[1:, 1]], 1)
    sample = np.array([O.std_normals(9, 1, 2, 3, 0, 4, tau) for tau in range(T)])   # sample k = 4's noise
    assert np.abs(z - sample).max() > 0.1
    other, _ = O.perturb_prediction(ot, st, T, 9, 1, 5, 3, 4, 1.0, 1.0, 6)
    assert np.abs(other - out).max() > 0.1


def test_zero_sigma_plan_is_the_sgtp_plan():
    T, K, L = 20, 64, 2
    sc = S.grid_race(S.fourier_track(621, n_points=900), 3, T, K, L, 622)
    p = S.params_fullscale()
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    a = O.ibr_plan(p, ot, sc.X0, sc.U0, sc.vref_scale, T, K, L, sc.ego, seed=4, want_hist=True)
    b = O.ibr_plan_perturbed(p, ot, sc.X0, sc.U0, sc.vref_scale, T, K, L, sc.ego, 0.0, 0.0, seed=4, want_hist=True)
    for k in ("k_star", "u_hist", "xi_hist", "xi", "u_nom"):
        np.testing.assert_array_equal(a[k], b[k])
    c = O.ibr_plan_perturbed(p, ot, sc.X0, sc.U0, sc.vref_scale, T, K, L, sc.ego, 0.4, 0.2, seed=4, want_hist=True)
    assert not np.array_equal(a["k_star"], c["k_star"])     # the noise reaches the responses


def test_perturbed_candidate_costs_reduce_to_the_plain_ones_at_zero_sigma():
    """The perturbed evaluation with unperturbed positions and zero shifts is
    the plain evaluation, candidate by candidate."""
    sc = S.single_br_oval(K=64, T=30)
    p = S.params_fullscale()
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    a = O.rollout_costs(p, ot, sc.X0[0], sc.U0[0], 1.0, sc.opp, sc.T, K=64, seed=2, rnd=1)
    b = O.rollout_costs_perturbed(p, ot, sc.X0[0], sc.U0[0], 1.0, sc.opp, sc.opp, np.zeros((1, 2)), sc.T, K=64,
                                  seed=2, rnd=1)
    for k in ("cost", "feasible", "violation", "margins"):
        np.testing.assert_array_equal(a[k], b[k])
