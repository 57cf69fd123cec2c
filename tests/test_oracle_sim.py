"""Pins of the closed-loop trial oracle (oracle/sim.py) against closed forms
and hand-counted cases (the racing scenarios of Sec. IV-B, the metrics of Sec. IV-C)."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import sim as OS
from paper_2607_25388_b300 import scenario as S

SP = dict(n_apply=5, max_steps=1000, tracker=0, pp_preview=5, contact_dist=4.5, wall_margin=0.0, close_ds=5.0,
          close_dd=2.5)


def _oval():
    td = S.oval_track()
    return td, O.Track(td.xr, td.wl, td.wr)


def _on_straight(s, d, v):
    """State on the oval's lower straight (y = 0, heading +x): s along x, d = y."""
    return np.array([s, d, 0.0, v])


def test_constant_speed_on_a_straight_gains_v_dt_per_step():
    td, ot = _oval()
    p = S.params_fullscale()
    X = np.stack([_on_straight(20.0, 0.5, 20.0)])
    U = np.zeros((1, 10, 2))
    st = OS.reset(ot, X, 0)
    X1, U1, st = OS.step(p, ot, SP, X, U, None, 0, st)
    dt = float(np.float32(p["dt"]))
    assert st["steps"] == 5 and st["alive"] == 1 and st["ego_collision"] == 0
    assert st["progress"][0] == pytest.approx(5 * 20.0 * dt, abs=1e-9)
    assert st["d"][0] == pytest.approx(0.5, abs=1e-9)
    assert X1[0, 0] == pytest.approx(20.0 + 5 * 20.0 * dt, abs=1e-9)
    assert st["ego_speed_sum"] == pytest.approx(5 * 20.0)
    assert st["ego_du2_sum"] == 0.0


def test_vehicle_contact_ends_the_trial():
    td, ot = _oval()
    p = S.params_fullscale()
    X = np.stack([_on_straight(20.0, -1.5, 30.0), _on_straight(22.0, 1.5, 30.0)])      # 3.6 m apart
    st = OS.reset(ot, X, 0)
    _, _, st = OS.step(p, ot, SP, X, np.zeros((2, 10, 2)), None, 0, st)
    assert st["ego_collision"] == 1 and st["alive"] == 0 and st["steps"] == 1
    X = np.stack([_on_straight(20.0, -1.5, 30.0), _on_straight(30.0, 1.5, 30.0)])      # 10.4 m apart
    st = OS.reset(ot, X, 0)
    _, _, st = OS.step(p, ot, SP, X, np.zeros((2, 10, 2)), None, 0, st)
    assert st["ego_collision"] == 0 and st["alive"] == 1 and st["steps"] == 5


def test_wall_contact_when_the_reference_point_leaves_the_track():
    td, ot = _oval()
    p = S.params_fullscale()
    w = float(td.wl[0])
    # heading outward at 0.2 rad: the lateral offset grows by v dt sin(0.2) per step
    X = np.array([[50.0, w - 0.5, 0.2, 20.0]])
    st = OS.reset(ot, X, 0)
    _, _, st = OS.step(p, ot, dict(SP, n_apply=10), X, np.zeros((1, 10, 2)), None, 0, st)
    dy = 20.0 * float(np.float32(p["dt"])) * math.sin(0.2)
    first = math.floor(0.5 / dy) + 1            # first step with d > w
    assert st["ego_collision"] == 2 and st["steps"] == first


def test_close_interaction_segments_are_counted():
    td, ot = _oval()
    p = S.params_fullscale()
    # alongside, 4.4 m ahead and 2.2 m across (4.92 m apart: no contact), same speed: close every step
    X = np.stack([_on_straight(30.0, -1.1, 25.0), _on_straight(34.4, 1.1, 25.0)])
    st = OS.reset(ot, X, 0)
    _, _, st = OS.step(p, ot, dict(SP, n_apply=6, max_steps=6), X, np.zeros((2, 10, 2)), None, 0, st)
    assert st["alive"] == 0 and st["close_segments"] == 1 and st["close_steps"] == 6
    # 2.6 m across: never close
    X = np.stack([_on_straight(30.0, -1.3, 25.0), _on_straight(34.4, 1.3, 25.0)])
    st = OS.reset(ot, X, 0)
    _, _, st = OS.step(p, ot, dict(SP, n_apply=6, max_steps=6), X, np.zeros((2, 10, 2)), None, 0, st)
    assert st["close_segments"] == 0 and st["close_steps"] == 0
    # the ego 4.45 m ahead and 2 m/s faster: 0.1 m more per step, close for 5 steps, then apart
    X = np.stack([_on_straight(34.45, -1.1, 27.0), _on_straight(30.0, 1.1, 25.0)])
    st = OS.reset(ot, X, 0)
    _, _, st = OS.step(p, ot, dict(SP, n_apply=8, max_steps=100), X, np.zeros((2, 10, 2)), None, 0, st)
    assert st["close_segments"] == 1 and st["close_steps"] == 5 and st["close_run"][1] == 0


def test_warm_start_shifts_by_the_steps_applied():
    td, ot = _oval()
    p = S.params_fullscale()
    X = np.stack([_on_straight(20.0, 0.0, 20.0)])
    U = np.arange(20, dtype=np.float64).reshape(1, 10, 2) * 0.01
    st = OS.reset(ot, X, 0)
    _, U1, st = OS.step(p, ot, dict(SP, n_apply=4), X, U, None, 0, st)
    want = np.concatenate([U[0, 4:], np.repeat(U[0, 9:], 4, axis=0)])
    np.testing.assert_array_equal(U1[0], want)
    # control smoothness: three differences of (0.02, 0.02) after the first applied control
    assert st["ego_du2_sum"] == pytest.approx(3 * 2 * 0.02 ** 2)


def test_pure_pursuit_on_a_circle_steers_with_curvature_one_over_r():
    """A target on the circle of radius R tangent to the heading at the
    vehicle: alpha = theta/2, l_d = 2R sin(theta/2), so the pure-pursuit
    curvature 2 sin(alpha)/l_d is exactly 1/R."""
    p = S.params_fullscale()
    for R, theta in ((80.0, 0.3), (200.0, 0.1), (-60.0, 0.4)):
        tgt = np.array([abs(R) * math.sin(theta), R * (1 - math.cos(theta)), 0.0, 30.0])
        plan = np.stack([np.array([0.0, 0.0, 0.0, 30.0])] + [tgt] * 6)
        u = OS.pure_pursuit(p, plan, 0, 5, np.array([0.0, 0.0, 0.0, 30.0]))
        assert u[1] == pytest.approx(math.atan(float(np.float32(p["wheelbase"])) / R), rel=1e-12)
        assert u[0] == 0.0


def test_pure_pursuit_tracks_the_planned_speed():
    p = S.params_fullscale()
    plan = np.array([[0.0, 0.0, 0.0, 30.0], [1.5, 0.0, 0.0, 30.2], [3.0, 0.0, 0.0, 30.4]] + [[4.5, 0.0, 0.0, 31]] * 4)
    u = OS.pure_pursuit(p, plan, 0, 2, np.array([0.0, 0.0, 0.0, 30.0]))
    assert u[1] == 0.0
    assert u[0] == pytest.approx(0.2 / float(np.float32(p["dt"])), rel=1e-6)
    u = OS.pure_pursuit(p, plan, 0, 2, np.array([0.0, 0.0, 0.0, 50.0]))      # far above: full braking
    assert u[0] == float(np.float32(p["a_min"]))
