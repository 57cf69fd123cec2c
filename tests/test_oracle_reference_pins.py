"""Pins of the oracle's reference trajectory and raceline interpolation.

Sec. III-A (overall ranking) defines the reference as s^r_0 = s_{i,t},
s^r_{tau+1} = s^r_tau + dt v^r(s^r_tau), x^r_tau = x^r(s^r_tau), and Sec. II
makes the raceline maps continuous in s (linear between waypoints, the
heading along the shorter arc).  These tests fix the oracle's reading
against values that follow from those definitions alone:

* on a straight whose reference speed rises linearly in s, the recursion
  is affine, s_{tau+1} = (1 + b dt) s_tau + a dt, with the geometric closed
  form s_tau = (s_0 + a/b)(1 + b dt)^tau - a/b; evaluating v^r at s^r_{tau+1}
  instead (an implicit step) misses it by decimetres within 40 steps;
* a ten-waypoint speed step between two constant stretches, iterated from a
  piecewise-linear v^r(s) written down from the track's construction;
* headings that straddle the +-pi seam interpolate along the short arc; a
  plain linear blend would pass through 0 instead;
* the reference keeps going straight through the track's start line.
"""
import math

import numpy as np

import oracle as O
from paper_2607_25388_b300 import scenario as S

F32 = np.float32


def f32(x):
    return float(np.float32(x))


def wrap_pi(a):
    return (np.asarray(a) + math.pi) % (2 * math.pi) - math.pi


def straight_loop(v_of_x, heading_of_i=None, straight=1000.0, radius=100.0, spacing=2.0, roll=0):
    """Stadium loop: lower straight from (0, 0) along +x with reference speed
    v_of_x(x) at its waypoints (exact float32 values), a semicircle, the
    return straight at y = 2 radius heading pi (or heading_of_i(i) at its
    i-th waypoint), and a closing semicircle at 20 m/s."""
    pts, heads, vs = [], [], []
    n_s = int(straight / spacing)
    for i in range(n_s):
        x = i * spacing
        pts.append((x, 0.0)); heads.append(0.0); vs.append(v_of_x(x))
    n_a = 157
    for i in range(n_a):
        a = math.pi * i / n_a
        pts.append((straight + radius * math.sin(a), radius - radius * math.cos(a))); heads.append(a); vs.append(20.0)
    for i in range(n_s):
        pts.append((straight - i * spacing, 2 * radius))
        heads.append(heading_of_i(i) if heading_of_i else math.pi)
        vs.append(20.0)
    for i in range(n_a):
        a = math.pi * i / n_a
        pts.append((-radius * math.sin(a), radius + radius * math.cos(a)))
        heads.append(math.atan2(math.sin(math.pi + a), math.cos(math.pi + a)))
        vs.append(20.0)
    xr = np.zeros((len(pts), 4), F32)
    xr[:, :2] = np.array(pts, dtype=F32)
    xr[:, 2] = np.array(heads, dtype=F32)
    xr[:, 3] = np.array(vs, dtype=F32)
    xr = np.roll(xr, -roll, axis=0)
    w = np.full(len(pts), 5.0, F32)
    return O.Track(xr, w, w)


def ramp_speed(x):
    """20 m/s up to x = 100, then +0.25 m/s per 2 m waypoint up to 30 m/s at
    x = 180 (every value exact in float32), then 30 m/s."""
    if x < 100.0:
        return 20.0
    if x > 180.0:
        return 30.0
    return 20.0 + 0.125 * (x - 100.0)


def test_reference_on_a_linear_speed_ramp_follows_the_geometric_closed_form():
    p = S.params_fullscale()
    dt = f32(p["dt"])
    tr = straight_loop(ramp_speed)
    T = 40
    for scale in (1.0, f32(0.9)):
        # inside the ramp v^r(s) = a + b s with a = 7.5, b = 0.125 (s = x on the lower straight)
        a, b = 7.5 * scale, 0.125 * scale
        s0 = 102.0
        ref = O.reference(p, tr, np.array([s0, 0.0, 0.0, 20.0]), scale, T)
        tau = np.arange(T + 1)
        s = (s0 + a / b) * (1.0 + b * dt) ** tau - a / b
        assert s[-1] < 180.0                                   # stays on the ramp
        np.testing.assert_allclose(ref[1:, 0], s[1:], rtol=0, atol=1e-9)
        np.testing.assert_allclose(ref[1:, 1], 0.0, atol=1e-12)
        np.testing.assert_allclose(ref[1:, 2], 0.0, atol=1e-12)
        # row tau carries the scaled reference speed at s^r_tau
        np.testing.assert_allclose(ref[1:, 3], a + b * s[1:], rtol=0, atol=1e-9)
        # the implicit reading (v^r at s^r_{tau+1}) is far from the oracle
        s_impl = (s0 + a / b) / (1.0 - b * dt) ** tau - a / b
        assert np.abs(s_impl[-1] - ref[-1, 0]) > 0.05


def test_reference_across_a_ten_waypoint_speed_step():
    """v^r steps from 20 to 30 m/s over ten waypoints (x = 100..120); the
    reference starts 20 m before the step and ends on the 30 m/s stretch."""
    p = S.params_fullscale()
    dt = f32(p["dt"])

    def step_speed(x):
        return 20.0 if x < 100.0 else 30.0 if x > 120.0 else 20.0 + 0.5 * (x - 100.0)

    tr = straight_loop(step_speed)
    T = 60
    ref = O.reference(p, tr, np.array([80.0, 0.0, 0.0, 20.0]), 1.0, T)
    s = [80.0]
    for _ in range(T):
        s.append(s[-1] + dt * step_speed(s[-1]))
    s = np.array(s)
    assert s[-1] > 130.0                                      # crossed the whole step
    np.testing.assert_allclose(ref[1:, 0], s[1:], rtol=0, atol=1e-9)
    np.testing.assert_allclose(ref[1:, 3], [step_speed(x) for x in s[1:]], rtol=0, atol=1e-9)


def test_heading_interpolates_along_the_short_arc_across_the_seam():
    """Return-straight headings alternate between pi - 0.02 and -(pi - 0.02):
    consecutive waypoints are 0.04 rad apart across the +-pi seam."""
    p = S.params_fullscale()
    dt = f32(p["dt"])
    h_even, h_odd = f32(math.pi - 0.02), f32(-(math.pi - 0.02))
    tr = straight_loop(lambda x: 20.0, heading_of_i=lambda i: h_even if i % 2 == 0 else h_odd)
    T = 40
    # ego 100 m into the return straight (x = 900, y = 200), heading pi
    ref = O.reference(p, tr, np.array([900.0, 200.0, math.pi, 20.0]), 1.0, T)
    tau = np.arange(1, T + 1)
    along = 100.0 + tau * dt * 20.0                           # metres past the straight's first waypoint
    i = np.floor(along / 2.0).astype(int)
    u = along / 2.0 - i
    h0 = np.where(i % 2 == 0, h_even, h_odd)
    short = wrap_pi(np.where(i % 2 == 0, h_odd, h_even) - h0)  # +-0.04: the short arc
    expect = h0 + u * short
    assert np.all(np.abs(short) < 0.05)
    np.testing.assert_allclose(wrap_pi(ref[1:, 2] - expect), 0.0, atol=1e-9)
    assert np.all(np.abs(wrap_pi(ref[1:, 2] - math.pi)) <= 0.0201)
    np.testing.assert_allclose(ref[1:, 0], 1000.0 - along, atol=1e-9)
    np.testing.assert_allclose(ref[1:, 1], 200.0, atol=1e-12)


def test_reference_runs_straight_through_the_start_line():
    """The start line (s = 0) in the middle of the lower straight: the
    reference's positions continue linearly across it."""
    p = S.params_fullscale()
    dt = f32(p["dt"])
    tr = straight_loop(lambda x: 20.0, roll=250)              # first waypoint at x = 500
    T = 40
    x0 = 490.0
    ref = O.reference(p, tr, np.array([x0, 0.0, 0.0, 20.0]), 1.0, T)
    tau = np.arange(1, T + 1)
    np.testing.assert_allclose(ref[1:, 0], x0 + tau * dt * 20.0, atol=1e-9)
    np.testing.assert_allclose(ref[1:, 3], 20.0, atol=1e-12)
