"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test checks the oracle against what the paper or mathematics fixes:
an independent library implementation (Philox), closed-form rollouts of the
bicycle model, exact geometric values on straight track, hand-worked cost
examples of the game terms (Sec. III-A), exact threshold behaviour of the
feasibility checks (Sec. III-B), brute-force ranking, and the bookkeeping of
Alg. 1.  No GPU is used.
"""
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as O
from paper_2607_25388_b300 import scenario as S

F32 = np.float32


def f32(x):
    return float(np.float32(x))


# ---------------------------------------------------------------- fixtures
def stadium(straight=1000.0, radius=100.0, spacing=2.0, width=10.0, vref=20.0, roll=0):
    """Closed track with long straights whose waypoints sit on exact float32
    coordinates; the lower straight runs from (0, 0) along +x.  roll shifts
    the first waypoint (and so the start line) along the list."""
    pts, heads = [], []
    n_s = int(straight / spacing)
    for i in range(n_s):
        pts.append((i * spacing, 0.0)); heads.append(0.0)
    n_a = 157
    for i in range(n_a):
        a = math.pi * i / n_a
        pts.append((straight + radius * math.sin(a), radius - radius * math.cos(a))); heads.append(a)
    for i in range(n_s):
        pts.append((straight - i * spacing, 2 * radius)); heads.append(math.pi)
    for i in range(n_a):
        a = math.pi * i / n_a
        pts.append((-radius * math.sin(a), radius + radius * math.cos(a)))
        heads.append(math.atan2(math.sin(math.pi + a), math.cos(math.pi + a)))
    xr = np.zeros((len(pts), 4), F32)
    xr[:, :2] = np.array(pts, dtype=F32)
    xr[:, 2] = np.array(heads, dtype=F32)
    xr[:, 3] = vref
    xr = np.roll(xr, -roll, axis=0)
    w = np.full(len(pts), width / 2, F32)
    return O.Track(xr, w, w)


def params(**over):
    p = S.params_fullscale()
    p.update(over)
    return p


# ---------------------------------------------------------------- Philox
TORCH_PHILOX_SRC = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdlib>
int main(int argc, char **argv) {
  unsigned c0, c1, c2, c3, k0, k1;
  while (scanf("%u %u %u %u %u %u", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
    at::philox_engine e(((unsigned long long)k1 << 32) | k0, ((unsigned long long)c3 << 32) | c2,
                        ((unsigned long long)c1 << 32) | c0);
    unsigned a = e(), b = e(), c = e(), d = e();
    printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


def test_philox_matches_torch_engine():
    """The oracle's Philox4x32-10 equals PyTorch's independent header-only
    implementation of the same published generator on 300 random
    counter/key pairs (counter = offset lo/hi, subsequence lo/hi)."""
    import torch
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    rng = np.random.default_rng(5)
    rows = rng.integers(0, 2**32, size=(300, 6), dtype=np.uint64)
    rows[:4] = [[0, 0, 0, 0, 0, 0], [1, 0, 0, 0, 0, 0], [0, 0, 0, 0, 2**32 - 1, 2**32 - 1],
                [2**32 - 1] * 6]
    with tempfile.TemporaryDirectory() as td:
        src = os.path.join(td, "p.cpp"); exe = os.path.join(td, "p")
        open(src, "w").write(TORCH_PHILOX_SRC)
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-I", inc, src, "-o", exe])
        inp = "\n".join(" ".join(str(int(v)) for v in r) for r in rows) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for r, line in zip(rows, out):
        want = [int(v) for v in line.split()]
        got = O.philox([r[0], r[1], r[2], r[3]], [r[4], r[5]])
        assert got == want, (r, got, want)


def test_normals_are_standard_gaussian():
    """Box-Muller draws: mean 0, variance 1, kurtosis 3, uncorrelated pair,
    and a Kolmogorov-Smirnov test against N(0, 1)."""
    from scipy import stats
    z = O.std_normals_batch(seed=1234, race=3, agent=2, rnd=1, stream=0, k0=0, nk=2000, T=64).reshape(-1, 2)
    n = z.shape[0]
    for c in range(2):
        x = z[:, c]
        assert abs(x.mean()) < 5 / math.sqrt(n)
        assert abs(x.var() - 1) < 5 * math.sqrt(2 / n)
        assert abs(stats.kurtosis(x, fisher=False) - 3) < 0.05
        assert stats.kstest(x, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 5 / math.sqrt(n)
    # consecutive steps (the two halves of one Philox block) are uncorrelated
    zz = O.std_normals_batch(7, 0, 0, 0, 0, 0, 4000, 2)
    assert abs(np.corrcoef(zz[:, 0, 0], zz[:, 1, 0])[0, 1]) < 5 / math.sqrt(4000)


def test_noise_streams_differ_by_every_counter_field():
    base = O.std_normals(9, 1, 2, 3, 0, 4, 5)
    for args in [(10, 1, 2, 3, 0, 4, 5), (9, 0, 2, 3, 0, 4, 5), (9, 1, 3, 3, 0, 4, 5), (9, 1, 2, 4, 0, 4, 5),
                 (9, 1, 2, 3, 1, 4, 5), (9, 1, 2, 3, 0, 5, 5), (9, 1, 2, 3, 0, 4, 4), (9, 1, 2, 3, 0, 4, 7)]:
        assert O.std_normals(*args) != base


# ---------------------------------------------------------------- Frenet
def test_frenet_exact_on_straights():
    tr = stadium()
    L = O.track_length(tr)
    assert L == pytest.approx(2000 + 2 * math.pi * 100, abs=0.2)
    xs = np.array([10.0, 123.25, 500.5, 987.0])
    ds = np.array([0.0, 2.5, -4.0, 3.75])
    s, d, _ = O.frenet(tr, np.stack([xs, ds], 1))
    np.testing.assert_array_equal(s, xs)
    np.testing.assert_array_equal(d, ds)
    # upper straight runs along -x: left of travel is -y
    s2, d2, _ = O.frenet(tr, np.stack([xs, 200.0 - ds], 1))
    s_top = O.frenet(tr, np.array([[1000.0 - 2.0 * 0, 200.0]]))[0][0]
    np.testing.assert_allclose(s2, s_top + (1000.0 - xs), atol=1e-9)
    np.testing.assert_allclose(d2, ds, atol=1e-12)


def test_frenet_matches_vectorised_brute_force():
    """Global-nearest projection cross-checked against an independent
    vectorised point-to-segment computation on a seeded Fourier track."""
    td = S.fourier_track(101, n_points=300)
    tr = O.Track(td.xr, td.wl, td.wr)
    rng = np.random.default_rng(0)
    P = td.xr[:, :2].astype(np.float64)
    Q = np.roll(P, -1, 0)
    E = Q - P
    cum = np.concatenate([[0], np.cumsum(np.hypot(*E.T))])
    idx = rng.integers(0, td.N, 400)
    pts = P[idx] + rng.normal(0, 6.0, (400, 2))
    s, d, seg = O.frenet(tr, pts)
    for i, p in enumerate(pts):
        u = np.clip(((p - P) * E).sum(1) / (E * E).sum(1), 0, 1)
        C = P + u[:, None] * E
        dist = np.hypot(*(p - C).T)
        j = int(np.argmin(dist))
        assert seg[i] == j
        assert s[i] == pytest.approx(cum[j] + u[j] * (cum[j + 1] - cum[j]), abs=1e-9)
        sign = 1.0 if E[j, 0] * (p[1] - P[j, 1]) - E[j, 1] * (p[0] - P[j, 0]) >= 0 else -1.0
        assert d[i] == pytest.approx(sign * dist[j], abs=1e-9)


def test_progress_unwraps_across_the_start_line():
    tr = stadium(roll=250)               # the lap starts at (500, 0), mid-straight
    L = O.track_length(tr)
    p = params(sigma_a=0.0, sigma_delta=0.0)
    x0 = np.array([498.5, 0.0, 0.0, 20.0])
    sd0 = O.frenet(tr, x0[None, :2])[0][0]
    assert sd0 == pytest.approx(L - 1.5, abs=1e-9)
    out = O.rollout_costs(p, tr, x0, np.zeros((10, 2)), 1.0, None, 10, K=1, zero_noise=True, want_frenet=True)
    s = out["frenet"][0, :, 0]
    step = 20.0 * f32(p["dt"])
    np.testing.assert_allclose(np.diff(s), step, rtol=0, atol=1e-9)
    assert s[-1] == pytest.approx(sd0 + 10 * step, abs=1e-9) and s[-1] > L


# ---------------------------------------------------------------- dynamics
def test_zero_noise_samples_equal_the_nominal_rollout():
    sc = S.single_br_oval(K=32, T=20)
    tr = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    p = params(sigma_a=0.0, sigma_delta=0.0)
    rng = np.random.default_rng(1)
    u = np.stack([rng.uniform(-20, 10, 20), rng.uniform(-0.5, 0.5, 20)], 1).astype(F32)  # exceeds limits
    out = O.rollout_costs(p, tr, sc.X0[0], u, 1.0, sc.opp, 20, K=32, seed=3, want_states=True)
    uc = np.stack([np.clip(u[:, 0], -12, 6), np.clip(u[:, 1], -f32(0.35), f32(0.35))], 1)
    nominal = O.rollout(p, sc.X0[0], uc, 20)
    for k in range(32):
        np.testing.assert_array_equal(out["states"][k], nominal)
    assert np.all(out["cost"] == out["cost"][0])
    br = O.best_response(p, tr, sc.X0[0], u, 1.0, sc.opp, 20, 32, seed=3)
    assert br["k_star"] == 0


def test_constant_speed_and_constant_acceleration_closed_forms():
    p = params()
    dt = f32(p["dt"])
    T = 30
    x0 = np.array([100.0, 0.0, 0.0, 20.0])
    st = O.rollout(p, x0, np.zeros((T, 2)), T)
    n = np.arange(T + 1)
    np.testing.assert_allclose(st[:, 0], 100.0 + n * dt * 20.0, rtol=0, atol=1e-10)
    np.testing.assert_array_equal(st[:, 1:3], 0.0)
    a = 2.0
    st = O.rollout(p, x0, np.tile([a, 0.0], (T, 1)), T)
    np.testing.assert_allclose(st[:, 3], 20.0 + n * a * dt, atol=1e-10)
    np.testing.assert_allclose(st[:, 0], 100.0 + dt * (n * 20.0 + a * dt * n * (n - 1) / 2), atol=1e-9)
    # speed clamps at v_max and v_min
    st = O.rollout(p, np.array([0, 0, 0, 89.0]), np.tile([6.0, 0.0], (T, 1)), T)
    assert st[:, 3].max() == f32(90.0)
    st = O.rollout(p, np.array([0, 0, 0, 1.0]), np.tile([-12.0, 0.0], (T, 1)), T)
    assert st[-1, 3] == 0.0 and st[:, 0].max() == pytest.approx(dt * 1.0 + dt * (1.0 - 12.0 * dt), abs=1e-12)


def test_constant_steer_traces_a_circle():
    p = params()
    dt, Lwb = f32(p["dt"]), f32(p["wheelbase"])
    v, delta, T = 20.0, 0.1, 40
    st = O.rollout(p, np.array([0.0, 0.0, 0.3, v]), np.tile([0.0, delta], (T, 1)), T)
    dpsi = dt * v * math.tan(delta) / Lwb
    np.testing.assert_allclose(np.diff(st[:, 2]), dpsi, atol=1e-12)
    chords = np.hypot(np.diff(st[:, 0]), np.diff(st[:, 1]))
    np.testing.assert_allclose(chords, dt * v, atol=1e-12)
    # all points on one circle of radius chord / (2 sin(dpsi/2))
    rho = dt * v / (2 * math.sin(dpsi / 2))
    a, b, c = st[0, :2], st[1, :2], st[2, :2]
    A = np.array([[b[0] - a[0], b[1] - a[1]], [c[0] - a[0], c[1] - a[1]]])
    rhs = 0.5 * np.array([b @ b - a @ a, c @ c - a @ a])
    ctr = np.linalg.solve(A, rhs)
    np.testing.assert_allclose(np.hypot(*(st[:, :2] - ctr).T), rho, rtol=1e-9)


# ---------------------------------------------------------------- tracking cost
def test_tracking_cost_vanishes_on_the_reference():
    tr = stadium(vref=20.0)
    p = params()
    T = 20
    x0 = np.array([100.0, 0.0, 0.0, 20.0])
    ref = O.reference(p, tr, x0, 1.0, T)
    np.testing.assert_allclose(ref[1:, 0], 100.0 + np.arange(1, T + 1) * f32(p["dt"]) * 20.0, atol=1e-9)
    np.testing.assert_allclose(ref[1:, 1:], np.tile([0.0, 0.0, 20.0], (T, 1)), atol=1e-12)
    out = O.eval_controls(p, tr, x0, np.zeros((T, 2)), 1.0, None, T, game_on=True)
    assert abs(out["cost"][0]) < 1e-12
    assert out["feasible"][0] == 1 and out["violation"][0] == 0.0


def test_tracking_cost_closed_forms_for_each_state_weight():
    p = params()
    Q = [f32(q) for q in p["Q"]]
    dt = f32(p["dt"])
    T = 20
    tr = stadium(vref=20.0)
    # lateral offset of 1 m: e_y = 1 at every step
    c = O.eval_controls(p, tr, np.array([100.0, 1.0, 0.0, 20.0]), np.zeros((T, 2)), 1.0, None, T)["cost"][0]
    assert c == pytest.approx(T * Q[1], rel=1e-12)
    # 1 m/s too fast: e_v = 1 and e_x = tau*dt
    c = O.eval_controls(p, tr, np.array([100.0, 0.0, 0.0, 21.0]), np.zeros((T, 2)), 1.0, None, T)["cost"][0]
    tau = np.arange(1, T + 1)
    assert c == pytest.approx(Q[3] * T + Q[0] * np.sum((tau * dt) ** 2), rel=1e-9)
    # reference speed scale 0.9 (Sec. IV-B): reference advances at 18 m/s
    c = O.eval_controls(p, tr, np.array([100.0, 0.0, 0.0, 18.0]), np.zeros((T, 2)), 0.9, None, T)["cost"][0]
    assert abs(c) < 1e-9
    # standing still on a zero-speed raceline: only the heading error counts, wrapped to (-pi, pi]
    tr0 = stadium(vref=0.0)
    for psi0, e in [(0.5, 0.5), (0.5 + 2 * math.pi, 0.5), (-3.0, -3.0), (3.5, 3.5 - 2 * math.pi)]:
        c = O.eval_controls(p, tr0, np.array([100.0, 0.0, psi0, 0.0]), np.zeros((T, 2)), 1.0, None, T)["cost"][0]
        assert c == pytest.approx(T * Q[2] * e * e, rel=1e-9)


def test_control_and_smoothness_cost_closed_forms():
    p = params(Q=[0, 0, 0, 0])
    R = [f32(r) for r in p["R"]]; Sw = [f32(s) for s in p["S"]]
    T = 16
    tr = stadium()
    x0 = np.array([100.0, 0.0, 0.0, 20.0])
    U = np.tile([0.5, 0.02], (T, 1))
    c = O.eval_controls(p, tr, x0, U, 1.0, None, T)["cost"][0]
    assert c == pytest.approx(T * (R[0] * 0.25 + R[1] * 0.02 ** 2), rel=1e-12)
    U = np.zeros((T, 2)); U[:, 0] = 0.5 * (-1.0) ** np.arange(T)
    c = O.eval_controls(p, tr, x0, U, 1.0, None, T)["cost"][0]
    assert c == pytest.approx(T * R[0] * 0.25 + (T - 1) * Sw[0] * 1.0, rel=1e-12)


# ---------------------------------------------------------------- feasibility
def test_boundary_check_is_inclusive_at_the_margin():
    """rho_bd >= m_bd passes (Eq. selection-boundary); exact values on the
    straight where w = 5 m and m_bd = 1 m."""
    p = params()
    tr = stadium()
    T = 5
    for y, feas, viol in [(4.0, 1, 0.0), (-4.0, 1, 0.0), (4.0 + 2 ** -10, 0, 2 ** -10), (-4.5, 0, 0.5),
                          (0.0, 1, 0.0)]:
        out = O.eval_controls(p, tr, np.array([300.0, y, 0.0, 0.0]), np.zeros((T, 2)), 1.0, None, T)
        assert out["feasible"][0] == feas, y
        assert out["violation"][0] == pytest.approx(viol, abs=1e-15)


def test_boundary_uses_min_over_steps_one_to_H():
    """A car drifting left: clearance at step tau is 5 - d_tau; the minimum
    over tau = 1..H decides, and tau = 0 is not checked."""
    p = params()
    tr = stadium()
    T = 10
    # start outside the margin (d0 = 4.5) but heading back to the centre
    psi = -0.2
    out = O.eval_controls(p, tr, np.array([300.0, 4.5, psi, 10.0]), np.zeros((T, 2)), 1.0, None, T,
                          want_states=True)
    d = out["frenet"][0, 1:, 1]
    assert out["violation"][0] == pytest.approx(max(0.0, 1.0 - (5.0 - d.max())), abs=1e-12)


def test_collision_check_and_game_terms_worked_example():
    """Ego stationary 4.5 m behind a stationary opponent on the straight:
    g_min = 4.5 = d_col passes (Eq. selection-vehicle); the game cost is
    contest -1, longitudinal -2*alpha*(-4.5), no block (gap < s_role... ego
    behind), safety 50*(5-4.5)^2 (Eqs. c_contest, c_long, c_block, c_safety)."""
    p = params(Q=[0, 0, 0, 0])
    tr = stadium()
    T = 6
    x0 = np.array([100.0, 0.0, 0.0, 0.0])
    opp = np.tile([104.5, 0.0, 0.0, 0.0], (T + 1, 1))[None]
    out = O.eval_controls(p, tr, x0, np.zeros((T, 2)), 1.0, opp, T, game_on=True)
    alpha = 1.0 / (1.0 + 4.5 / (40.0 + f32(1e-3)))
    c_game = -1.0 - 2.0 * alpha * (-4.5) + 50.0 * 0.5 ** 2
    assert out["cost"][0] == pytest.approx(60.0 * c_game, rel=1e-12)
    assert out["feasible"][0] == 1
    out0 = O.eval_controls(p, tr, x0, np.zeros((T, 2)), 1.0, opp, T, game_on=False)
    assert out0["cost"][0] == 0.0
    opp2 = np.tile([104.375, 0.0, 0.0, 0.0], (T + 1, 1))[None]
    out2 = O.eval_controls(p, tr, x0, np.zeros((T, 2)), 1.0, opp2, T, game_on=True)
    assert out2["feasible"][0] == 0 and out2["violation"][0] == pytest.approx(0.125, abs=1e-15)
    # only tau = 1..H counts: an overlap at tau = 0 alone is feasible
    opp3 = np.tile([200.0, 0.0, 0.0, 0.0], (T + 1, 1))[None]; opp3[0, 0, 0] = 100.0
    assert O.eval_controls(p, tr, x0, np.zeros((T, 2)), 1.0, opp3, T)["feasible"][0] == 1


def test_blocking_gate_on_and_off():
    """Ego ahead by s_role + 0.5 = 5.5 m activates gamma = w_block; ahead by
    4.5 m does not (Eq. c_block, strict inequalities)."""
    p = params(Q=[0, 0, 0, 0])
    tr = stadium()
    T = 10
    sc = f32(40.0) + f32(1e-3)
    for gap, on in [(5.5, True), (4.5, False)]:
        x0 = np.array([100.0 + gap, 1.0, 0.0, 0.0])
        opp = np.tile([100.0, -1.0, 0.0, 0.0], (T + 1, 1))[None]
        c = O.eval_controls(p, tr, x0, np.zeros((T, 2)), 1.0, opp, T, game_on=True)["cost"][0]
        alpha = 1.0 / (1.0 + gap / sc)
        g = math.hypot(gap, 2.0)
        want = -1.0 - 2.0 * alpha * gap - (10.0 / (1.0 + 2.0) if on else 0.0) + 50.0 * max(0.0, 5.0 - g) ** 2
        assert c == pytest.approx(60.0 * want, rel=1e-12), gap
    # outside the contest window: no contest reward, no block
    x0 = np.array([160.0, 1.0, 0.0, 0.0])
    opp = np.tile([100.0, -1.0, 0.0, 0.0], (T + 1, 1))[None]
    c = O.eval_controls(p, tr, x0, np.zeros((T, 2)), 1.0, opp, T, game_on=True)["cost"][0]
    assert c == pytest.approx(60.0 * (-2.0 * 60.0 / (1.0 + 60.0 / sc)), rel=1e-12)


def test_tail_count():
    assert O.tail_count(0.3, 60) == 18
    assert O.tail_count(0.3, 12) == 4
    assert O.tail_count(0.3, 1) == 1
    assert O.tail_count(0.001, 50) == 1
    assert O.tail_count(1.0, 7) == 7


def test_tail_mean_of_lateral_offset():
    """A car at constant d: d_bar_i = d; an opponent whose prediction only
    changes d inside the tail shows the tail mean (blocking term)."""
    p = params(Q=[0, 0, 0, 0])
    tr = stadium()
    T = 10                             # n_tail = ceil(3) = 3 -> steps 8, 9, 10
    x0 = np.array([105.5, 1.0, 0.0, 0.0])
    opp = np.tile([100.0, -1.0, 0.0, 0.0], (T + 1, 1))
    opp[8:, 1] = [-2.0, -3.0, -4.0]    # tail mean -3
    opp[:8, 1] = 7.0                   # outside the tail: ignored
    c = O.eval_controls(p, tr, x0, np.zeros((T, 2)), 1.0, opp[None], T, game_on=True)["cost"][0]
    sc = f32(40.0) + f32(1e-3)
    alpha = 1.0 / (1.0 + 5.5 / sc)
    g = min(math.hypot(5.5, 1.0 - y) for y in opp[1:, 1])
    want = -1.0 - 2.0 * alpha * 5.5 - 10.0 / (1.0 + 4.0) + 50.0 * max(0.0, 5.0 - g) ** 2
    assert c == pytest.approx(60.0 * want, rel=1e-12)


# ---------------------------------------------------------------- selection
def test_selection_against_brute_force_sort():
    rng = np.random.default_rng(2)
    for trial in range(300):
        n = int(rng.integers(1, 17))
        cost = rng.choice([-1.0, 0.0, 1.5, 2.0, np.nan, np.inf], n) if trial % 3 == 0 else rng.normal(0, 1, n)
        feas = rng.integers(0, 2, n).astype(np.uint8) if trial % 4 else np.zeros(n, np.uint8)
        viol = rng.choice([0.5, 0.25, np.nan, 1.0], n)
        k, anyf = O.select(cost, feas, viol)
        key = [((0 if feas[i] else 1), (cost[i] if feas[i] else viol[i]), i) for i in range(n)]
        key = [(a, (math.inf if math.isnan(b) else b), i) for a, b, i in key]
        want = sorted(key)[0][2]
        assert k == want and anyf == bool(feas.any())


def test_best_response_is_the_brute_force_minimum():
    sc = S.single_br_oval(K=64, T=24)
    tr = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    p = S.params_fullscale()
    out = O.rollout_costs(p, tr, sc.X0[0], sc.U0[0], 1.0, sc.opp[:, :25], 24, K=64, seed=11, rnd=1,
                          want_states=True, want_controls=True)
    br = O.best_response(p, tr, sc.X0[0], sc.U0[0], 1.0, sc.opp[:, :25], 24, 64, seed=11, rnd=1)
    order = sorted(range(64), key=lambda i: (0 if out["feasible"][i] else 1,
                                             out["cost"][i] if out["feasible"][i] else out["violation"][i], i))
    assert br["k_star"] == order[0]
    np.testing.assert_array_equal(br["xi_star"], out["states"][order[0]])
    np.testing.assert_array_equal(br["u_star"], out["controls"][order[0]])


def test_fallback_picks_least_violation_when_nothing_is_feasible():
    """Start 4.9 m left of centre on a 5 m half-width: every candidate
    violates the boundary margin; the least violation wins (Sec. III-B)."""
    p = params(sigma_delta=0.1)
    tr = stadium()
    T = 8
    x0 = np.array([300.0, 4.9, 0.0, 20.0])
    out = O.rollout_costs(p, tr, x0, np.zeros((T, 2)), 1.0, None, T, K=48, seed=5)
    assert not out["feasible"].any()
    br = O.best_response(p, tr, x0, np.zeros((T, 2)), 1.0, None, T, 48, seed=5)
    assert br["any_feasible"] is False
    assert br["k_star"] == int(np.argmin(out["violation"]))


# ---------------------------------------------------------------- Alg. 1
def test_ibr_plan_follows_algorithm_1():
    """Round 0 answers the others' nominal rollouts without the game term;
    each later round answers the previous round (Jacobi); the ego answers
    once more at the end; nominal controls are warm-started."""
    sc = S.two_car_race(100, K=48, T=16, L=2)
    tr = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    p = S.params_fullscale()
    T, K, L = sc.T, sc.K, sc.L
    plan = O.ibr_plan(p, tr, sc.X0, sc.U0, sc.vref_scale, T, K, L, sc.ego, seed=21, race=4, want_hist=True)
    n_v = 2
    U = sc.U0.astype(np.float64).copy()
    xi = np.stack([O.rollout(p, sc.X0[i], np.clip(U[i], [-12, -f32(0.35)], [6, f32(0.35)]), T)
                   for i in range(n_v)])
    ks = []
    for rnd in range(L + 1):
        new = []
        for i in range(n_v):
            br = O.best_response(p, tr, sc.X0[i], U[i], sc.vref_scale[i], xi[1 - i][None], T, K, seed=21, race=4,
                                 agent=i, rnd=rnd, game_on=rnd > 0)
            ks.append(br["k_star"]); new.append(br)
        for i in range(n_v):
            xi[i] = new[i]["xi_star"]; U[i] = new[i]["u_star"]
        np.testing.assert_array_equal(plan["xi_hist"][rnd], xi)
        np.testing.assert_array_equal(plan["u_hist"][rnd], U)
    br = O.best_response(p, tr, sc.X0[0], U[0], 1.0, xi[1][None], T, K, seed=21, race=4, agent=0, rnd=L + 1)
    ks.append(br["k_star"])
    xi[0] = br["xi_star"]; U[0] = br["u_star"]
    assert list(plan["k_star"]) == ks
    np.testing.assert_array_equal(plan["xi"], xi)
    np.testing.assert_array_equal(plan["u_nom"], U)
