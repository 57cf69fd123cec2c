"""Seeded synthetic inputs for the SGTP best-response path.

This module generates *inputs only*: racelines, starting grids, parameter
presets and constant-velocity opponent predictions.  It holds none of the
planner's arithmetic (no sampling, rollout, projection, cost or selection) and
is shared by the CUDA path and the CPU oracle, which both receive the float32
arrays it returns.

The paper evaluates on MapZoo tracks with minimum-curvature racelines
(Sec. IV-B); neither is available here.  Synthetic tracks stand in:

* ``oval_track``: two 200 m straights joined by R = 50 m semicircles,
  width 10 m, 400 waypoints (the single best-response workload);
* ``fourier_track``: a closed curve r(theta) = 500 + sum_{m=2..9}
  A_m cos(m theta + phi_m), A_m ~ U(0, 5) m (so the modes sum to <= 40 m),
  resampled to 2000 waypoints at uniform arc length, one width W ~ U(10, 15) m
  per track split equally left/right.

The reference speed of a waypoint is v^r = min(v_cap, sqrt(a_lat / |kappa|))
(v_cap = 60 m/s, a_lat = 15 m/s^2), kappa being the discrete curvature of the
waypoint polygon; the heading is the direction of the central difference.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

F32 = np.float32


# --------------------------------------------------------------- parameters
def params_fullscale() -> dict:
    """Cost weights of Sec. IV-B (Q, R, S, w_game, w_* , mu_tail); distance
    thresholds scaled by 5 from the paper's 1/10-scale cars to full-size
    vehicles (s_contest 40, s_role 5, g_safe 5, d_col 4.5, m_bd 1.0 m);
    sampling spreads sigma_a = 1.0 m/s^2, sigma_delta = 0.05 rad; vehicle
    limits of a full-size car (wheelbase 3 m, a in [-12, 6], |delta| <= 0.35,
    v in [0, 90])."""
    return dict(
        dt=0.05, wheelbase=3.0, a_min=-12.0, a_max=6.0, delta_max=0.35, v_min=0.0, v_max=90.0,
        sigma_a=1.0, sigma_delta=0.05,
        Q=[60.0, 60.0, 47.75, 39.48], R=[8.43, 20.0], S=[1.0, 19.26],
        w_game=60.0, w_contest=1.0, w_long=2.0, w_block=10.0, w_safety=50.0,
        s_contest=40.0, s_role=5.0, mu_tail=0.3, g_safe=5.0, eps_alpha=1e-3, m_bd=1.0, d_col=4.5,
    )


# The paper's sample budget, horizon and IBR rounds (Sec. IV-B): K, H, L_IBR.
PAPER_SAMPLES = (128, 12, 2)


def params_paper() -> dict:
    """The paper's own 1/10-scale setup (Sec. IV-B): sampling spreads, cost
    weights, game weights and thresholds as printed, dt = 1.2 s / 12 steps.
    The vehicle limits (wheelbase, acceleration, steering and speed ranges)
    are not printed; these are our choice for a 1/10-scale car (wheelbase
    0.33 m, a in [-9.5, 9.5], |delta| <= 0.4189, v in [0, 7])."""
    return dict(
        dt=0.1, wheelbase=0.33, a_min=-9.5, a_max=9.5, delta_max=0.4189, v_min=0.0, v_max=7.0,
        sigma_a=0.335, sigma_delta=0.025,
        Q=[60.0, 60.0, 47.75, 39.48], R=[8.43, 20.0], S=[1.0, 19.26],
        w_game=60.0, w_contest=1.0, w_long=2.0, w_block=10.0, w_safety=50.0,
        s_contest=8.0, s_role=1.0, mu_tail=0.3, g_safe=1.0, eps_alpha=1e-3, m_bd=0.515, d_col=0.9,
    )


# --------------------------------------------------------------- tracks
@dataclass
class TrackData:
    xr: np.ndarray          # (N, 4) float32: x, y, psi, v^r
    wl: np.ndarray          # (N,) float32
    wr: np.ndarray          # (N,) float32
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def N(self):
        return self.xr.shape[0]


def _resample_closed(px, py, n):
    """Resample a dense closed polygon at n points of uniform arc length."""
    qx = np.append(px, px[0]); qy = np.append(py, py[0])
    seg = np.hypot(np.diff(qx), np.diff(qy))
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    s = np.arange(n) * (cum[-1] / n)
    return np.interp(s, cum, qx), np.interp(s, cum, qy)


def _headings_and_vref(x, y, v_cap, a_lat):
    n = x.shape[0]
    xn, yn = np.roll(x, -1), np.roll(y, -1)
    xp, yp = np.roll(x, 1), np.roll(y, 1)
    psi = np.arctan2(yn - yp, xn - xp)
    h_out = np.arctan2(yn - y, xn - x)          # heading of the segment leaving j
    h_in = np.arctan2(y - yp, x - xp)           # heading of the segment entering j
    turn = np.angle(np.exp(1j * (h_out - h_in)))
    ds = 0.5 * (np.hypot(xn - x, yn - y) + np.hypot(x - xp, y - yp))
    kappa = turn / ds
    k5 = np.zeros(n)
    for sh in range(-2, 3):                      # 5-point moving average
        k5 += np.roll(kappa, sh)
    k5 /= 5.0
    with np.errstate(divide="ignore"):
        v = np.minimum(v_cap, np.sqrt(a_lat / np.maximum(np.abs(k5), 1e-12)))
    return psi, v


def _pack(x, y, psi, v, wl, wr, name, meta):
    xr = np.stack([x, y, psi, v], axis=1).astype(F32)
    return TrackData(xr=np.ascontiguousarray(xr), wl=np.asarray(wl, dtype=F32), wr=np.asarray(wr, dtype=F32),
                     name=name, meta=meta)


def oval_track(n_points=400, straight=200.0, radius=50.0, width=10.0, v_cap=60.0, a_lat=15.0) -> TrackData:
    """Oval of two straights joined by semicircles, counter-clockwise, starting
    at the beginning of the lower straight (0, 0) heading +x."""
    L = 2 * straight + 2 * math.pi * radius
    s = np.arange(n_points) * (L / n_points)
    x = np.zeros(n_points); y = np.zeros(n_points)
    for i, si in enumerate(s):
        if si < straight:
            x[i], y[i] = si, 0.0
        elif si < straight + math.pi * radius:
            a = (si - straight) / radius
            x[i], y[i] = straight + radius * math.sin(a), radius - radius * math.cos(a)
        elif si < 2 * straight + math.pi * radius:
            x[i], y[i] = straight - (si - straight - math.pi * radius), 2 * radius
        else:
            a = (si - 2 * straight - math.pi * radius) / radius
            x[i], y[i] = -radius * math.sin(a), radius + radius * math.cos(a)
    psi, v = _headings_and_vref(x, y, v_cap, a_lat)
    w = np.full(n_points, width / 2)
    return _pack(x, y, psi, v, w, w, "oval", dict(length=L, straight=straight, radius=radius, width=width))


def fourier_track(seed: int, n_points=2000, r0=500.0, n_modes=8, amp_max=5.0, width_lo=10.0, width_hi=15.0,
                  v_cap=60.0, a_lat=15.0, dense=20000) -> TrackData:
    """Seeded closed track: circle of radius r0 perturbed by modes m=2..n_modes+1."""
    rng = np.random.default_rng(seed)
    amps = rng.uniform(0.0, amp_max, n_modes)
    phases = rng.uniform(0.0, 2 * math.pi, n_modes)
    width = rng.uniform(width_lo, width_hi)
    th = np.arange(dense) * (2 * math.pi / dense)
    r = np.full(dense, r0)
    for m, (A, ph) in enumerate(zip(amps, phases), start=2):
        r += A * np.cos(m * th + ph)
    x, y = _resample_closed(r * np.cos(th), r * np.sin(th), n_points)
    psi, v = _headings_and_vref(x, y, v_cap, a_lat)
    w = np.full(n_points, width / 2)
    return _pack(x, y, psi, v, w, w, f"fourier{seed}", dict(seed=seed, width=width, amps=amps, phases=phases))


# --------------------------------------------------------------- placing vehicles
def _arc(track: TrackData):
    P = track.xr[:, :2].astype(np.float64)
    Q = np.roll(P, -1, axis=0)
    seg = np.hypot(*(Q - P).T)
    return P, Q, seg, np.concatenate([[0.0], np.cumsum(seg)])


def pose_at(track: TrackData, s: float, d: float):
    """World pose (x, y, psi) at progress s (m) and lateral offset d (left +)."""
    P, Q, seg, cum = _arc(track)
    L = cum[-1]
    s = s % L
    j = int(np.searchsorted(cum, s, side="right") - 1)
    j = min(max(j, 0), track.N - 1)
    u = (s - cum[j]) / seg[j]
    t = (Q[j] - P[j]) / seg[j]
    c = P[j] + u * (Q[j] - P[j])
    nrm = np.array([-t[1], t[0]])
    p = c + d * nrm
    return float(p[0]), float(p[1]), float(math.atan2(t[1], t[0]))


def track_length(track: TrackData) -> float:
    return float(_arc(track)[3][-1])


def constant_velocity_prediction(x0, T, dt):
    """Opponent prediction that keeps heading and speed: the states of a
    vehicle moving on a straight line at constant speed (a simple prediction
    model, used as the fixed opponent trajectory of the single-response case)."""
    x0 = np.asarray(x0, dtype=np.float64)
    tau = np.arange(T + 1, dtype=np.float64)
    out = np.zeros((T + 1, 4))
    out[:, 0] = x0[0] + tau * dt * x0[3] * math.cos(x0[2])
    out[:, 1] = x0[1] + tau * dt * x0[3] * math.sin(x0[2])
    out[:, 2] = x0[2]
    out[:, 3] = x0[3]
    return out.astype(F32)


# --------------------------------------------------------------- workloads
@dataclass
class Scenario:
    track: TrackData
    X0: np.ndarray            # (n_v, 4) float32
    U0: np.ndarray            # (n_v, T, 2) float32 (zeros: Sec. II, nominal reset)
    vref_scale: np.ndarray    # (n_v,) float32: 1 for the ego, 0.9 for opponents (Sec. IV-B)
    ego: int
    T: int
    K: int
    L: int
    opp: np.ndarray | None = None   # fixed opponent predictions (single-response case)
    name: str = ""


def single_br_oval(K=1024, T=40) -> Scenario:
    """Oval, ego at the start of a straight (d = 0, v = 20 m/s), one opponent
    10 m ahead at d = +2 m, v = 18 m/s, whose fixed prediction keeps speed and
    heading."""
    tr = oval_track()
    dt = params_fullscale()["dt"]
    ex, ey, ep = pose_at(tr, 0.0, 0.0)
    ox, oy, op = pose_at(tr, 10.0, 2.0)
    X0 = np.array([[ex, ey, ep, 20.0], [ox, oy, op, 18.0]], dtype=F32)
    opp = constant_velocity_prediction(X0[1], T, dt)[None]
    return Scenario(track=tr, X0=X0, U0=np.zeros((2, T, 2), F32), vref_scale=np.array([1.0, 0.9], F32), ego=0,
                    T=T, K=K, L=1, opp=opp, name="oval-1v1")


def grid_race(track: TrackData, n_v: int, T: int, K: int, L: int, seed: int, s0=None, row_gap=8.0,
              d_side=2.5, v_lo=40.0, v_hi=60.0) -> Scenario:
    """Starting grid two wide, rows row_gap apart, d = +/- d_side, speeds
    U(v_lo, v_hi), headings along the raceline; the ego is the rearmost car
    (Sec. IV-B places the ego last)."""
    rng = np.random.default_rng(seed)
    if s0 is None:
        s0 = float(rng.uniform(0.0, track_length(track)))
    X0 = np.zeros((n_v, 4), F32)
    for i in range(n_v):
        row, col = divmod(i, 2)
        x, y, psi = pose_at(track, s0 + row * row_gap, d_side if col == 0 else -d_side)
        X0[i] = (x, y, psi, rng.uniform(v_lo, v_hi))
    vs = np.full(n_v, 0.9, F32)
    vs[0] = 1.0
    return Scenario(track=track, X0=X0, U0=np.zeros((n_v, T, 2), F32), vref_scale=vs, ego=0, T=T, K=K, L=L,
                    name=f"{track.name}-grid{n_v}")


def trial_race(track: TrackData, n_v: int, T: int, K: int, L: int, seed: int, s0: float, gap_lo=8.0, gap_hi=20.0,
               v_lo=40.0, v_hi=55.0) -> Scenario:
    """One closed-loop trial (Sec. IV-B): the ego (vehicle 0) starts behind
    every opponent; opponent j starts gap_lo..gap_hi m ahead of the previous
    car, d ~ U(-3, 3) m; speeds U(v_lo, v_hi); headings along the raceline;
    reference speed scale 1 for the ego and 0.9 for the opponents."""
    rng = np.random.default_rng(seed)
    X0 = np.zeros((n_v, 4), F32)
    s = s0
    for i in range(n_v):
        if i > 0:
            s += float(rng.uniform(gap_lo, gap_hi))
        x, y, psi = pose_at(track, s, float(rng.uniform(-3.0, 3.0)) if i > 0 else 0.0)
        X0[i] = (x, y, psi, rng.uniform(v_lo, v_hi))
    vs = np.full(n_v, 0.9, F32)
    vs[0] = 1.0
    return Scenario(track=track, X0=X0, U0=np.zeros((n_v, T, 2), F32), vref_scale=vs, ego=0, T=T, K=K, L=L,
                    name=f"{track.name}-trial{n_v}")


def trial_set(n_tracks=7, starts=6, n_v=3, T=60, K=4096, L=2, seed0=400):
    """n_tracks seeded Fourier tracks x `starts` evenly spaced starting points
    (the paper's 7 tracks x 6 starts; its MapZoo tracks are replaced by
    synthetic ones)."""
    out = []
    for t in range(n_tracks):
        tr = fourier_track(seed0 + t)
        Lt = track_length(tr)
        for k in range(starts):
            out.append(trial_race(tr, n_v, T, K, L, seed0 * 100 + t * starts + k, s0=k * Lt / starts))
    return out


def two_car_race(seed: int, K=8192, T=50, L=3) -> Scenario:
    """Two cars 5-15 m apart on a seeded Fourier track, d ~ U(-2, 2),
    v ~ U(40, 60); the rear car is the ego."""
    tr = fourier_track(seed)
    rng = np.random.default_rng(seed + 7)
    s0 = float(rng.uniform(0.0, track_length(tr)))
    gap = float(rng.uniform(5.0, 15.0))
    X0 = np.zeros((2, 4), F32)
    for i, s in enumerate((s0, s0 + gap)):
        x, y, psi = pose_at(tr, s, float(rng.uniform(-2.0, 2.0)))
        X0[i] = (x, y, psi, rng.uniform(40.0, 60.0))
    return Scenario(track=tr, X0=X0, U0=np.zeros((2, T, 2), F32), vref_scale=np.array([1.0, 0.9], F32), ego=0,
                    T=T, K=K, L=L, name=f"fourier{seed}-2car")


def ten_car_race(seed: int, K=16384, T=60, L=5) -> Scenario:
    """Ten cars on a 2-wide grid with 8 m rows on a seeded Fourier track."""
    return grid_race(fourier_track(seed), 10, T, K, L, seed + 11)


def batched_races(n_races=256, K=4096, L=3, seed0=1000, n_points=2000):
    """Independent races with per-race seeds seed0+r: n_v ~ U{2..10},
    T ~ U{30..80}, each on its own Fourier track."""
    out = []
    for r in range(n_races):
        rng = np.random.default_rng(seed0 + r)
        n_v = int(rng.integers(2, 11))
        T = int(rng.integers(30, 81))
        tr = fourier_track(seed0 + r, n_points=n_points)
        out.append(grid_race(tr, n_v, T, K, L, seed0 + r + 50000))
    return out
