"""FP64 oracle of one closed-loop trial step (the receding-horizon
racing scenarios of Sec. IV-B and the Evaluation Metrics of Sec. IV-C).

TEST INFRASTRUCTURE ONLY: imported by the test-suite alone.  It shares no
code with the CUDA path; the dynamics and the Frenet projection are the
oracle's own (``rollout``: Sec. II bicycle model, ``frenet``: global nearest
point of the raceline), everything else is written out here in double
precision.  Parameters are rounded to float32 first, as the library
receives them.

Readings (the paper races in a simulator with a cited vehicle model and a
cited pure-pursuit tracker and gives no parameters for either):
* plant: the planner's kinematic bicycle;
* tracker 0 applies the plan's controls U[i, m]; tracker 1 is pure pursuit
  toward the planned position ``pp_preview`` steps after substep m:
  delta = clip(atan(2 wheelbase sin(alpha) / l_d)), alpha the target's
  bearing relative to the heading, l_d its distance, and
  a = clip((v_plan[m+1] - v) / dt);
* all vehicles step together; after each step every vehicle is projected,
  unwrapped progress advances by the half-lap-wrapped change of s;
* the ego is in contact with an opponent when their reference points are
  closer than contact_dist, else with a wall when min(w^R(s) + d,
  w^L(s) - d) < wall_margin (widths linear in s between waypoints); a trial
  ends at its first contact or at max_steps;
* close interaction with opponent j: |wrap(s_e - s_j)| < close_ds and
  |d_e - d_j| < close_dd; runs are counted as segments when they end
  (or when the trial ends);
* the ego's control smoothness sums ||u_k - u_{k-1}||^2 over applied
  controls after its first; its speed is summed after every step;
* the warm start shifts by the steps applied, the last control repeated.
"""
from __future__ import annotations

import copy
import math

import numpy as np

from . import Track, frenet, rollout


def _f32(v):
    return float(np.float32(v))


def _wrap(x, L):
    return x - L * math.ceil(x / L - 0.5)


def _arc(track: Track):
    P = track.xr[:, :2]
    Q = np.roll(P, -1, axis=0)
    seg = np.hypot(Q[:, 0] - P[:, 0], Q[:, 1] - P[:, 1])
    return np.concatenate([[0.0], np.cumsum(seg)]), seg


def project(track: Track, x: float, y: float):
    """(s, d, w^L(s), w^R(s)) at the globally nearest point."""
    s, d, seg = frenet(track, [[x, y]])
    j = int(seg[0])
    cum, ln = _arc(track)
    t = (s[0] - cum[j]) / ln[j]
    jn = (j + 1) % track.N
    wl = track.wl[j] + t * (track.wl[jn] - track.wl[j])
    wr = track.wr[j] + t * (track.wr[jn] - track.wr[j])
    return float(s[0]), float(d[0]), float(wl), float(wr)


def track_len(track: Track) -> float:
    return float(_arc(track)[0][-1])


def reset(track: Track, X, ego: int) -> dict:
    X = np.asarray(X, np.float64)
    n = X.shape[0]
    L = track_len(track)
    pr = [project(track, X[i, 0], X[i, 1]) for i in range(n)]
    s = np.array([p[0] for p in pr])
    return dict(alive=1, steps=0, ego_collision=0, close_segments=0, close_steps=0, ego_speed_sum=0.0,
                ego_du2_sum=0.0, progress=np.zeros(n), rel0=np.array([_wrap(s[i] - s[ego], L) for i in range(n)]),
                d=np.array([p[1] for p in pr]), s_raw=s, close_run=np.zeros(n, dtype=np.int64), u_prev=np.zeros(2))


def pure_pursuit(params: dict, plan, m: int, preview: int, x):
    """Controls of the tracker toward plan[(m + preview)] ((T+1) x 4 states)."""
    plan = np.asarray(plan, np.float64)
    T = plan.shape[0] - 1
    tgt = plan[min(m + preview, T)]
    dx, dy = tgt[0] - x[0], tgt[1] - x[1]
    ld = math.hypot(dx, dy)
    delta = 0.0
    if ld > 1e-6:
        alpha = math.atan2(dy, dx) - x[2]
        delta = math.atan(2.0 * _f32(params["wheelbase"]) * math.sin(alpha) / ld)
    dm = _f32(params["delta_max"])
    delta = min(max(delta, -dm), dm)
    vp = plan[min(m + 1, T), 3]
    acc = min(max((vp - x[3]) / _f32(params["dt"]), _f32(params["a_min"])), _f32(params["a_max"]))
    return np.array([acc, delta])


def step(params: dict, track: Track, sp: dict, X, U, xi, ego: int, state: dict, margins=None):
    """One sgtp_sim_step of one trial: returns (X', U', state').  X (n, 4),
    U (n, T, 2), xi (n, T+1, 4) as float64 copies of the device values.
    margins (a list, optional) receives, per substep, the smallest distance
    of any decision argument to its threshold: (contact, wall, close-box
    longitudinal, close-box lateral)."""
    X = np.array(X, np.float64)
    U = np.array(U, np.float64)
    st = copy.deepcopy(state)
    if not st["alive"]:
        return X, U, st
    n, T = U.shape[0], U.shape[1]
    L = track_len(track)
    contact = _f32(sp["contact_dist"])
    wall = _f32(sp["wall_margin"])
    cds, cdd = _f32(sp["close_ds"]), _f32(sp["close_dd"])
    applied = 0
    for m in range(int(sp["n_apply"])):
        if not st["alive"]:
            break
        for i in range(n):
            u = pure_pursuit(params, xi[i], m, int(sp["pp_preview"]), X[i]) if sp["tracker"] == 1 else U[i, m].copy()
            if i == ego:
                if st["steps"] > 0:
                    st["ego_du2_sum"] += float(np.sum((u - st["u_prev"]) ** 2))
                st["u_prev"] = u.copy()
            X[i] = rollout(params, X[i], u[None, :], 1)[1]
            if i == ego:
                st["ego_speed_sum"] += X[i, 3]
        pr = [project(track, X[i, 0], X[i, 1]) for i in range(n)]
        for i in range(n):
            st["progress"][i] += _wrap(pr[i][0] - st["s_raw"][i], L)
            st["s_raw"][i] = pr[i][0]
            st["d"][i] = pr[i][1]
        st["steps"] += 1
        coll = 0
        mg = [math.inf] * 4
        for j in range(n):
            if j == ego:
                continue
            dist = math.hypot(X[j, 0] - X[ego, 0], X[j, 1] - X[ego, 1])
            mg[0] = min(mg[0], abs(dist - contact))
            if dist < contact:
                coll = 1
        _, de, wl, wr = pr[ego]
        mg[1] = abs(min(wr + de, wl - de) - wall)
        if not coll and min(wr + de, wl - de) < wall:
            coll = 2
        for j in range(n):
            if j == ego:
                continue
            ds = _wrap(pr[ego][0] - pr[j][0], L)
            dd = pr[ego][1] - pr[j][1]
            mg[2] = min(mg[2], abs(abs(ds) - cds))
            mg[3] = min(mg[3], abs(abs(dd) - cdd))
            if abs(ds) < cds and abs(dd) < cdd:
                st["close_run"][j] += 1
            elif st["close_run"][j] > 0:
                st["close_segments"] += 1
                st["close_steps"] += int(st["close_run"][j])
                st["close_run"][j] = 0
        if coll or st["steps"] >= int(sp["max_steps"]):
            if coll:
                st["ego_collision"] = coll
            st["alive"] = 0
            for j in range(n):
                if st["close_run"][j] > 0:
                    st["close_segments"] += 1
                    st["close_steps"] += int(st["close_run"][j])
                    st["close_run"][j] = 0
        if margins is not None:
            margins.append(mg)
        applied = m + 1
    Un = U.copy()
    for tau in range(T):
        Un[:, tau] = U[:, tau + applied] if tau + applied < T else U[:, T - 1]
    return X, Un, st
