"""FP64 oracle of the learned proposal's input features (not part of the
SGTP paper).

TEST INFRASTRUCTURE ONLY: imported by the test-suite alone.

Features of vehicle i before one of its best responses, all from the Frenet
frame of Sec. II (global-nearest projection, brute force):

  0     d_i / 5
  1, 2  sin e, cos e with e = wrap(psi_i - psi_ref(s_i)), psi_ref the
        raceline heading interpolated along the nearest segment
  3     v_i / 60
  4..7  100 kappa at s_i + {0, 20, 40, 80} m, kappa of a segment = its
        wrapped heading increment over its length
  8 + 6q .. 13 + 6q for the q-th nearest opponent (q = 0..8), opponents
        ordered by (floor(1000 |Delta s|), index), Delta s = wrap(s_j - s_i):
        [1, Delta s / 40, d_j / 5, (v_j - v_i) / 10, wrap(psi_j - psi_i),
         (g_j - v_i T dt) / 40], g_j the progress gain s_H - s_0 of opponent
        j's predicted trajectory; zeros for absent slots
  62    n_opp / 9
  63    1 if the best response uses the game term, else 0

Parity status: pinned -- closed forms on the oval track (straights and
semicircles of known radius) in the oracle's own tests.
"""
from __future__ import annotations

import math

import numpy as np

from . import Track, frenet


def _wrap(x, L):
    return x - L * math.ceil(x / L - 0.5)


def _wrap_pi(a):
    return a - 2.0 * math.pi * math.ceil(a / (2.0 * math.pi) - 0.5)


def arc_lengths(track: Track):
    """Cumulative arc length s_j of every waypoint and the lap length L."""
    xy = track.xr[:, :2]
    seg = np.roll(xy, -1, axis=0) - xy
    lens = np.sqrt((seg ** 2).sum(axis=1))
    s = np.concatenate([[0.0], np.cumsum(lens)])
    return s, float(s[-1]), lens


def progress_gain(track: Track, states):
    """s_H - s_0 of a state trajectory ((H+1) x 4), the progress unwrapped
    step by step."""
    st = np.asarray(states, dtype=np.float64).reshape(-1, 4)
    s, _, _ = frenet(track, st[:, :2])
    _, L, _ = arc_lengths(track)
    acc = s[0]
    for t in range(1, st.shape[0]):
        acc = acc + _wrap(s[t] - acc, L)
    return acc - s[0]


def features(track: Track, X, gains, i, T, dt, game_on):
    """The 64 features of vehicle i; X (n_v x 4) the states at the start of
    the plan, gains (n_v) each vehicle's predicted progress gain."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 4)
    n_v = X.shape[0]
    s_all, d_all, seg_all = frenet(track, X[:, :2])
    sj, L, lens = arc_lengths(track)
    xr = track.xr
    N = track.N
    f = np.zeros(64)
    s_i, d_i, j0 = s_all[i], d_all[i], int(seg_all[i])
    u = (s_i - sj[j0]) / lens[j0]
    psi_ref = xr[j0, 2] + u * _wrap_pi(xr[(j0 + 1) % N, 2] - xr[j0, 2])
    e = _wrap_pi(X[i, 2] - psi_ref)
    f[0] = d_i / 5.0
    f[1] = math.sin(e)
    f[2] = math.cos(e)
    f[3] = X[i, 3] / 60.0
    for q, ahead in enumerate((0.0, 20.0, 40.0, 80.0)):
        sm = math.fmod(s_i + ahead, L)
        j = int(np.searchsorted(sj, sm, side="right")) - 1
        j = min(max(j, 0), N - 1)
        f[4 + q] = 100.0 * _wrap_pi(xr[(j + 1) % N, 2] - xr[j, 2]) / lens[j]
    others = [j for j in range(n_v) if j != i]
    others.sort(key=lambda j: (math.floor(abs(_wrap(s_all[j] - s_i, L)) * 1000.0), j))
    for q, j in enumerate(others[:9]):
        o = 8 + 6 * q
        f[o:o + 6] = [1.0, _wrap(s_all[j] - s_i, L) / 40.0, d_all[j] / 5.0, (X[j, 3] - X[i, 3]) / 10.0,
                      _wrap_pi(X[j, 2] - X[i, 2]), (gains[j] - X[i, 3] * T * dt) / 40.0]
    f[62] = len(others) / 9.0
    f[63] = 1.0 if game_on else 0.0
    return f


def order_keys(track: Track, X, i):
    """The sort keys 1000 |Delta s| (before flooring) of every opponent of i,
    for recognising near-ties in parity checks."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 4)
    s_all, _, _ = frenet(track, X[:, :2])
    _, L, _ = arc_lengths(track)
    return {j: abs(_wrap(s_all[j] - s_all[i], L)) * 1000.0 for j in range(X.shape[0]) if j != i}
