"""FP64 CPU oracle of the SGTP best-response hot path.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The
product library never calls it and shares no code with it.

The arithmetic lives in ``sgtp_oracle.c`` (plain C, double precision); this
module compiles it with gcc on first use and marshals numpy arrays through
ctypes.  Every entry point mirrors a step of the paper:

* :func:`philox`             Philox4x32-10 counter-based generator (Salmon et al., SC'11)
* :func:`std_normals`        Box-Muller noise of sample k, step tau (Sec. II)
* :func:`frenet`             global-nearest Frenet projection s, d (Sec. II)
* :func:`rollout_costs`      per-candidate cost (Eq. allc), flags (Eq. selection), violation
* :func:`best_response`      one best response with selection and fallback (Sec. III-B)
* :func:`ibr_plan`           the SGTP planning call (Alg. 1)
* :func:`best_response_mppi` GA-IBR-MPPI best response: path-integral update (Sec. IV-A ablation)
* :func:`ibr_plan_mppi`      the GA-IBR-MPPI planning call
* :func:`perturb_prediction` a perturbed opponent prediction (Table II robustness study)
* :func:`ibr_plan_perturbed` the SGTP planning call with perturbed predictions

Parity status of each function is listed in the header of ``sgtp_oracle.c``'s
tests (``tests/test_oracle_*.py``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgtp_oracle.c")
_LIB = os.path.join(_HERE, "libsgtp_oracle.so")
_lock = threading.Lock()
_lib = None

PARAM_FIELDS = [
    "dt", "wheelbase", "a_min", "a_max", "delta_max", "v_min", "v_max", "sigma_a", "sigma_delta",
    "Q", "R", "S", "w_game", "w_contest", "w_long", "w_block", "w_safety",
    "s_contest", "s_role", "mu_tail", "g_safe", "eps_alpha", "m_bd", "d_col",
]


class OrcParams(C.Structure):
    _fields_ = [
        ("dt", C.c_double), ("wheelbase", C.c_double),
        ("a_min", C.c_double), ("a_max", C.c_double), ("delta_max", C.c_double),
        ("v_min", C.c_double), ("v_max", C.c_double),
        ("sigma_a", C.c_double), ("sigma_delta", C.c_double),
        ("Q", C.c_double * 4), ("R", C.c_double * 2), ("S", C.c_double * 2),
        ("w_game", C.c_double), ("w_contest", C.c_double), ("w_long", C.c_double),
        ("w_block", C.c_double), ("w_safety", C.c_double),
        ("s_contest", C.c_double), ("s_role", C.c_double), ("mu_tail", C.c_double),
        ("g_safe", C.c_double), ("eps_alpha", C.c_double), ("m_bd", C.c_double), ("d_col", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                                   "-ffp-contract=off", _SRC, "-o", tmp, "-lm", "-lpthread"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.orc_std_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                      C.c_int, dp, dp]
        L.orc_tail_count.argtypes = [C.c_double, C.c_int]
        L.orc_tail_count.restype = C.c_int
        L.orc_frenet.argtypes = [dp, dp, dp, C.c_int, dp, C.c_int, dp, dp, C.POINTER(C.c_int32)]
        L.orc_track_length.argtypes = [dp, C.c_int]
        L.orc_track_length.restype = C.c_double
        L.orc_rollout_costs.argtypes = [
            C.POINTER(OrcParams), dp, dp, dp, C.c_int, dp, dp, C.c_double, dp, C.c_int, C.c_int,
            C.POINTER(C.c_int32), C.c_int, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int,
            C.c_int, dp, C.POINTER(C.c_ubyte), dp, dp, dp, dp, dp, dp, dp, dp, C.c_int, C.c_int]
        L.orc_eval_controls.argtypes = [
            C.POINTER(OrcParams), dp, dp, dp, C.c_int, dp, dp, C.c_int, C.c_double, dp, C.c_int, C.c_int,
            C.c_int, dp, C.POINTER(C.c_ubyte), dp, dp, dp]
        L.orc_best_response.argtypes = [
            C.POINTER(OrcParams), dp, dp, dp, C.c_int, dp, dp, C.c_double, dp, C.c_int, C.c_int, C.c_int,
            C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, C.POINTER(C.c_int), dp, dp,
            C.POINTER(C.c_int), dp, C.c_int]
        L.orc_best_response_mixed.argtypes = [
            C.POINTER(OrcParams), dp, dp, dp, C.c_int, dp, dp, C.c_double, dp, C.c_int, C.c_int, C.c_int,
            C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, dp, C.c_int, C.POINTER(C.c_int),
            dp, dp, C.POINTER(C.c_int), dp, dp, C.c_int]
        L.orc_select.argtypes = [dp, C.POINTER(C.c_ubyte), dp, C.c_int, C.POINTER(C.c_int)]
        L.orc_select.restype = C.c_int
        L.orc_ibr_plan.argtypes = [
            C.POINTER(OrcParams), dp, dp, dp, C.c_int, C.c_int, dp, dp, dp, C.c_int, C.c_int, C.c_int,
            C.c_int, C.c_uint64, C.c_uint32, dp, C.POINTER(C.c_int), dp, dp, C.c_int]
        L.orc_best_response_mppi.argtypes = [
            C.POINTER(OrcParams), dp, dp, dp, C.c_int, dp, dp, C.c_double, dp, C.c_int, C.c_int, C.c_int,
            C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, C.c_double, C.POINTER(C.c_int), dp, dp, dp,
            C.c_int]
        L.orc_ibr_plan_mppi.argtypes = [
            C.POINTER(OrcParams), dp, dp, dp, C.c_int, C.c_int, dp, dp, dp, C.c_int, C.c_int, C.c_int,
            C.c_int, C.c_uint64, C.c_uint32, C.c_double, dp, C.POINTER(C.c_int), dp, dp, C.c_int]
        L.orc_perturb_prediction.argtypes = [dp, dp, dp, C.c_int, dp, C.c_int, C.c_uint64, C.c_uint32, C.c_uint32,
                                             C.c_uint32, C.c_uint32, C.c_double, C.c_double, C.c_int, dp, dp]
        L.orc_rollout_costs_perturbed.argtypes = [
            C.POINTER(OrcParams), dp, dp, dp, C.c_int, dp, dp, C.c_double, dp, dp, dp, C.c_int, C.c_int,
            C.POINTER(C.c_int32), C.c_int, C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, dp,
            C.POINTER(C.c_ubyte), dp, dp, dp, dp, C.c_int]
        L.orc_ibr_plan_perturbed.argtypes = [
            C.POINTER(OrcParams), dp, dp, dp, C.c_int, C.c_int, dp, dp, dp, C.c_int, C.c_int, C.c_int,
            C.c_int, C.c_uint64, C.c_uint32, C.c_double, C.c_double, dp, C.POINTER(C.c_int), dp, dp, C.c_int]
        L.orc_reference.argtypes = [C.POINTER(OrcParams), dp, dp, dp, C.c_int, dp, C.c_double, C.c_int, dp]
        L.orc_rollout.argtypes = [C.POINTER(OrcParams), dp, dp, C.c_int, dp]
        L.orc_philox_batch.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, C.c_uint32,
                                       C.c_uint32, C.POINTER(C.c_uint32)]
        L.orc_std_normals_batch.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                            C.c_uint32, C.c_int, C.c_int, dp]
        _lib = L
    return _lib


# ---------------------------------------------------------------- helpers
def _d(a):
    """Contiguous float64 copy (inputs are the float32 values the GPU sees)."""
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(params: dict) -> OrcParams:
    """Params dict -> struct; each value is first rounded to float32, exactly
    as the GPU receives it, then widened to double."""
    P = OrcParams()
    for f in PARAM_FIELDS:
        v = params[f]
        if f in ("Q", "R", "S"):
            arr = getattr(P, f)
            for i, x in enumerate(v):
                arr[i] = float(np.float32(x))
        else:
            setattr(P, f, float(np.float32(v)))
    return P


def _nthreads(n):
    return int(n) if n else max(1, os.cpu_count() or 1)


class Track:
    """Raceline arrays as doubles: xr (N,4) = x, y, psi, v^r; wl, wr (N,)."""

    def __init__(self, xr, wl, wr):
        self.xr = _d(xr).reshape(-1, 4)
        self.wl = _d(wl).reshape(-1)
        self.wr = _d(wr).reshape(-1)
        self.N = self.xr.shape[0]

    def args(self):
        return _p(self.xr), _p(self.wl), _p(self.wr), self.N


# ---------------------------------------------------------------- API
def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def philox_batch(c1, c2, c3, k0, n, seed):
    """Philox4x32-10 blocks of counters (k0 + i, c1, c2, c3), i < n, key = seed
    split into 32-bit halves: (n, 4) uint32."""
    out = np.zeros((n, 4), dtype=np.uint32)
    lib().orc_philox_batch(c1, c2, c3, k0, n, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF,
                           out.ctypes.data_as(C.POINTER(C.c_uint32)))
    return out


def std_normals(seed, race, agent, rnd, stream, k, tau):
    za, zd = C.c_double(), C.c_double()
    lib().orc_std_normals(seed, race, agent, rnd, stream, k, tau, C.byref(za), C.byref(zd))
    return za.value, zd.value


def std_normals_batch(seed, race, agent, rnd, stream, k0, nk, T):
    out = np.zeros((nk, T, 2))
    lib().orc_std_normals_batch(seed, race, agent, rnd, stream, k0, nk, T, _p(out))
    return out


def tail_count(mu_tail, H):
    return lib().orc_tail_count(float(np.float32(mu_tail)), int(H))


def track_length(track: Track):
    return lib().orc_track_length(_p(track.xr), track.N)


def frenet(track: Track, pts):
    pts = _d(pts).reshape(-1, 2)
    n = pts.shape[0]
    s = np.zeros(n); d = np.zeros(n); seg = np.zeros(n, dtype=np.int32)
    rc = lib().orc_frenet(*track.args(), _p(pts), n, _p(s), _p(d), seg.ctypes.data_as(C.POINTER(C.c_int32)))
    assert rc == 0
    return s, d, seg


def reference(params, track: Track, x0, vref_scale, T):
    out = np.zeros((T + 1, 4))
    rc = lib().orc_reference(C.byref(make_params(params)), *track.args(), _p(_d(x0)), float(np.float32(vref_scale)),
                             T, _p(out))
    assert rc == 0
    return out


def rollout(params, x0, u, T):
    st = np.zeros((T + 1, 4))
    lib().orc_rollout(C.byref(make_params(params)), _p(_d(x0)), _p(_d(u)), T, _p(st))
    return st


def rollout_costs(params, track: Track, x0, u_nom, vref_scale, opp, T, K=None, k_list=None, seed=0, race=0,
                  agent=0, rnd=0, stream=0, game_on=True, zero_noise=False, want_states=False,
                  want_frenet=False, want_controls=False, nthreads=None, prop=None, K_prop=0):
    """Per-candidate outputs for k in k_list (or 0..K-1); prop / K_prop as
    in :func:`best_response`."""
    opp = _d(opp).reshape(-1, T + 1, 4) if opp is not None and np.size(opp) else np.zeros((0, T + 1, 4))
    n_opp = opp.shape[0]
    if k_list is not None:
        kl = np.ascontiguousarray(np.asarray(k_list, dtype=np.int32))
        n = kl.shape[0]
        klp = kl.ctypes.data_as(C.POINTER(C.c_int32))
    else:
        n = int(K)
        klp = None
    cost = np.zeros(n); viol = np.zeros(n); feas = np.zeros(n, dtype=np.uint8)
    ctr = np.zeros(n); cg = np.zeros(n); mg = np.zeros((n, 3))
    states = np.zeros((n, T + 1, 4)) if want_states else None
    fr = np.zeros((n, T + 1, 2)) if want_frenet else None
    ctl = np.zeros((n, T, 2)) if want_controls else None
    pr = _d(prop).reshape(T, 4) if prop is not None else None
    rc = lib().orc_rollout_costs(
        C.byref(make_params(params)), *track.args(), _p(_d(x0)), _p(_d(u_nom)), float(np.float32(vref_scale)),
        _p(opp) if n_opp else None, n_opp, T, klp, n, seed, race, agent, rnd, stream, int(bool(game_on)),
        int(bool(zero_noise)), _p(cost), feas.ctypes.data_as(C.POINTER(C.c_ubyte)), _p(viol), _p(states),
        _p(fr), _p(ctl), _p(ctr), _p(cg), _p(mg), _p(pr), int(K_prop) if pr is not None else 0,
        _nthreads(nthreads))
    assert rc == 0
    out = dict(cost=cost, feasible=feas, violation=viol, c_track=ctr, c_game=cg, margins=mg)
    if want_states:
        out["states"] = states
    if want_frenet:
        out["frenet"] = fr
    if want_controls:
        out["controls"] = ctl
    return out


def eval_controls(params, track: Track, x0, U, vref_scale, opp, T, game_on=True, want_states=False):
    U = _d(U).reshape(-1, T, 2)
    n = U.shape[0]
    opp = _d(opp).reshape(-1, T + 1, 4) if opp is not None and np.size(opp) else np.zeros((0, T + 1, 4))
    cost = np.zeros(n); viol = np.zeros(n); feas = np.zeros(n, dtype=np.uint8)
    states = np.zeros((n, T + 1, 4)) if want_states else None
    fr = np.zeros((n, T + 1, 2)) if want_states else None
    rc = lib().orc_eval_controls(C.byref(make_params(params)), *track.args(), _p(_d(x0)), _p(U), n,
                                 float(np.float32(vref_scale)), _p(opp) if opp.shape[0] else None, opp.shape[0], T,
                                 int(bool(game_on)), _p(cost), feas.ctypes.data_as(C.POINTER(C.c_ubyte)), _p(viol),
                                 _p(states), _p(fr))
    assert rc == 0
    out = dict(cost=cost, feasible=feas, violation=viol)
    if want_states:
        out["states"] = states
        out["frenet"] = fr
    return out


def select(cost, feas, viol):
    cost = _d(cost); viol = _d(viol); feas = np.ascontiguousarray(np.asarray(feas, dtype=np.uint8))
    anyf = C.c_int()
    k = lib().orc_select(_p(cost), feas.ctypes.data_as(C.POINTER(C.c_ubyte)), _p(viol), cost.shape[0],
                         C.byref(anyf))
    return k, bool(anyf.value)


def best_response(params, track: Track, x0, u_nom, vref_scale, opp, T, K, seed=0, race=0, agent=0, rnd=0,
                  stream=0, game_on=True, want_costs=False, nthreads=None, prop=None, K_prop=0):
    """One best response.  ``prop`` (T x 4: mean a, mean delta, sigma a,
    sigma delta) with ``K_prop`` draws the first K_prop samples from the
    proposal (noise stream 1); the rest come from the plain sampler."""
    opp = _d(opp).reshape(-1, T + 1, 4) if opp is not None and np.size(opp) else np.zeros((0, T + 1, 4))
    ks = C.c_int(); anyf = C.c_int()
    u_star = np.zeros((T, 2)); xi = np.zeros((T + 1, 4))
    costs = np.zeros(K) if want_costs else None
    viols = np.zeros(K) if want_costs else None
    pr = _d(prop).reshape(T, 4) if prop is not None else None
    rc = lib().orc_best_response_mixed(
        C.byref(make_params(params)), *track.args(), _p(_d(x0)), _p(_d(u_nom)), float(np.float32(vref_scale)),
        _p(opp) if opp.shape[0] else None, opp.shape[0], T, K, seed, race, agent, rnd, stream,
        int(bool(game_on)), _p(pr), int(K_prop) if pr is not None else 0, C.byref(ks), _p(u_star), _p(xi),
        C.byref(anyf), _p(costs), _p(viols), _nthreads(nthreads))
    assert rc == 0
    out = dict(k_star=ks.value, u_star=u_star, xi_star=xi, any_feasible=bool(anyf.value))
    if want_costs:
        out["costs"] = costs
        out["viols"] = viols
    return out


def ibr_plan(params, track: Track, X0, U_nom, vref_scale, T, K, L, ego, seed=0, race=0, nthreads=None,
             want_hist=False):
    X0 = _d(X0).reshape(-1, 4)
    n_v = X0.shape[0]
    U = _d(U_nom).reshape(n_v, T, 2).copy()
    vs = _d([float(np.float32(v)) for v in vref_scale])
    xi = np.zeros((n_v, T + 1, 4))
    ks = np.zeros((L + 1) * n_v + 1, dtype=np.int32)
    xh = np.zeros((L + 2, n_v, T + 1, 4)) if want_hist else None
    uh = np.zeros((L + 2, n_v, T, 2)) if want_hist else None
    rc = lib().orc_ibr_plan(C.byref(make_params(params)), *track.args(), n_v, _p(X0), _p(U), _p(vs), T, K, L, ego,
                            seed, race, _p(xi), ks.ctypes.data_as(C.POINTER(C.c_int)), _p(xh), _p(uh),
                            _nthreads(nthreads))
    assert rc == 0
    out = dict(xi=xi, u_nom=U, k_star=ks)
    if want_hist:
        out["xi_hist"] = xh
        out["u_hist"] = uh
    return out


def best_response_mppi(params, track: Track, x0, u_nom, vref_scale, opp, T, K, lam, seed=0, race=0, agent=0, rnd=0,
                       game_on=True, want_costs=False, nthreads=None):
    """One GA-IBR-MPPI best response at temperature ``lam``: the
    importance-weighted mean of the K sampled control sequences
    (``u_new``), its rollout (``xi_new``) and the lowest-cost sample."""
    opp = _d(opp).reshape(-1, T + 1, 4) if opp is not None and np.size(opp) else np.zeros((0, T + 1, 4))
    km = C.c_int()
    u_new = np.zeros((T, 2)); xi = np.zeros((T + 1, 4))
    costs = np.zeros(K) if want_costs else None
    rc = lib().orc_best_response_mppi(
        C.byref(make_params(params)), *track.args(), _p(_d(x0)), _p(_d(u_nom)), float(np.float32(vref_scale)),
        _p(opp) if opp.shape[0] else None, opp.shape[0], T, K, seed, race, agent, rnd, int(bool(game_on)),
        float(lam), C.byref(km), _p(u_new), _p(xi), _p(costs), _nthreads(nthreads))
    assert rc == 0
    out = dict(k_min=km.value, u_new=u_new, xi_new=xi)
    if want_costs:
        out["costs"] = costs
    return out


def ibr_plan_mppi(params, track: Track, X0, U_nom, vref_scale, T, K, L, ego, lam, seed=0, race=0, nthreads=None,
                  want_hist=False):
    """The GA-IBR-MPPI planning call: :func:`ibr_plan` with the
    path-integral update at temperature ``lam``."""
    X0 = _d(X0).reshape(-1, 4)
    n_v = X0.shape[0]
    U = _d(U_nom).reshape(n_v, T, 2).copy()
    vs = _d([float(np.float32(v)) for v in vref_scale])
    xi = np.zeros((n_v, T + 1, 4))
    ks = np.zeros((L + 1) * n_v + 1, dtype=np.int32)
    xh = np.zeros((L + 2, n_v, T + 1, 4)) if want_hist else None
    uh = np.zeros((L + 2, n_v, T, 2)) if want_hist else None
    rc = lib().orc_ibr_plan_mppi(C.byref(make_params(params)), *track.args(), n_v, _p(X0), _p(U), _p(vs), T, K, L,
                                 ego, seed, race, float(lam), _p(xi), ks.ctypes.data_as(C.POINTER(C.c_int)), _p(xh),
                                 _p(uh), _nthreads(nthreads))
    assert rc == 0
    out = dict(xi=xi, u_nom=U, k_star=ks)
    if want_hist:
        out["xi_hist"] = xh
        out["u_hist"] = uh
    return out


def perturb_prediction(track: Track, states, T, seed, race, observer, rnd, jv, sigma_lon, sigma_lat, n_tail):
    """Opponent jv's prediction (T+1 x 4 states) as perturbed for vehicle
    ``observer`` in round ``rnd``; returns (states', (d gain, d tail mean))."""
    st = _d(states).reshape(T + 1, 4)
    out = np.zeros_like(st)
    delta = np.zeros(2)
    rc = lib().orc_perturb_prediction(*track.args(), _p(st), T, seed, race, observer, rnd, jv, float(sigma_lon),
                                      float(sigma_lat), int(n_tail), _p(out), _p(delta))
    assert rc == 0
    return out, delta


def ibr_plan_perturbed(params, track: Track, X0, U_nom, vref_scale, T, K, L, ego, sigma_lon, sigma_lat, seed=0, race=0,
                       nthreads=None, want_hist=False):
    """:func:`ibr_plan` with every opponent prediction perturbed before each
    best response (:func:`perturb_prediction`)."""
    X0 = _d(X0).reshape(-1, 4)
    n_v = X0.shape[0]
    U = _d(U_nom).reshape(n_v, T, 2).copy()
    vs = _d([float(np.float32(v)) for v in vref_scale])
    xi = np.zeros((n_v, T + 1, 4))
    ks = np.zeros((L + 1) * n_v + 1, dtype=np.int32)
    xh = np.zeros((L + 2, n_v, T + 1, 4)) if want_hist else None
    uh = np.zeros((L + 2, n_v, T, 2)) if want_hist else None
    rc = lib().orc_ibr_plan_perturbed(C.byref(make_params(params)), *track.args(), n_v, _p(X0), _p(U), _p(vs), T, K,
                                      L, ego, seed, race, float(sigma_lon), float(sigma_lat), _p(xi),
                                      ks.ctypes.data_as(C.POINTER(C.c_int)), _p(xh), _p(uh), _nthreads(nthreads))
    assert rc == 0
    out = dict(xi=xi, u_nom=U, k_star=ks)
    if want_hist:
        out["xi_hist"] = xh
        out["u_hist"] = uh
    return out


def rollout_costs_perturbed(params, track: Track, x0, u_nom, vref_scale, opp, opp_pos, sum_delta, T, K=None,
                            k_list=None, seed=0, race=0, agent=0, rnd=0, game_on=True, want_states=False,
                            want_controls=False, nthreads=None):
    """:func:`rollout_costs` with perturbed opponent data: positions of the
    distance terms from ``opp_pos``, summaries of ``opp`` shifted by
    ``sum_delta`` (n_opp x 2), as :func:`perturb_prediction` returns them."""
    opp = _d(opp).reshape(-1, T + 1, 4)
    opp_pos = _d(opp_pos).reshape(-1, T + 1, 4)
    sd = _d(sum_delta).reshape(-1, 2)
    n_opp = opp.shape[0]
    if k_list is not None:
        kl = np.ascontiguousarray(np.asarray(k_list, dtype=np.int32))
        n = kl.shape[0]
        klp = kl.ctypes.data_as(C.POINTER(C.c_int32))
    else:
        n = int(K)
        klp = None
    cost = np.zeros(n); viol = np.zeros(n); feas = np.zeros(n, dtype=np.uint8); mg = np.zeros((n, 3))
    states = np.zeros((n, T + 1, 4)) if want_states else None
    ctl = np.zeros((n, T, 2)) if want_controls else None
    rc = lib().orc_rollout_costs_perturbed(
        C.byref(make_params(params)), *track.args(), _p(_d(x0)), _p(_d(u_nom)), float(np.float32(vref_scale)),
        _p(opp), _p(opp_pos), _p(sd), n_opp, T, klp, n, seed, race, agent, rnd, int(bool(game_on)), _p(cost),
        feas.ctypes.data_as(C.POINTER(C.c_ubyte)), _p(viol), _p(states), _p(ctl), _p(mg), _nthreads(nthreads))
    assert rc == 0
    out = dict(cost=cost, feasible=feas, violation=viol, margins=mg)
    if want_states:
        out["states"] = states
    if want_controls:
        out["controls"] = ctl
    return out
