"""Thin PyTorch binding of the SGTP best-response engine (``include/sgtp.h``).

Tensors supply device memory and the current CUDA stream; every computation
runs in ``libsgtp.so``.  There is no CPU path: calling any compute function
without a CUDA device raises.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import check, lib, make_params

__all__ = ["sync_status", "Track", "rollout_costs", "best_response", "best_response_noalloc", "best_response_mixed", "PlanGraph", "ibr_plan", "Batch", "launch_opts",
           "stream_ptr", "br_workspace_bytes", "plan_workspace_bytes"]


def sync_status(status: torch.Tensor, stream=None) -> int:
    """Wait for the stream and return a planning call's device status word
    (0, or SGTP_E_* in the low byte with flag bits above it)."""
    _dev(status, "status", dtype=torch.int32, shape=(1,))
    out = C.c_int32()
    check(lib().sgtp_sync_status(status.data_ptr(), stream_ptr(stream), C.byref(out)), "sgtp_sync_status")
    return int(out.value)


def stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev(t: torch.Tensor, name: str, dtype=torch.float32, shape=None) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.data_ptr()


def _opt(t, name, dtype=torch.float32, shape=None):
    return None if t is None else _dev(t, name, dtype, shape)


def _ws(nbytes: int, device) -> torch.Tensor:
    # 256-byte alignment: the caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


SCHEDULE_DEFAULT, SCHEDULE_LOCKSTEP, SCHEDULE_QUEUE = 0, 1, 2


def launch_opts(block=0, samples_per_thread=0, ctas_per_sm=0, window=0, wait_timeout_ns=0, debug_flags=0,
                trace=None, schedule=SCHEDULE_DEFAULT):
    """Launch shape of the persistent kernel (0 = library default).  trace:
    optional int64 CUDA tensor of 3*L+8 entries for per-phase timestamps.
    schedule: SCHEDULE_LOCKSTEP (grid barrier after every phase) or
    SCHEDULE_QUEUE (per-race round progression from a device work queue);
    the default takes the queue for batches."""
    return _lib.LaunchOpts(int(block), int(samples_per_thread), int(ctas_per_sm), int(window), int(wait_timeout_ns),
                           int(debug_flags), int(schedule), None if trace is None else trace.data_ptr())


class Track:
    """Device raceline(s).  xr: (N, 4) float32 waypoints (x, y, psi, v^r),
    wl, wr: (N,) widths; several tracks concatenate with ``offsets``."""

    def __init__(self, xr, wl, wr, offsets=None, stream=None):
        xr = np.ascontiguousarray(np.asarray(xr, dtype=np.float32).reshape(-1, 4))
        wl = np.ascontiguousarray(np.asarray(wl, dtype=np.float32).reshape(-1))
        wr = np.ascontiguousarray(np.asarray(wr, dtype=np.float32).reshape(-1))
        if offsets is None:
            offsets = [0, xr.shape[0]]
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
        h = C.c_void_p()
        st = lib().sgtp_track_create_many(xr.ctypes.data, wl.ctypes.data, wr.ctypes.data, off.ctypes.data,
                                          off.shape[0] - 1, stream_ptr(stream) if torch.cuda.is_available() else None,
                                          C.byref(h))
        check(st, "sgtp_track_create_many")
        self._h = h
        self.n_tracks = off.shape[0] - 1

    @classmethod
    def from_data(cls, td, stream=None):
        return cls(td.xr, td.wl, td.wr, stream=stream)

    @classmethod
    def from_many(cls, tds, stream=None):
        off = np.concatenate([[0], np.cumsum([t.N for t in tds])])
        return cls(np.concatenate([t.xr for t in tds]), np.concatenate([t.wl for t in tds]),
                   np.concatenate([t.wr for t in tds]), offsets=off, stream=stream)

    @property
    def handle(self):
        return self._h

    def info(self, track_id=0):
        n = C.c_int32(); N = C.c_int32(); L = C.c_float()
        check(lib().sgtp_track_info(self._h, track_id, C.byref(n), C.byref(N), C.byref(L)), "sgtp_track_info")
        return dict(n_tracks=n.value, N=N.value, length=L.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.sgtp_track_destroy(h)
            self._h = None


def br_workspace_bytes(n_opp: int, T: int) -> int:
    return int(lib().sgtp_br_workspace_bytes(n_opp, T))


def plan_workspace_bytes(n_v: int, T: int, L: int) -> int:
    return int(lib().sgtp_plan_workspace_bytes(n_v, T, L))


def plan_mppi_workspace_bytes(n_v: int, T: int, L: int, K: int) -> int:
    return int(lib().sgtp_plan_mppi_workspace_bytes(n_v, T, L, K))


def _br_inputs(x0, u_nom, opp, T):
    dev = x0.device
    _dev(x0, "x0", shape=(4,))
    _dev(u_nom, "u_nom", shape=(T, 2))
    if opp is None or opp.numel() == 0:
        return 0, None, dev
    n_opp = opp.shape[0]
    _dev(opp, "opp", shape=(n_opp, T + 1, 4))
    return n_opp, opp.data_ptr(), dev


def rollout_costs(track: Track, params: dict, x0, u_nom, vref_scale, opp, T, K, seed=0, race=0, agent=0, rnd=0,
                  game_on=True, track_id=0, want_states=False, want_frenet=False, want_controls=False,
                  workspace=None, stream=None):
    """Per-candidate cost, feasibility and violation of one best response."""
    n_opp, opp_p, dev = _br_inputs(x0, u_nom, opp, T)
    cost = torch.empty(K, dtype=torch.float32, device=dev)
    feas = torch.empty(K, dtype=torch.uint8, device=dev)
    viol = torch.empty(K, dtype=torch.float32, device=dev)
    states = torch.empty((K, T + 1, 4), dtype=torch.float32, device=dev) if want_states else None
    fr = torch.empty((K, T + 1, 2), dtype=torch.float32, device=dev) if want_frenet else None
    ctl = torch.empty((K, T, 2), dtype=torch.float32, device=dev) if want_controls else None
    nb = br_workspace_bytes(n_opp, T)
    ws = workspace if workspace is not None else _ws(nb, dev)
    P = make_params(params)
    st = lib().sgtp_rollout_costs(track.handle, track_id, C.byref(P), x0.data_ptr(), u_nom.data_ptr(),
                                  float(vref_scale), opp_p, n_opp, T, K, int(seed), race, agent, rnd, int(game_on),
                                  cost.data_ptr(), feas.data_ptr(), viol.data_ptr(),
                                  None if states is None else states.data_ptr(), None if fr is None else fr.data_ptr(),
                                  None if ctl is None else ctl.data_ptr(), ws.data_ptr(), ws.numel(),
                                  stream_ptr(stream))
    check(st, "sgtp_rollout_costs")
    out = dict(cost=cost, feasible=feas, violation=viol)
    if want_states:
        out["states"] = states
    if want_frenet:
        out["frenet"] = fr
    if want_controls:
        out["controls"] = ctl
    return out


def best_response(track: Track, params: dict, x0, u_nom, vref_scale, opp, T, K, seed=0, race=0, agent=0, rnd=0,
                  game_on=True, track_id=0, workspace=None, out=None, stream=None):
    """One best response: selection (Eq. selection, least-violation fallback)
    and the re-rolled winner.  Returns device tensors."""
    n_opp, opp_p, dev = _br_inputs(x0, u_nom, opp, T)
    if out is None:
        out = dict(k_star=torch.empty(1, dtype=torch.int32, device=dev),
                   u_star=torch.empty((T, 2), dtype=torch.float32, device=dev),
                   xi_star=torch.empty((T + 1, 4), dtype=torch.float32, device=dev),
                   any_feasible=torch.empty(1, dtype=torch.int32, device=dev))
    nb = br_workspace_bytes(n_opp, T)
    ws = workspace if workspace is not None else _ws(nb, dev)
    P = make_params(params)
    st = lib().sgtp_best_response(track.handle, track_id, C.byref(P), x0.data_ptr(), u_nom.data_ptr(),
                                  float(vref_scale), opp_p, n_opp, T, K, int(seed), race, agent, rnd, int(game_on),
                                  out["k_star"].data_ptr(), out["u_star"].data_ptr(), out["xi_star"].data_ptr(),
                                  out["any_feasible"].data_ptr(), ws.data_ptr(), ws.numel(), stream_ptr(stream))
    check(st, "sgtp_best_response")
    return out


def best_response_noalloc(track: Track, params: dict, x0, u_nom, vref_scale, opp, T, K, seed=0, race=0, agent=0,
                          rnd=0, game_on=True, track_id=0, out=None, stream=None):
    """sgtp_best_response with the library's static scratch instead of a
    workspace.  Calls that overlap in time share that scratch: issue them on
    one stream."""
    n_opp, opp_p, dev = _br_inputs(x0, u_nom, opp, T)
    if out is None:
        out = dict(k_star=torch.empty(1, dtype=torch.int32, device=dev),
                   u_star=torch.empty((T, 2), dtype=torch.float32, device=dev),
                   xi_star=torch.empty((T + 1, 4), dtype=torch.float32, device=dev),
                   any_feasible=torch.empty(1, dtype=torch.int32, device=dev))
    P = make_params(params)
    st = lib().sgtp_best_response_noalloc(track.handle, track_id, C.byref(P), x0.data_ptr(), u_nom.data_ptr(),
                                          float(vref_scale), opp_p, n_opp, T, K, int(seed), race, agent, rnd,
                                          int(game_on), out["k_star"].data_ptr(), out["u_star"].data_ptr(),
                                          out["xi_star"].data_ptr(), out["any_feasible"].data_ptr(),
                                          stream_ptr(stream))
    check(st, "sgtp_best_response_noalloc")
    return out


def best_response_mixed(track: Track, params: dict, x0, u_nom, vref_scale, opp, T, K, prop, K_prop, seed=0, race=0,
                        agent=0, rnd=0, game_on=True, track_id=0, workspace=None, stream=None):
    """One best response with the first K_prop samples drawn from the
    per-step proposal prop (T, 4) (mean a, mean delta, sigma a, sigma
    delta); also returns the selected cost."""
    n_opp, opp_p, dev = _br_inputs(x0, u_nom, opp, T)
    _dev(prop, "prop", shape=(T, 4))
    out = dict(k_star=torch.empty(1, dtype=torch.int32, device=dev),
               u_star=torch.empty((T, 2), dtype=torch.float32, device=dev),
               xi_star=torch.empty((T + 1, 4), dtype=torch.float32, device=dev),
               any_feasible=torch.empty(1, dtype=torch.int32, device=dev),
               cost=torch.empty(1, dtype=torch.float32, device=dev))
    nb = br_workspace_bytes(n_opp, T)
    ws = workspace if workspace is not None else _ws(nb, dev)
    P = make_params(params)
    st = lib().sgtp_best_response_mixed(track.handle, track_id, C.byref(P), x0.data_ptr(), u_nom.data_ptr(),
                                        float(vref_scale), opp_p, n_opp, T, K, int(seed), race, agent, rnd,
                                        int(game_on), prop.data_ptr(), int(K_prop), out["k_star"].data_ptr(),
                                        out["u_star"].data_ptr(), out["xi_star"].data_ptr(),
                                        out["any_feasible"].data_ptr(), out["cost"].data_ptr(), ws.data_ptr(),
                                        ws.numel(), stream_ptr(stream))
    check(st, "sgtp_best_response_mixed")
    return out


def ibr_plan(track: Track, params: dict, X0, U_io, vref_scale, T, K, L, ego=0, seed=0, race=0, track_id=0,
             want_hist=False, opts=None, workspace=None, out=None, stream=None, mlp=None, K_prop=0,
             want_features=False, want_prop=False, mppi_lambda=None, pred_sigma=None):
    """The SGTP planning call (Alg. 1) for one race; U_io is updated in place
    (warm start).  Returns device tensors xi (n_v, T+1, 4), k_star, status.
    With ``mlp`` (a :class:`learned.Mlp`) K_prop samples of every best
    response come from the network's proposal; ``want_features`` returns
    the features of every best response ((L+2, n_v, 64)), ``want_prop`` the
    proposals ((L+2, n_v, T, 4)).  With ``mppi_lambda`` the call is the
    GA-IBR-MPPI ablation (sgtp_ibr_plan_mppi): every response's controls
    become the path-integral mean at that temperature, and k_star holds the
    lowest-cost samples.  With ``pred_sigma = (sigma_lon, sigma_lat)`` every
    opponent prediction is perturbed before use (sgtp_ibr_plan_perturbed)."""
    n_v = X0.shape[0]
    dev = X0.device
    _dev(X0, "X0", shape=(n_v, 4))
    _dev(U_io, "U_io", shape=(n_v, T, 2))
    _dev(vref_scale, "vref_scale", shape=(n_v,))
    if out is None:
        out = dict(xi=torch.empty((n_v, T + 1, 4), dtype=torch.float32, device=dev),
                   k_star=torch.empty((L + 1) * n_v + 1, dtype=torch.int32, device=dev),
                   status=torch.zeros(1, dtype=torch.int32, device=dev))
        if want_hist:
            out["xi_hist"] = torch.empty((L + 2, n_v, T + 1, 4), dtype=torch.float32, device=dev)
            out["u_hist"] = torch.empty((L + 2, n_v, T, 2), dtype=torch.float32, device=dev)
    if mppi_lambda is not None and (mlp is not None or want_features or want_prop):
        raise ValueError("GA-IBR-MPPI takes the plain sampler only")
    if pred_sigma is not None and (mppi_lambda is not None or mlp is not None or want_features or want_prop):
        raise ValueError("perturbed predictions take the plain SGTP call only")
    nb = plan_workspace_bytes(n_v, T, L) if mppi_lambda is None else plan_mppi_workspace_bytes(n_v, T, L, K)
    ws = workspace if workspace is not None else _ws(nb, dev)
    P = make_params(params)
    if isinstance(opts, str):
        if opts != "auto":
            raise ValueError("opts must be launch options, None or 'auto'")
        from . import autotune
        opts = autotune.lookup(n_v, T, K, L)
    o = opts if opts is not None else launch_opts()
    if mlp is not None or want_features or want_prop:
        if want_features and "features" not in out:
            out["features"] = torch.zeros((L + 2, n_v, 64), dtype=torch.float32, device=dev)
        if want_prop and mlp is not None and "prop" not in out:
            out["prop"] = torch.zeros((L + 2, n_v, T, 4), dtype=torch.float32, device=dev)
        st = lib().sgtp_ibr_plan_learned(
            track.handle, track_id, C.byref(P), n_v, X0.data_ptr(), U_io.data_ptr(), vref_scale.data_ptr(), T, K, L,
            ego, int(seed), race, None if mlp is None else mlp.handle, int(K_prop), out["xi"].data_ptr(),
            out["k_star"].data_ptr(), out["xi_hist"].data_ptr() if "xi_hist" in out else None,
            out["u_hist"].data_ptr() if "u_hist" in out else None,
            out["features"].data_ptr() if "features" in out else None,
            out["prop"].data_ptr() if "prop" in out else None,
            out["status"].data_ptr(), C.byref(o), ws.data_ptr(), ws.numel(), stream_ptr(stream))
        check(st, "sgtp_ibr_plan_learned")
        return out
    if pred_sigma is not None:
        st = lib().sgtp_ibr_plan_perturbed(track.handle, track_id, C.byref(P), n_v, X0.data_ptr(), U_io.data_ptr(),
                                           vref_scale.data_ptr(), T, K, L, ego, int(seed), race,
                                           float(pred_sigma[0]), float(pred_sigma[1]), out["xi"].data_ptr(),
                                           out["k_star"].data_ptr(),
                                           out["xi_hist"].data_ptr() if "xi_hist" in out else None,
                                           out["u_hist"].data_ptr() if "u_hist" in out else None,
                                           out["status"].data_ptr(), C.byref(o), ws.data_ptr(), ws.numel(),
                                           stream_ptr(stream))
        check(st, "sgtp_ibr_plan_perturbed")
        return out
    if mppi_lambda is not None:
        st = lib().sgtp_ibr_plan_mppi(track.handle, track_id, C.byref(P), n_v, X0.data_ptr(), U_io.data_ptr(),
                                      vref_scale.data_ptr(), T, K, L, ego, int(seed), race, float(mppi_lambda),
                                      out["xi"].data_ptr(), out["k_star"].data_ptr(),
                                      out["xi_hist"].data_ptr() if "xi_hist" in out else None,
                                      out["u_hist"].data_ptr() if "u_hist" in out else None,
                                      out["status"].data_ptr(), C.byref(o), ws.data_ptr(), ws.numel(),
                                      stream_ptr(stream))
        check(st, "sgtp_ibr_plan_mppi")
        return out
    st = lib().sgtp_ibr_plan(track.handle, track_id, C.byref(P), n_v, X0.data_ptr(), U_io.data_ptr(),
                             vref_scale.data_ptr(), T, K, L, ego, int(seed), race, out["xi"].data_ptr(),
                             out["k_star"].data_ptr(),
                             out["xi_hist"].data_ptr() if "xi_hist" in out else None,
                             out["u_hist"].data_ptr() if "u_hist" in out else None,
                             out["status"].data_ptr(), C.byref(o), ws.data_ptr(), ws.numel(), stream_ptr(stream))
    check(st, "sgtp_ibr_plan")
    return out


class PlanGraph:
    """One planning call captured into a CUDA graph (``sgtp_graph_*``).

    The graph replays with the tensors given here: rewrite X0, U_io and
    vref_scale in place between launches (U_io keeps its warm start).
    ``out`` holds the output tensors (xi, k_star, status, and xi_hist /
    u_hist with want_hist)."""

    def __init__(self, handle, keep, out):
        self._h = handle
        self._keep = keep
        self.out = out

    @classmethod
    def capture_plan(cls, track: Track, params: dict, X0, U_io, vref_scale, T, K, L, ego=0, seed=0, race=0,
                     track_id=0, want_hist=False, opts=None):
        n_v = X0.shape[0]
        dev = X0.device
        _dev(X0, "X0", shape=(n_v, 4))
        _dev(U_io, "U_io", shape=(n_v, T, 2))
        _dev(vref_scale, "vref_scale", shape=(n_v,))
        out = dict(xi=torch.empty((n_v, T + 1, 4), dtype=torch.float32, device=dev),
                   k_star=torch.empty((L + 1) * n_v + 1, dtype=torch.int32, device=dev),
                   status=torch.zeros(1, dtype=torch.int32, device=dev))
        if want_hist:
            out["xi_hist"] = torch.empty((L + 2, n_v, T + 1, 4), dtype=torch.float32, device=dev)
            out["u_hist"] = torch.empty((L + 2, n_v, T, 2), dtype=torch.float32, device=dev)
        ws = _ws(plan_workspace_bytes(n_v, T, L), dev)
        P = make_params(params)
        o = opts if opts is not None else launch_opts()
        h = C.c_void_p()
        st = lib().sgtp_graph_capture_plan(
            track.handle, track_id, C.byref(P), n_v, X0.data_ptr(), U_io.data_ptr(), vref_scale.data_ptr(), T, K, L,
            ego, int(seed), race, out["xi"].data_ptr(), out["k_star"].data_ptr(),
            out["xi_hist"].data_ptr() if want_hist else None, out["u_hist"].data_ptr() if want_hist else None,
            out["status"].data_ptr(), C.byref(o), ws.data_ptr(), ws.numel(), C.byref(h))
        check(st, "sgtp_graph_capture_plan")
        return cls(h, (track, X0, U_io, vref_scale, ws, P, o), out)

    @classmethod
    def capture_batch(cls, batch: "Batch", params: dict, X0, U_io, vref_scale, seed=0, want_hist=False, opts=None):
        _dev(X0, "X0", shape=(batch.agents, 4))
        _dev(U_io, "U_io", shape=(batch.u_elems,))
        _dev(vref_scale, "vref_scale", shape=(batch.agents,))
        out = batch._outputs(X0.device, want_hist)
        ws = _ws(batch.workspace_bytes, X0.device)
        P = make_params(params)
        o = opts if opts is not None else launch_opts()
        h = C.c_void_p()
        st = lib().sgtp_graph_capture_batch(
            batch.handle, C.byref(P), X0.data_ptr(), U_io.data_ptr(), vref_scale.data_ptr(), int(seed),
            out["xi"].data_ptr(), out["k_star"].data_ptr(), out["xi_hist"].data_ptr() if want_hist else None,
            out["u_hist"].data_ptr() if want_hist else None, out["status"].data_ptr(), C.byref(o), ws.data_ptr(),
            ws.numel(), C.byref(h))
        check(st, "sgtp_graph_capture_batch")
        return cls(h, (batch, X0, U_io, vref_scale, ws, P, o), out)

    def set_seed(self, seed: int):
        check(lib().sgtp_graph_set_seed(self._h, int(seed)), "sgtp_graph_set_seed")

    def launch(self, stream=None):
        check(lib().sgtp_graph_launch(self._h, stream_ptr(stream)), "sgtp_graph_launch")
        return self.out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().sgtp_graph_destroy(h)
            except Exception:
                pass
            self._h = C.c_void_p()


class Batch:
    """Independent races planned in one persistent launch (sgtp_batch_*)."""

    def __init__(self, track: Track, races, K: int, L: int):
        arr = (_lib.Race * len(races))()
        for i, r in enumerate(races):
            arr[i] = _lib.Race(int(r["track_id"]), int(r["n_v"]), int(r["T"]), int(r.get("ego", 0)),
                               int(r.get("race_tag", i)))
        h = C.c_void_p()
        check(lib().sgtp_batch_create(track.handle, arr, len(races), K, L, C.byref(h)), "sgtp_batch_create")
        self._h = h
        self.track = track
        self.races = races
        self.K, self.L = K, L
        a, u, x, k = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        w = C.c_size_t()
        check(lib().sgtp_batch_sizes(h, C.byref(a), C.byref(u), C.byref(x), C.byref(k), C.byref(w)),
              "sgtp_batch_sizes")
        self.agents, self.u_elems, self.xi_elems, self.ks, self.workspace_bytes = a.value, u.value, x.value, \
            k.value, w.value

    @property
    def handle(self):
        return self._h

    def _outputs(self, dev, want_hist):
        out = dict(xi=torch.empty(self.xi_elems, dtype=torch.float32, device=dev),
                   k_star=torch.empty(self.ks, dtype=torch.int32, device=dev),
                   status=torch.zeros(1, dtype=torch.int32, device=dev))
        if want_hist:
            out["xi_hist"] = torch.empty((self.L + 2) * self.xi_elems, dtype=torch.float32, device=dev)
            out["u_hist"] = torch.empty((self.L + 2) * self.u_elems, dtype=torch.float32, device=dev)
        return out

    @property
    def mppi_workspace_bytes(self):
        w = C.c_size_t()
        check(lib().sgtp_batch_mppi_workspace_bytes(self._h, C.byref(w)), "sgtp_batch_mppi_workspace_bytes")
        return w.value

    def plan(self, params, X0, U_io, vref_scale, seed=0, want_hist=False, opts=None, workspace=None, out=None,
             stream=None, mlp=None, K_prop=0, mppi_lambda=None, pred_sigma=None):
        """Plan every race in one launch (``opts="auto"``: the autotuner's
        cached shape for this batch, if any); with ``mlp`` (a learned.Mlp) K_prop
        samples of every best response come from the network's proposal; with
        ``mppi_lambda`` every race runs the GA-IBR-MPPI ablation; with
        ``pred_sigma = (sigma_lon, sigma_lat)`` the opponent predictions are
        perturbed (sgtp_batch_plan_perturbed)."""
        dev = X0.device
        if isinstance(opts, str):
            if opts != "auto":
                raise ValueError("opts must be launch options, None or 'auto'")
            from . import autotune
            opts = autotune.lookup_batch(self)
        _dev(X0, "X0", shape=(self.agents, 4))
        _dev(U_io, "U_io", shape=(self.u_elems,))
        _dev(vref_scale, "vref_scale", shape=(self.agents,))
        if out is None:
            out = self._outputs(dev, want_hist)
        if mppi_lambda is not None and mlp is not None:
            raise ValueError("GA-IBR-MPPI takes the plain sampler only")
        ws = workspace if workspace is not None else _ws(
            self.workspace_bytes if mppi_lambda is None else self.mppi_workspace_bytes, dev)
        P = make_params(params)
        o = opts if opts is not None else launch_opts()
        if pred_sigma is not None:
            if mlp is not None or mppi_lambda is not None:
                raise ValueError("perturbed predictions take the plain SGTP call only")
            st = lib().sgtp_batch_plan_perturbed(self._h, C.byref(P), float(pred_sigma[0]), float(pred_sigma[1]),
                                                 X0.data_ptr(), U_io.data_ptr(), vref_scale.data_ptr(), int(seed),
                                                 out["xi"].data_ptr(), out["k_star"].data_ptr(),
                                                 out["xi_hist"].data_ptr() if "xi_hist" in out else None,
                                                 out["u_hist"].data_ptr() if "u_hist" in out else None,
                                                 out["status"].data_ptr(), C.byref(o), ws.data_ptr(), ws.numel(),
                                                 stream_ptr(stream))
            check(st, "sgtp_batch_plan_perturbed")
            return out
        if mppi_lambda is not None:
            st = lib().sgtp_batch_plan_mppi(self._h, C.byref(P), float(mppi_lambda), X0.data_ptr(), U_io.data_ptr(),
                                            vref_scale.data_ptr(), int(seed), out["xi"].data_ptr(),
                                            out["k_star"].data_ptr(),
                                            out["xi_hist"].data_ptr() if "xi_hist" in out else None,
                                            out["u_hist"].data_ptr() if "u_hist" in out else None,
                                            out["status"].data_ptr(), C.byref(o), ws.data_ptr(), ws.numel(),
                                            stream_ptr(stream))
            check(st, "sgtp_batch_plan_mppi")
            return out
        if mlp is not None:
            st = lib().sgtp_batch_plan_learned(
                self._h, C.byref(P), mlp.handle, int(K_prop), X0.data_ptr(), U_io.data_ptr(), vref_scale.data_ptr(),
                int(seed), out["xi"].data_ptr(), out["k_star"].data_ptr(),
                out["xi_hist"].data_ptr() if "xi_hist" in out else None,
                out["u_hist"].data_ptr() if "u_hist" in out else None, None, None, out["status"].data_ptr(),
                C.byref(o), ws.data_ptr(), ws.numel(), stream_ptr(stream))
            check(st, "sgtp_batch_plan_learned")
            return out
        st = lib().sgtp_batch_plan(self._h, C.byref(P), X0.data_ptr(), U_io.data_ptr(), vref_scale.data_ptr(),
                                   int(seed), out["xi"].data_ptr(), out["k_star"].data_ptr(),
                                   out["xi_hist"].data_ptr() if "xi_hist" in out else None,
                                   out["u_hist"].data_ptr() if "u_hist" in out else None,
                                   out["status"].data_ptr(), C.byref(o), ws.data_ptr(), ws.numel(),
                                   stream_ptr(stream))
        check(st, "sgtp_batch_plan")
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.sgtp_batch_destroy(h)
            self._h = None
