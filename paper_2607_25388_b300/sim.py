"""Closed-loop race trials on the GPU (receding horizon) and their metrics
(Sec. IV-C, Evaluation Metrics).

Every trial is one race of an ``sgtp_batch``.  Each control period runs one
batched planning call (SGTP, SGTP without the game-aware cost, or the
GA-IBR-MPPI ablation) and one ``sgtp_sim_step`` on the same stream: the
plan's first ``n_apply`` control steps are applied (its controls, or pure
pursuit on its trajectory), every vehicle is stepped and projected, the
ego's contacts are checked and the metric sums are kept on the device.

Metrics over a set of trials (the paper's definitions; distances in metres,
times in seconds):

* Wins: share of trials with ego progress gain > every opponent's + eps_s;
* CFW: share of the winning trials in which the ego made no contact;
* FPR: mean over trials of the share of opponents the ego is ahead of at
  the end (by more than eps_s in unwrapped Frenet progress);
* D_max, D_mean, D_ratio: trial durations (a trial ends at the ego's first
  contact or at the limit) and D_mean over the limit;
* CSD: mean length of the close-interaction segments;
* v_ego: mean ego speed over all simulated steps of all trials;
* MCS: mean over trials of the mean of ||u_k - u_{k-1}||^2 over the ego's
  applied controls;
* CT: wall time of each planning call (CUDA events), mean / std / max.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from ._lib import SimParams, SimRace, check, lib
from .planner import Batch, Track, launch_opts, make_params, stream_ptr

TRACK_CONTROLS, TRACK_PURE_PURSUIT = 0, 1
_INTS_PER_RACE = C.sizeof(SimRace) // 4


def sim_params(n_apply=1, max_steps=1000, tracker=TRACK_CONTROLS, pp_preview=3, contact_dist=2.5, wall_margin=0.0,
               close_ds=5.0, close_dd=2.5) -> SimParams:
    """Defaults at the full scale of these scenarios: physical contact below
    2.5 m between reference points (the planner's collision threshold d_col =
    4.5 m keeps a margin over it, as the paper's 0.9 m does over its
    1/10-scale cars' contact distance, a ratio of about 1.8), wall contact
    when the reference point leaves the track, and the paper's
    close-interaction box (1.0 m x 0.5 m at 1/10 scale) scaled by 5."""
    return SimParams(int(n_apply), int(max_steps), int(tracker), int(pp_preview), float(contact_dist),
                     float(wall_margin), float(close_ds), float(close_dd))


class Trials:
    """A set of closed-loop trials run together (one batch)."""

    def __init__(self, scenarios, params: dict, K: int, L: int, sp: SimParams, mppi_lambda=None, opts=None,
                 device="cuda", pred_sigma=None):
        self.scenarios = scenarios
        self.params = params
        self.sp = sp
        self.mppi_lambda = mppi_lambda
        self.pred_sigma = pred_sigma
        self.track = Track.from_many([sc.track for sc in scenarios])
        self.batch = Batch(self.track, [dict(track_id=r, n_v=sc.X0.shape[0], T=sc.T, ego=sc.ego, race_tag=r)
                                        for r, sc in enumerate(scenarios)], K=K, L=L)
        dev = torch.device(device)
        self.X0 = torch.as_tensor(np.concatenate([sc.X0 for sc in scenarios])).to(dev)
        self.U0 = torch.as_tensor(np.concatenate([sc.U0.reshape(-1) for sc in scenarios])).to(dev)
        self.vs = torch.as_tensor(np.concatenate([sc.vref_scale for sc in scenarios])).to(dev)
        self.X = self.X0.clone()
        self.U = self.U0.clone()
        self.state = torch.zeros(len(scenarios) * C.sizeof(SimRace), dtype=torch.uint8, device=dev)
        self.out = self.batch._outputs(dev, False)
        nb = self.batch.workspace_bytes if mppi_lambda is None else self.batch.mppi_workspace_bytes
        self.ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=dev)
        self.P = make_params(params)
        self.opts = opts if opts is not None else launch_opts()
        self.k = 0

    def reset(self):
        self.X.copy_(self.X0)
        self.U.copy_(self.U0)
        self.k = 0
        check(lib().sgtp_sim_reset(self.batch.handle, self.X.data_ptr(), self.state.data_ptr(), stream_ptr(None)),
              "sgtp_sim_reset")

    def plan(self):
        self.batch.plan(self.params, self.X, self.U, self.vs, seed=self.k, opts=self.opts, workspace=self.ws,
                        out=self.out, mppi_lambda=self.mppi_lambda, pred_sigma=self.pred_sigma)

    def sim_step(self):
        check(lib().sgtp_sim_step(self.batch.handle, C.byref(self.P), C.byref(self.sp), self.X.data_ptr(),
                                  self.U.data_ptr(), self.out["xi"].data_ptr(), self.state.data_ptr(),
                                  stream_ptr(None)), "sgtp_sim_step")

    def step(self):
        """One control period: plan (seed = period index), then simulate."""
        self.plan()
        self.sim_step()
        self.k += 1

    def alive(self) -> int:
        return int(self.state.view(torch.int32).view(-1, _INTS_PER_RACE)[:, 0].sum().item())

    def run(self, max_periods=None, check_every=25, timing=True):
        """Run control periods until every trial has ended (or max_periods).
        Returns the planning calls' times in ms (CUDA events) when timing."""
        n = max_periods if max_periods is not None else math.ceil(self.sp.max_steps / self.sp.n_apply)
        ev = []
        s = torch.cuda.current_stream()
        for q in range(n):
            if timing:
                a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                a.record(s)
                self.plan()
                b.record(s)
                self.sim_step()
                c.record(s)
                ev.append((a, b, c))
                self.k += 1
            else:
                self.step()
            if (q + 1) % check_every == 0 and self.alive() == 0:
                break
        torch.cuda.synchronize()
        self.sim_times = [b.elapsed_time(c) for a, b, c in ev]
        return [a.elapsed_time(b) for a, b, c in ev]

    def results(self):
        """Per-trial records (sgtp_sim_race fields) as dicts."""
        raw = self.state.cpu().numpy().tobytes()
        arr = (SimRace * len(self.scenarios)).from_buffer_copy(raw)
        out = []
        for sc, r in zip(self.scenarios, arr):
            n_v = sc.X0.shape[0]
            out.append(dict(n_v=n_v, ego=sc.ego, alive=r.alive, steps=r.steps, ego_collision=r.ego_collision,
                            close_segments=r.close_segments, close_steps=r.close_steps,
                            ego_speed_sum=r.ego_speed_sum, ego_du2_sum=r.ego_du2_sum,
                            progress=np.array(r.progress[:n_v]), rel0=np.array(r.rel0[:n_v]),
                            d=np.array(r.d[:n_v])))
        return out


def trial_metrics(results, dt: float, limit_s: float, eps_s: float = 0.025) -> dict:
    """The paper's trial metrics from per-trial records (see module doc).
    eps_s: the paper's 5e-3 m margin scaled with the scenarios (x5)."""
    wins, clean_wins, fpr, dur, mcs = [], 0, [], [], []
    seg_n = seg_steps = 0
    v_sum, v_cnt = 0.0, 0
    for r in results:
        n_v, e = r["n_v"], r["ego"]
        ds, rel0 = np.asarray(r["progress"], np.float64), np.asarray(r["rel0"], np.float64)
        opp = [j for j in range(n_v) if j != e]
        win = bool(not opp or ds[e] > max(ds[j] for j in opp) + eps_s)
        wins.append(win)
        if win and r["ego_collision"] == 0:
            clean_wins += 1
        if opp:
            # s_e,T - s_j,T = (s_e,0 - s_j,0) + ds_e - ds_j, with rel0_j = s_j,0 - s_e,0
            fpr.append(float(np.mean([ds[e] - ds[j] - rel0[j] > eps_s for j in opp])))
        dur.append(r["steps"] * dt)
        seg_n += r["close_segments"]
        seg_steps += r["close_steps"]
        v_sum += r["ego_speed_sum"]
        v_cnt += r["steps"]
        if r["steps"] > 1:
            mcs.append(r["ego_du2_sum"] / (r["steps"] - 1))
    n_w = sum(wins)
    return dict(trials=len(results), wins=n_w / max(1, len(results)),
                cfw=clean_wins / n_w if n_w else float("nan"),
                fpr=float(np.mean(fpr)) if fpr else float("nan"),
                csd=seg_steps * dt / seg_n if seg_n else 0.0,
                d_mean=float(np.mean(dur)) if dur else 0.0, d_max=float(np.max(dur)) if dur else 0.0,
                d_ratio=(float(np.mean(dur)) / limit_s) if dur else 0.0,
                v_ego=v_sum / v_cnt if v_cnt else 0.0,
                mcs=float(np.mean(mcs)) if mcs else float("nan"),
                contacts=float(np.mean([r["ego_collision"] != 0 for r in results])) if results else 0.0)


def ct_stats(times_ms, n_races: int) -> dict:
    """CT of the planning calls: mean / std / max per launch, and the mean
    per race (a launch plans every trial at once)."""
    t = np.asarray(times_ms, np.float64)
    if t.size == 0:
        return dict(ct_mean_ms=0.0, ct_std_ms=0.0, ct_max_ms=0.0, ct_mean_per_race_ms=0.0)
    return dict(ct_mean_ms=float(t.mean()), ct_std_ms=float(t.std()), ct_max_ms=float(t.max()),
                ct_mean_per_race_ms=float(t.mean() / n_races))
