"""The learned proposal (not part of the SGTP paper): network handle,
closed-loop data generation from the plain planner, training, and the
learned-vs-plain comparison.

A small BF16 network (``include/sgtp_mlp.h``) maps the 64 Frenet-relative
features of a best response to a per-step Gaussian over its controls.  In a
learned plan, K_prop of the K samples of each best response come from that
Gaussian and the rest from the plain sampler of Sec. II, so the plain
sampler remains the fallback; selection is the paper's (Sec. III-B).

Every computation runs in ``libsgtp.so``; tensors only hold device memory.
The data generator advances races in closed loop: each vehicle applies the
first ``advance`` steps of its planned trajectory, its controls shift by as
many steps (warm start), and the next plan starts there (receding horizon).
"""
from __future__ import annotations

import ctypes as C
import json
import math
import time

import numpy as np
import torch

from . import scenario as S
from ._lib import check, lib
from .planner import Track, best_response_mixed, ibr_plan, launch_opts, stream_ptr

IN = 64


class Mlp:
    """Device network for horizon T (FP32 master + BF16 working weights,
    Adam state), created with Kaiming-uniform weights from Philox(seed)."""

    def __init__(self, T: int, seed: int = 0, stream=None):
        h = C.c_void_p()
        check(lib().sgtp_mlp_create(int(T), int(seed), stream_ptr(stream), C.byref(h)), "sgtp_mlp_create")
        self._h = h
        self.T = int(T)
        self.n_params = int(lib().sgtp_mlp_param_count(self.T))

    @property
    def handle(self):
        return self._h

    def reserve(self, batch: int):
        check(lib().sgtp_mlp_reserve(self._h, int(batch)), "sgtp_mlp_reserve")

    def forward(self, x: torch.Tensor, stream=None) -> torch.Tensor:
        B = x.shape[0]
        out = torch.empty((B, 4 * self.T), dtype=torch.float32, device=x.device)
        check(lib().sgtp_mlp_forward(self._h, x.data_ptr(), B, out.data_ptr(), stream_ptr(stream)), "sgtp_mlp_forward")
        return out

    def proposal(self, x: torch.Tensor, sigma_a: float, sigma_delta: float, u_nom=None, stream=None) -> torch.Tensor:
        """Per-step Gaussians (B, T, 4) around the rows' nominal controls
        u_nom (B, T, 2) (None: zero)."""
        B = x.shape[0]
        prop = torch.empty((B, self.T, 4), dtype=torch.float32, device=x.device)
        if u_nom is not None:
            assert u_nom.shape == (B, self.T, 2) and u_nom.is_contiguous() and u_nom.dtype == torch.float32
        check(lib().sgtp_mlp_proposal(self._h, x.data_ptr(), None if u_nom is None else u_nom.data_ptr(), B,
                                      float(sigma_a), float(sigma_delta), prop.data_ptr(), stream_ptr(stream)),
              "sgtp_mlp_proposal")
        return prop

    def train_step(self, x, target, lr=1e-3, apply=True, want_grad=False, loss_out=None, stream=None):
        """One Adam step on the batch (or only the gradient with apply=False).
        Returns (loss tensor [1], gradient tensor or None)."""
        B = x.shape[0]
        loss = loss_out if loss_out is not None else torch.empty(1, dtype=torch.float32, device=x.device)
        grad = torch.empty(self.n_params, dtype=torch.float32, device=x.device) if want_grad else None
        check(lib().sgtp_mlp_train_step(self._h, x.data_ptr(), target.data_ptr(), B, float(lr), loss.data_ptr(),
                                        None if grad is None else grad.data_ptr(), int(bool(apply)),
                                        stream_ptr(stream)), "sgtp_mlp_train_step")
        return loss, grad

    def get_params(self) -> np.ndarray:
        w = np.empty(self.n_params, dtype=np.float32)
        check(lib().sgtp_mlp_get_params(self._h, w.ctypes.data), "sgtp_mlp_get_params")
        return w

    def set_params(self, w) -> None:
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float32))
        if w.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {w.size}")
        check(lib().sgtp_mlp_set_params(self._h, w.ctypes.data), "sgtp_mlp_set_params")

    def info(self) -> dict:
        T = C.c_int32(); n = C.c_int64(); st = C.c_int64(); wb = C.c_void_p()
        check(lib().sgtp_mlp_info(self._h, C.byref(T), C.byref(n), C.byref(st), C.byref(wb)), "sgtp_mlp_info")
        return dict(T=T.value, n_params=n.value, step=st.value)

    def save(self, path: str) -> None:
        """Raw little-endian float32 parameters after a one-line JSON header."""
        hdr = json.dumps(dict(format="sgtp-mlp", T=self.T, n_params=self.n_params, dtype="<f4",
                              layout="per layer W[out][in] then b[out]; 64-256-256-256-4T")).encode()
        with open(path, "wb") as f:
            f.write(hdr + b"\n")
            f.write(self.get_params().astype("<f4").tobytes())

    @classmethod
    def load(cls, path: str, seed: int = 0) -> "Mlp":
        with open(path, "rb") as f:
            hdr = json.loads(f.readline())
            w = np.frombuffer(f.read(), dtype="<f4")
        m = cls(hdr["T"], seed)
        m.set_params(w)
        return m

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().sgtp_mlp_destroy(h)
            except Exception:
                pass
            self._h = C.c_void_p()


# ------------------------------------------------------------------ closed-loop races
class Race:
    """One race on the device, advanced in closed loop between plans."""

    def __init__(self, sc: S.Scenario, device="cuda"):
        self.sc = sc
        self.track = Track.from_data(sc.track)
        self.X = torch.tensor(sc.X0, device=device)
        self.U = torch.tensor(sc.U0, device=device)
        self.vs = torch.tensor(sc.vref_scale, device=device)
        self.n_v, self.T, self.K, self.L = sc.X0.shape[0], sc.T, sc.K, sc.L

    def advance(self, xi: torch.Tensor, steps: int):
        """Every vehicle applies the first `steps` steps of its plan."""
        self.X = xi[:, steps].contiguous()
        U = self.U.clone()
        U[:, :-steps] = self.U[:, steps:]
        U[:, -steps:] = self.U[:, -1:]
        self.U = U.contiguous()


def _targets(u: torch.Tensor, u_nom: torch.Tensor, params) -> torch.Tensor:
    """(n, T, 2) selected controls and the nominal controls they were sampled
    around -> (n, 2T) targets, the residuals in units of the plain sigmas:
    [(a - a_nom) / sigma_a, (delta - delta_nom) / sigma_delta]."""
    sa, sd = float(np.float32(params["sigma_a"])), float(np.float32(params["sigma_delta"]))
    r = u - u_nom
    return torch.cat([r[..., 0] / sa, r[..., 1] / sd], dim=-1)


def nominal_controls(u_start: torch.Tensor, u_hist: torch.Tensor, L: int) -> torch.Tensor:
    """The nominal controls of every best response of a plan, (L+2, n_v, T, 2):
    round 0 starts from the warm start, round r from round r-1's selection,
    and the extra ego response from round L's."""
    return torch.cat([u_start[None], u_hist[:L + 1]], dim=0)


def generate_dataset(seeds, plans_per_race: int, advance: int = 10, K=16384, T=60, L=5, params=None, seed0=0,
                     device="cuda", log=None):
    """(features [N, 64], targets [N, 2T]) from plain plans of ten-car races:
    every best response of every plan contributes its features and the
    residual of the controls it selected around its nominal controls
    ((L+1) n_v + 1 per plan)."""
    params = params or S.params_fullscale()
    xs, ys = [], []
    t0 = time.time()
    for n, seed in enumerate(seeds):
        race = Race(S.ten_car_race(int(seed), K=K, T=T, L=L), device)
        ego = race.sc.ego
        for q in range(plans_per_race):
            u_start = race.U.clone()
            out = ibr_plan(race.track, params, race.X, race.U, race.vs, T, K, L, ego=ego,
                           seed=seed0 + 7919 * int(seed) + q, want_hist=True, want_features=True)
            f, uh = out["features"], out["u_hist"]
            un = nominal_controls(u_start, uh, L)
            xs.append(f[:L + 1].reshape(-1, IN))
            ys.append(_targets(uh[:L + 1].reshape(-1, T, 2), un[:L + 1].reshape(-1, T, 2), params))
            xs.append(f[L + 1, ego:ego + 1])
            ys.append(_targets(uh[L + 1, ego:ego + 1], un[L + 1, ego:ego + 1], params))
            race.advance(out["xi"], advance)
        if log and (n + 1) % 10 == 0:
            log(f"dataset: {n + 1}/{len(seeds)} races, {sum(x.shape[0] for x in xs)} examples, "
                f"{time.time() - t0:.1f} s")
    return torch.cat(xs).contiguous(), torch.cat(ys).contiguous()


def train(mlp: Mlp, X: torch.Tensor, Y: torch.Tensor, epochs: int, batch=4096, lr=1e-3, seed=0, log=None,
          cosine=False):
    """Adam on the Gaussian NLL over shuffled mini-batches; returns the mean
    loss of each epoch.  With ``cosine`` the learning rate follows a cosine
    decay from lr to 0 over the epochs."""
    g = torch.Generator(device=X.device)
    g.manual_seed(seed)
    n = X.shape[0]
    mlp.reserve(batch)
    losses = []
    loss = torch.zeros(1, device=X.device)
    for ep in range(epochs):
        perm = torch.randperm(n, device=X.device, generator=g)
        acc = torch.zeros(1, device=X.device)
        nb = 0
        lr_e = lr * 0.5 * (1.0 + math.cos(math.pi * ep / epochs)) if cosine else lr
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            mlp.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr_e, loss_out=loss)
            acc += loss
            nb += 1
        losses.append(float(acc.item() / max(nb, 1)))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4f}")
    return losses


def compare(mlp: Mlp, seeds, states_per_race: int, advance=10, K=16384, K_eq=4096, K_prop=2048, T=60, L=5,
            params=None, device="cuda"):
    """Learned vs plain on the same best-response inputs (teacher-forced).

    Races advance in closed loop under the plain planner (K samples).  At
    each state, every game-on best response of the plain plan (rounds 1..L
    and the extra ego response) is re-solved three ways on its exact inputs:
    plain with K samples, plain with K_eq samples (equal budget), and learned
    with K_prop proposal + (K_eq - K_prop) plain samples.  End to end, the
    learned planner also plans from the same state and warm start, and the
    ego's final trajectory of each plan is scored against its own plan's
    round-L predictions.  Returns the selected costs and feasibility of
    each, per response and per plan."""
    params = params or S.params_fullscale()
    sa, sd = float(np.float32(params["sigma_a"])), float(np.float32(params["sigma_delta"]))
    rec = {k: [] for k in ("plain", "plain_eq", "learned", "feas_plain", "feas_plain_eq", "feas_learned",
                           "k_match", "e2e_plain", "e2e_learned", "e2e_feas_plain", "e2e_feas_learned")}

    def ego_final(out_, X0_, ego_, n_v_, seed_, race_):
        """Cost (violation if infeasible) and feasibility of the ego's final
        trajectory of a plan against the round-L predictions of that plan:
        its selected controls evaluated as the single, noise-free sample."""
        u = out_["u_hist"][L + 1, ego_].contiguous()
        opp = out_["xi_hist"][L, [j for j in range(n_v_) if j != ego_]].contiguous()
        prop = torch.stack([u[:, 0], u[:, 1], torch.full_like(u[:, 0], 1e-30), torch.full_like(u[:, 0], 1e-30)],
                           dim=1).contiguous()
        r_ = best_response_mixed(race_.track, params, X0_[ego_].contiguous(), u, float(race_.vs[ego_]), opp, T, 1,
                                 prop, 1, seed=seed_, agent=ego_, rnd=L + 1, game_on=True)
        return r_["cost"], r_["any_feasible"]

    for seed in seeds:
        race = Race(S.ten_car_race(int(seed), K=K, T=T, L=L), device)
        ego, n_v = race.sc.ego, race.n_v
        for q in range(states_per_race):
            pseed = 1_000_003 * int(seed) + q
            X0 = race.X.clone()
            U0 = race.U.clone()
            # end to end: the learned planner from the same state and warm start
            UL = U0.clone()
            outl = ibr_plan(race.track, params, X0, UL, race.vs, T, K_eq, L, ego=ego, seed=pseed, want_hist=True,
                            mlp=mlp, K_prop=K_prop)
            out = ibr_plan(race.track, params, race.X, race.U, race.vs, T, K, L, ego=ego, seed=pseed,
                           want_hist=True, want_features=True)
            for key, o_ in (("plain", out), ("learned", outl)):
                c_, f_ = ego_final(o_, X0, ego, n_v, pseed, race)
                rec["e2e_" + key].append(c_)
                rec["e2e_feas_" + key].append(f_)
            xh, uh, feat, ks = out["xi_hist"], out["u_hist"], out["features"], out["k_star"].cpu().numpy()
            jobs = [(r, i) for r in range(1, L + 2) for i in range(n_v) if r <= L or i == ego]
            F = torch.stack([feat[r, i] for r, i in jobs]).contiguous()
            UN = torch.stack([uh[r - 1, i] for r, i in jobs]).contiguous()
            P = mlp.proposal(F, sa, sd, UN)
            for n, (r, i) in enumerate(jobs):
                others = [j for j in range(n_v) if j != i]
                opp = xh[r - 1, others].contiguous()
                u_nom = uh[r - 1, i].contiguous()
                x0 = X0[i].contiguous()
                vs = float(race.vs[i])
                common = dict(seed=pseed, race=0, agent=i, rnd=r, game_on=True)
                a = best_response_mixed(race.track, params, x0, u_nom, vs, opp, T, K, P[n], 0, **common)
                b = best_response_mixed(race.track, params, x0, u_nom, vs, opp, T, K_eq, P[n], 0, **common)
                c = best_response_mixed(race.track, params, x0, u_nom, vs, opp, T, K_eq, P[n], K_prop, **common)
                rec["plain"].append(a["cost"]); rec["plain_eq"].append(b["cost"]); rec["learned"].append(c["cost"])
                rec["feas_plain"].append(a["any_feasible"]); rec["feas_plain_eq"].append(b["any_feasible"])
                rec["feas_learned"].append(c["any_feasible"])
                kpos = r * n_v + i if r <= L else (L + 1) * n_v
                rec["k_match"].append((a["k_star"], int(ks[kpos])))
            race.advance(out["xi"], advance)   # U was warm-started in place by the plan
    res = {}
    for k in ("plain", "plain_eq", "learned", "feas_plain", "feas_plain_eq", "feas_learned", "e2e_plain",
              "e2e_learned", "e2e_feas_plain", "e2e_feas_learned"):
        res[k] = torch.cat(rec[k]).float().cpu().numpy()
    km = [(int(a.item()), b) for a, b in rec["k_match"]]
    res["k_match"] = float(np.mean([a == b for a, b in km]))
    return res


def summarize(res: dict) -> dict:
    """Feasibility rates, and mean selected costs over the responses where
    both compared samplers found a feasible sample (the cost of an
    infeasible response is its violation, a different quantity).  The gap
    is relative to |mean plain cost|, since costs can be negative."""
    fp, fe, fl = (res[k].astype(bool) for k in ("feas_plain", "feas_plain_eq", "feas_learned"))
    out = dict(n_responses=int(fp.size), feasible_plain=float(fp.mean()), feasible_plain_eq=float(fe.mean()),
               feasible_learned=float(fl.mean()), k_match=res["k_match"])
    if "e2e_plain" in res:
        # end to end: the ego's final trajectory of each planner, in its own plan
        gp, gl = res["e2e_feas_plain"].astype(bool), res["e2e_feas_learned"].astype(bool)
        both = gp & gl
        out.update(e2e_plans=int(gp.size), e2e_feasible_plain=float(gp.mean()), e2e_feasible_learned=float(gl.mean()))
        if both.any():
            mp, ml = float(res["e2e_plain"][both].mean()), float(res["e2e_learned"][both].mean())
            out.update(e2e_mean_cost_plain=mp, e2e_mean_cost_learned=ml, e2e_cost_gap_abs=ml - mp,
                       e2e_cost_gap=(ml - mp) / abs(mp))
    for name, f2, c2 in (("learned", fl, res["learned"]), ("plain_eq", fe, res["plain_eq"])):
        both = fp & f2
        mp = float(res["plain"][both].mean()) if both.any() else float("nan")
        m2 = float(c2[both].mean()) if both.any() else float("nan")
        out[f"n_both_feasible_{name}"] = int(both.sum())
        out[f"mean_cost_plain_vs_{name}"] = mp
        out[f"mean_cost_{name}"] = m2
        out[f"gap_{name}"] = (m2 - mp) / abs(mp) if both.any() else float("nan")
        nb = ~fp & ~f2
        out[f"mean_violation_plain_vs_{name}"] = float(res["plain"][nb].mean()) if nb.any() else float("nan")
        out[f"mean_violation_{name}"] = float(c2[nb].mean()) if nb.any() else float("nan")
    return out


def plan_latency_ms(race: Race, params, K, L, mlp=None, K_prop=0, reps=50, warmup=5, seed=0):
    """Mean CUDA-event time of one plan at the race's current state."""
    T = race.T
    X, U0 = race.X, race.U.clone()
    U = U0.clone()
    out = None
    opts = launch_opts()
    for _ in range(warmup):
        U.copy_(U0)
        out = ibr_plan(race.track, params, X, U, race.vs, T, K, L, ego=race.sc.ego, seed=seed, opts=opts, out=out,
                       mlp=mlp, K_prop=K_prop)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        U.copy_(U0)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        out = ibr_plan(race.track, params, X, U, race.vs, T, K, L, ego=race.sc.ego, seed=seed, opts=opts, out=out,
                       mlp=mlp, K_prop=K_prop)
        e1.record(s)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.mean(ts))
