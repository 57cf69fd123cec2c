"""Closed-loop trials of SGTP and its two ablations on synthetic tracks
(the evaluation of Sec. IV-B and IV-C: Wins, CFW, FPR, CSD, D, mean ego speed, MCS,
CT), one JSON line per planner.

    python -m paper_2607_25388_b300.closed_loop [--tracks 7 --starts 6 --seconds 50]

Every trial: one ego starting behind n_v - 1 opponents (reference speed
scale 0.9) on a seeded Fourier track; all vehicles run the same planner and
re-plan every control period (receding horizon); the trial ends at the
ego's first contact or at the time limit.  All trials of a planner run
together: each control period is one batched planning call and one
simulation step.  Planners: SGTP, SGTP without the game-aware cost
(w_game = 0, the paper's first ablation), GA-IBR-MPPI (the second), and
SGTP with perturbed opponent predictions (Table II: mild and severe noise,
the paper's (0.03, 0.015) and (0.08, 0.04) at 1/10 scale, x5 here).
The paper's MapZoo tracks, its simulator and its 1/10-scale parameters are
replaced by synthetic full-scale tracks and the planner's own bicycle model.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import scenario as S
from . import sim as SM


def run_variant(name, scs, params, K, L, sp, lam=None, pred_sigma=None):
    tr = SM.Trials(scs, params, K, L, sp, mppi_lambda=lam, pred_sigma=pred_sigma)
    tr.reset()
    # warm-up of the launch path, then the timed trial set from a fresh reset
    tr.plan()
    torch.cuda.synchronize()
    tr.reset()
    t0 = time.perf_counter()
    times = tr.run()
    wall = time.perf_counter() - t0
    res = tr.results()
    m = SM.trial_metrics(res, dt=params["dt"], limit_s=sp.max_steps * params["dt"])
    m.update(SM.ct_stats(times, len(scs)))
    steps = int(sum(r["steps"] for r in res))
    m.update(planner=name, periods=len(times), trial_steps=steps, wall_s=wall,
             sim_step_ms_mean=float(np.mean(tr.sim_times)) if tr.sim_times else 0.0,
             trial_steps_per_s=steps / wall if wall > 0 else 0.0)
    return m


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--tracks", type=int, default=7)
    ap.add_argument("--starts", type=int, default=6)
    ap.add_argument("--n-v", type=int, default=3)
    ap.add_argument("--seconds", type=float, default=50.0)
    ap.add_argument("--K", type=int, default=4096)
    ap.add_argument("--T", type=int, default=60)
    ap.add_argument("--L", type=int, default=2)
    ap.add_argument("--n-apply", type=int, default=1)
    ap.add_argument("--tracker", choices=["controls", "pure_pursuit"], default="pure_pursuit")
    ap.add_argument("--pp-preview", type=int, default=3, help="pure pursuit look-ahead in plan steps")
    ap.add_argument("--contact", type=float, default=2.5, help="vehicle contact distance (m)")
    ap.add_argument("--lam", type=float, default=1.0e4, help="GA-IBR-MPPI temperature")
    ap.add_argument("--variants", type=str, default="sgtp,no_game_cost,ga_ibr_mppi,sgtp_mild_noise,sgtp_severe_noise")
    args = ap.parse_args(argv)
    params = S.params_fullscale()
    scs = S.trial_set(args.tracks, args.starts, args.n_v, args.T, args.K, args.L)
    sp = SM.sim_params(n_apply=args.n_apply, max_steps=int(round(args.seconds / params["dt"])),
                       tracker=SM.TRACK_PURE_PURSUIT if args.tracker == "pure_pursuit" else SM.TRACK_CONTROLS,
                       pp_preview=args.pp_preview, contact_dist=args.contact)
    noise = {"sgtp_mild_noise": (0.15, 0.075), "sgtp_severe_noise": (0.40, 0.20)}
    for v in args.variants.split(","):
        p, lam, sig = params, None, None
        if v == "no_game_cost":
            p = dict(params, w_game=0.0)
        elif v == "ga_ibr_mppi":
            lam = args.lam
        elif v in noise:
            sig = noise[v]
        elif v != "sgtp":
            raise SystemExit(f"unknown planner {v}")
        m = run_variant(v, scs, p, args.K, args.L, sp, lam, sig)
        m.update(config=dict(trials=len(scs), n_v=args.n_v, seconds=args.seconds, K=args.K, T=args.T, L=args.L,
                             n_apply=args.n_apply, tracker=args.tracker, pp_preview=args.pp_preview,
                             contact=args.contact, lam=lam, pred_sigma=sig))
        print(json.dumps(m), flush=True)


if __name__ == "__main__":
    main()
