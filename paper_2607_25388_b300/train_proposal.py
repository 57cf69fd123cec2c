"""Train the learned proposal on best responses of the plain planner and
compare it with the plain planner.

    python -m paper_2607_25388_b300.train_proposal --races 400 --plans 41 \\
        --epochs 30 --out proposal_T60.bin

Data: ten-car races (5 IBR rounds, K = 16384, T = 60) on seeded Fourier
tracks, advanced in closed loop between plans; every best response of every
plan gives one (features, selected controls) example.  Training: Adam on
the Gaussian NLL (batch 4096, lr 1e-3).  Evaluation on held-out track seeds:
per-response costs teacher-forced (learned 2048 + 2048 vs plain 16384 and
plain 4096 on identical inputs) and plan latency.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np
import torch

from . import learned as LR
from . import scenario as S


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--races", type=int, default=400, help="training races (track seeds 10000+)")
    ap.add_argument("--plans", type=int, default=41, help="closed-loop plans per training race")
    ap.add_argument("--advance", type=int, default=10, help="steps applied between plans")
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--cosine", action="store_true", help="cosine learning-rate decay to 0")
    ap.add_argument("--eval-seeds", type=str, default="200-209")
    ap.add_argument("--eval-states", type=int, default=4, help="closed-loop states per evaluation race")
    ap.add_argument("--k-prop", type=int, default=2048)
    ap.add_argument("--k-eq", type=int, default=4096)
    ap.add_argument("--out", type=str, default="", help="save the trained weights here")
    ap.add_argument("--load", type=str, default="", help="skip training: load weights")
    ap.add_argument("--quiet", action="store_true")
    args = ap.parse_args(argv)
    log = (lambda m: None) if args.quiet else (lambda m: print(m, file=sys.stderr, flush=True))
    params = S.params_fullscale()
    T, K, L = 60, 16384, 5
    rec = dict(advance=args.advance)
    if args.load:
        mlp = LR.Mlp.load(args.load)
        rec["weights"] = args.load
    else:
        rec.update(races=args.races, plans_per_race=args.plans, epochs=args.epochs, cosine=args.cosine)
        t0 = time.time()
        X, Y = LR.generate_dataset(range(10000, 10000 + args.races), args.plans, args.advance, K, T, L, params,
                                   log=log)
        torch.cuda.synchronize()
        rec["examples"] = int(X.shape[0])
        rec["datagen_s"] = time.time() - t0
        mlp = LR.Mlp(T, seed=1)
        t0 = time.time()
        losses = LR.train(mlp, X, Y, args.epochs, args.batch, args.lr, log=log, cosine=args.cosine)
        torch.cuda.synchronize()
        rec["train_s"] = time.time() - t0
        rec["loss_first_epoch"], rec["loss_last_epoch"] = losses[0], losses[-1]
        del X, Y
        if args.out:
            mlp.save(args.out)
    a, b = (int(v) for v in args.eval_seeds.split("-"))
    res = LR.compare(mlp, range(a, b + 1), args.eval_states, args.advance, K, args.k_eq, args.k_prop, T, L, params)
    rec["ab"] = LR.summarize(res)
    # plan latency at the first evaluation race's start
    race = LR.Race(S.ten_car_race(a, K=K, T=T, L=L))
    rec["plan_ms_plain"] = LR.plan_latency_ms(race, params, K, L)
    rec["plan_ms_plain_eq"] = LR.plan_latency_ms(race, params, args.k_eq, L)
    rec["plan_ms_learned"] = LR.plan_latency_ms(race, params, args.k_eq, L, mlp=mlp, K_prop=args.k_prop)
    rec["latency_ratio"] = rec["plan_ms_plain"] / rec["plan_ms_learned"]
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
