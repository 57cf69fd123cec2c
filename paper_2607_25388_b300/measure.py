"""Timings of every workload configuration on the GPU (one JSON line each).

    python -m paper_2607_25388_b300.measure [--reps 50]

1. single best response on the oval (K = 1024, T = 40, one opponent);
2. two-car plan (K = 8192, T = 50, L = 3);
3. ten-car plan (K = 16384, T = 60, L = 5), direct launch and CUDA-graph replay (median and p99 over at
   least 200 replays);
4. 256 independent races in one launch (n_v ~ U{2..10}, T ~ U{30..80}, K = 4096, L = 3), direct and graph;
5. plan latency of the ten-car race: plain K = 16384, plain K = 4096, and the learned sampler with
   2048 proposal + 2048 plain samples (network weights do not change the work);
5b. the same three samplers with 32 ten-car races per launch (per-plan time when the GPU is full);
6. the GA-IBR-MPPI ablation (path-integral update, lambda = 1e4) of the ten-car plan next to SGTP at the
   same K, direct launch;
7. planning time against the number of vehicles (n_v = 2..10 on one track), at the full-scale sampling
   and at the paper's sample counts (K = 128, H = 12, L = 2);
oracle: the FP64 CPU oracle on the host's cores for configurations 1 (in full), 2 and 3 (plans at
   reduced K, scaled linearly in K, and one full-K ten-car response for the record) and 4 (a subset of
   the races at reduced K), with the core count and CPU model.

Times are CUDA-event medians over `reps` calls after warm-up, inputs resident on the device.  FP32
fractions are against the FMA peak measured in the same run (roofline.measure_fma_peak).
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import roofline as R
from . import scenario as S
from .planner import Batch, PlanGraph, Track, best_response, br_workspace_bytes, ibr_plan, launch_opts


def _times_ms(fn, reps, warmup=5):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    ev = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        ev.append((a, b))
    torch.cuda.synchronize()
    return np.array([a.elapsed_time(b) for a, b in ev])


def _median_ms(fn, reps, warmup=5):
    return float(np.median(_times_ms(fn, reps, warmup)))


_PEAK = {}


def _peak():
    if "tf" not in _PEAK:
        _PEAK["tf"], _PEAK["form"] = R.measure_fma_peak()
        print(json.dumps(dict(config="measured FP32 FMA peak", tflops=_PEAK["tf"], form=_PEAK["form"],
                              nominal_max_clock=R.fp32_peak_tflops())), flush=True)
    return _PEAK["tf"]


def _line(config, ms, steps, flops, **extra):
    peak = _peak()
    d = dict(config=config, ms=ms, rollout_steps=steps, rollout_steps_per_s=steps / (ms / 1e3),
             tflops=flops / (ms / 1e3) / 1e12, fp32_frac=flops / (ms / 1e3) / 1e12 / peak)
    d.update(extra)
    print(json.dumps(d), flush=True)
    return d


def config1(reps):
    sc = S.single_br_oval()
    p = S.params_fullscale()
    trk = Track.from_data(sc.track)
    x0, u = torch.as_tensor(sc.X0[0]).cuda(), torch.as_tensor(sc.U0[0]).cuda()
    opp = torch.as_tensor(sc.opp).cuda()
    ms = _median_ms(lambda: best_response(trk, p, x0, u, 1.0, opp, sc.T, sc.K, seed=1), reps)
    res = _line("1: oval single best response, K=1024, T=40, 1 opponent", ms, sc.K * sc.T,
                R.flops_best_response(sc.K, sc.T, 1), launches_per_call=3)
    # the same three launches captured once in a CUDA graph (workspace and
    # outputs reused): the response's device time without launch gaps
    ws = torch.empty(br_workspace_bytes(1, sc.T), dtype=torch.uint8, device="cuda")
    out = best_response(trk, p, x0, u, 1.0, opp, sc.T, sc.K, seed=1, workspace=ws)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        best_response(trk, p, x0, u, 1.0, opp, sc.T, sc.K, seed=1, workspace=ws, out=out)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        best_response(trk, p, x0, u, 1.0, opp, sc.T, sc.K, seed=1, workspace=ws, out=out)
    ms_g = _median_ms(g.replay, reps)
    _line("1: oval single best response, K=1024, T=40, 1 opponent (CUDA graph replay)", ms_g, sc.K * sc.T,
          R.flops_best_response(sc.K, sc.T, 1), launches_per_call=3)
    return res


def _plan_lines(name, sc, reps, graph=True, min_graph_reps=0):
    p = S.params_fullscale()
    trk = Track.from_data(sc.track)
    n_v, T, K, L = sc.X0.shape[0], sc.T, sc.K, sc.L
    X0, vs = torch.as_tensor(sc.X0).cuda(), torch.as_tensor(sc.vref_scale).cuda()
    U0 = torch.as_tensor(sc.U0).cuda()
    U = U0.clone()
    out = {}
    holder = {}

    def direct():
        U.copy_(U0)
        holder["o"] = ibr_plan(trk, p, X0, U, vs, T, K, L, ego=sc.ego, seed=3, out=holder.get("o"))

    steps, flops = R.rollout_steps_plan(n_v, K, T, L), R.flops_plan(n_v, K, T, L)
    out["direct"] = _line(name + " (direct launch)", _median_ms(direct, reps), steps, flops)
    if graph:
        g = PlanGraph.capture_plan(trk, p, X0, U, vs, T, K, L, ego=sc.ego, seed=3)

        def replay():
            U.copy_(U0)
            g.launch()

        t = _times_ms(replay, max(reps, min_graph_reps), warmup=10)
        out["graph"] = _line(name + " (CUDA graph replay)", float(np.median(t)), steps, flops, plans=int(t.size),
                             p99_ms=float(np.percentile(t, 99)))
    return out


def config2(reps):
    return _plan_lines("2: two-car plan, K=8192, T=50, L=3", S.two_car_race(101), reps)


def config3(reps):
    # median and p99 of at least 200 graph replays after 10 warm-up plans
    return _plan_lines("3: ten-car plan, K=16384, T=60, L=5", S.ten_car_race(200), reps, min_graph_reps=200)


def config4(reps):
    p = S.params_fullscale()
    races = S.batched_races()
    K, L = races[0].K, races[0].L
    trk = Track.from_many([sc.track for sc in races])
    b = Batch(trk, [dict(track_id=r, n_v=sc.X0.shape[0], T=sc.T, ego=sc.ego, race_tag=r)
                    for r, sc in enumerate(races)], K=K, L=L)
    X0 = torch.as_tensor(np.concatenate([sc.X0 for sc in races])).cuda()
    U0 = torch.as_tensor(np.concatenate([sc.U0.reshape(-1) for sc in races])).cuda()
    vs = torch.as_tensor(np.concatenate([sc.vref_scale for sc in races])).cuda()
    U = U0.clone()
    ws = torch.empty(max(b.workspace_bytes, 256), dtype=torch.uint8, device="cuda")
    holder = {}

    def direct():
        U.copy_(U0)
        holder["o"] = b.plan(p, X0, U, vs, seed=5, workspace=ws, out=holder.get("o"))

    steps = sum(R.rollout_steps_plan(sc.X0.shape[0], K, sc.T, L) for sc in races)
    flops = sum(R.flops_plan(sc.X0.shape[0], K, sc.T, L) for sc in races)
    n_agents = int(sum(sc.X0.shape[0] for sc in races))
    res = {"direct": _line("4: 256 batched races, K=4096, L=3 (direct launch)", _median_ms(direct, reps), steps,
                           flops, races=len(races), agents=n_agents)}
    g = PlanGraph.capture_batch(b, p, X0, U, vs, seed=5)

    def replay():
        U.copy_(U0)
        g.launch()

    res["graph"] = _line("4: 256 batched races, K=4096, L=3 (CUDA graph replay)", _median_ms(replay, reps), steps,
                         flops, races=len(races), agents=n_agents)
    return res


def config5(reps):
    from .learned import Mlp
    p = S.params_fullscale()
    sc = S.ten_car_race(200)
    trk = Track.from_data(sc.track)
    n_v, T, L = 10, 60, 5
    X0, vs = torch.as_tensor(sc.X0).cuda(), torch.as_tensor(sc.vref_scale).cuda()
    U0 = torch.as_tensor(sc.U0).cuda()
    U = U0.clone()
    mlp = Mlp(T, seed=1)
    res = {}
    for name, K, net, kp in (("plain K=16384", 16384, None, 0), ("plain K=4096", 4096, None, 0),
                             ("learned 2048+2048", 4096, mlp, 2048)):
        holder = {}

        def run():
            U.copy_(U0)
            holder["o"] = ibr_plan(trk, p, X0, U, vs, T, K, L, ego=0, seed=3, out=holder.get("o"), mlp=net, K_prop=kp)

        res[name] = _line(f"5: ten-car plan latency, {name}", _median_ms(run, reps), R.rollout_steps_plan(n_v, K, T, L),
                          R.flops_plan(n_v, K, T, L))
    print(json.dumps(dict(config="5: latency ratio plain 16384 / learned 2048+2048",
                          ratio=res["plain K=16384"]["ms"] / res["learned 2048+2048"]["ms"])), flush=True)
    return res


def config5_batched(reps, n_races=32):
    """Per-plan time when many ten-car races share one launch (a serving
    setting): plain K=16384 vs learned 2048+2048 vs plain K=4096."""
    from .learned import Mlp
    p = S.params_fullscale()
    races = [S.ten_car_race(300 + r) for r in range(n_races)]
    trk = Track.from_many([sc.track for sc in races])
    X0 = torch.as_tensor(np.concatenate([sc.X0 for sc in races])).cuda()
    U0 = torch.as_tensor(np.concatenate([sc.U0.reshape(-1) for sc in races])).cuda()
    vs = torch.as_tensor(np.concatenate([sc.vref_scale for sc in races])).cuda()
    U = U0.clone()
    mlp = Mlp(60, seed=1)
    res = {}
    for name, K, net, kp in (("plain K=16384", 16384, None, 0), ("plain K=4096", 4096, None, 0),
                             ("learned 2048+2048", 4096, mlp, 2048)):
        b = Batch(trk, [dict(track_id=r, n_v=10, T=60, ego=0, race_tag=r) for r in range(n_races)], K=K, L=5)
        holder = {}

        def run():
            U.copy_(U0)
            holder["o"] = b.plan(p, X0, U, vs, seed=3, out=holder.get("o"), mlp=net, K_prop=kp)

        ms = _median_ms(run, max(5, reps // 5))
        res[name] = _line(f"5b: {n_races} ten-car races in one launch, {name} (ms per launch)", ms,
                          n_races * R.rollout_steps_plan(10, K, 60, 5), n_races * R.flops_plan(10, K, 60, 5),
                          ms_per_plan=ms / n_races)
    print(json.dumps(dict(config=f"5b: per-plan time ratio plain 16384 / learned 2048+2048 ({n_races} races per launch)",
                          ratio=res["plain K=16384"]["ms"] / res["learned 2048+2048"]["ms"])), flush=True)
    return res


def config6(reps, lam=1.0e4):
    """Ten-car plan (K = 16384, T = 60, L = 5): SGTP and GA-IBR-MPPI."""
    p = S.params_fullscale()
    sc = S.ten_car_race(200)
    trk = Track.from_data(sc.track)
    n_v, T, K, L = 10, 60, 16384, 5
    X0, vs = torch.as_tensor(sc.X0).cuda(), torch.as_tensor(sc.vref_scale).cuda()
    U0 = torch.as_tensor(sc.U0).cuda()
    U = U0.clone()
    res = {}
    for name, lam_i in (("SGTP", None), (f"GA-IBR-MPPI lambda={lam:g}", lam)):
        holder = {}

        def run():
            U.copy_(U0)
            holder["o"] = ibr_plan(trk, p, X0, U, vs, T, K, L, ego=0, seed=3, out=holder.get("o"), mppi_lambda=lam_i)

        res[name] = _line(f"6: ten-car plan, {name}", _median_ms(run, reps), R.rollout_steps_plan(n_v, K, T, L),
                          R.flops_plan(n_v, K, T, L))
    return res


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_line(config, seconds, steps, **extra):
    d = dict(config=config, oracle_s=seconds, rollout_steps=steps, oracle_rollout_steps_per_s=steps / seconds,
             cores=os.cpu_count(), cpu=_cpu_model())
    d.update(extra)
    print(json.dumps(d), flush=True)
    return d


def config7(reps):
    """Planning time against the number of vehicles (the scalability study of
    Sec. IV-G): grid starts of n_v = 2..10 cars on one Fourier track, at the
    full-scale sampling (K = 16384, T = 60, L = 5) and at the paper's sample
    counts (K = 128, H = 12, L = 2; the full-scale tracks and parameters)."""
    p = S.params_fullscale()
    track = S.fourier_track(200)
    trk = Track.from_data(track)
    Kp, Tp, Lp = S.PAPER_SAMPLES
    for K, T, L in ((16384, 60, 5), (Kp, Tp, Lp)):
        for n_v in (2, 3, 4, 6, 8, 10):
            sc = S.grid_race(track, n_v, T, K, L, 211)
            X0, vs = torch.as_tensor(sc.X0).cuda(), torch.as_tensor(sc.vref_scale).cuda()
            U0 = torch.as_tensor(sc.U0).cuda()
            U = U0.clone()
            holder = {}

            def direct():
                U.copy_(U0)
                holder["o"] = ibr_plan(trk, p, X0, U, vs, T, K, L, ego=sc.ego, seed=3, out=holder.get("o"))

            _line(f"7: planning time vs vehicles, n_v={n_v}, K={K}, T={T}, L={L}", _median_ms(direct, reps),
                  R.rollout_steps_plan(n_v, K, T, L), R.flops_plan(n_v, K, T, L), n_v=n_v)


def oracle(reps):
    """The FP64 oracle's rate on this host (all cores; the oracle's own
    thread pool over samples)."""
    import oracle as O
    p = S.params_fullscale()
    # 1: the oval best response in full
    sc = S.single_br_oval()
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    t0 = time.perf_counter()
    O.best_response(p, ot, sc.X0[0], sc.U0[0], 1.0, sc.opp, sc.T, sc.K, seed=1, rnd=1)
    _oracle_line("oracle 1: oval single best response, K=1024, T=40 (in full)", time.perf_counter() - t0,
                 sc.K * sc.T)
    # 2 and 3: whole plans at reduced K, scaled linearly to the configuration's K
    for name, sc, k_red in (("2: two-car plan, K=8192, T=50, L=3", S.two_car_race(100), 1024),
                            ("3: ten-car plan, K=16384, T=60, L=5", S.ten_car_race(200), 256)):
        ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
        n_v = sc.X0.shape[0]
        t0 = time.perf_counter()
        O.ibr_plan(p, ot, sc.X0, sc.U0, sc.vref_scale, sc.T, k_red, sc.L, sc.ego, seed=3)
        dt = time.perf_counter() - t0
        steps = R.rollout_steps_plan(n_v, k_red, sc.T, sc.L)
        _oracle_line(f"oracle {name} at K={k_red}", dt, steps,
                     plan_s_scaled_to_full_K=dt * sc.K / k_red)
    # 3: one full-K ten-car response for the record (round 1 against the nominal predictions)
    sc = S.ten_car_race(200)
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    lo = np.float32([p["a_min"], -p["delta_max"]]); hi = np.float32([p["a_max"], p["delta_max"]])
    nominal = np.stack([O.rollout(p, sc.X0[i], np.clip(sc.U0[i], lo, hi), sc.T) for i in range(10)])
    t0 = time.perf_counter()
    O.best_response(p, ot, sc.X0[0], sc.U0[0], sc.vref_scale[0], nominal[1:], sc.T, sc.K, seed=3, rnd=1)
    _oracle_line("oracle 3: one ten-car best response, K=16384, T=60, 9 opponents (in full)",
                 time.perf_counter() - t0, sc.K * sc.T)
    # 4: a subset of the 256 batched races at reduced K
    races = S.batched_races()[:4]
    k_red = 256
    t0 = time.perf_counter()
    steps = 0
    for r, sc in enumerate(races):
        ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
        O.ibr_plan(p, ot, sc.X0, sc.U0, sc.vref_scale, sc.T, k_red, sc.L, sc.ego, seed=5, race=r)
        steps += R.rollout_steps_plan(sc.X0.shape[0], k_red, sc.T, sc.L)
    _oracle_line(f"oracle 4: races 0-3 of the 256-race batch at K={k_red}", time.perf_counter() - t0, steps)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--reps", type=int, default=50)
    ap.add_argument("--configs", type=str, default="1,2,3,4,5,5b,6,7,oracle")
    args = ap.parse_args(argv)
    fns = {"1": config1, "2": config2, "3": config3, "4": config4, "5": config5, "5b": config5_batched,
           "6": config6, "7": config7, "oracle": oracle}
    for c in args.configs.split(","):
        fns[c.strip()](args.reps)


if __name__ == "__main__":
    main()
