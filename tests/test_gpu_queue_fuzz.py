"""The two schedules of a batch on fuzzed shapes: per-race progression
from the device queue and lock-step rounds must give the same plans bit
for bit (selection is an exact integer minimum and every sample is
computed by the same code), for batches of 1 to 7 races with 1 to 16
vehicles, horizons 1 to 128, ragged K, L = 0 to 3, random egos, over both
thread builds, and with the perturbed predictions and the GA-IBR-MPPI
update as well."""
import numpy as np
import pytest

from paper_2607_25388_b300 import scenario as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def P():
    from paper_2607_25388_b300 import planner
    return planner


def _batch(seed):
    rng = np.random.default_rng(seed)
    n_r = int(rng.integers(1, 8))
    K = int(rng.integers(40, 700))
    L = int(rng.integers(0, 4))
    races = []
    for r in range(n_r):
        n_v = int(rng.choice([1, 2, 3, 5, 9, 10, 16]))
        T = int(rng.choice([1, 2, 7, 30, 61, 80, 128]))
        sc = S.grid_race(S.fourier_track(7000 + 31 * seed + r, n_points=500), n_v, T, K, L, 900 + seed * 13 + r)
        sc.ego = int(rng.integers(0, n_v))
        sc.U0 = rng.normal(0.0, [0.8, 0.03], size=(n_v, T, 2)).astype(np.float32)
        races.append(sc)
    return races, K, L


@pytest.mark.parametrize("seed", range(6))
def test_queue_equals_lockstep_on_fuzzed_batches(seed):
    Pm = P()
    races, K, L = _batch(seed)
    trk = Pm.Track.from_many([sc.track for sc in races])
    b = Pm.Batch(trk, [dict(track_id=r, n_v=sc.X0.shape[0], T=sc.T, ego=sc.ego, race_tag=40 + r)
                       for r, sc in enumerate(races)], K=K, L=L)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    X0 = dev(np.concatenate([sc.X0 for sc in races]))
    U0 = np.concatenate([sc.U0.reshape(-1) for sc in races])
    vs = dev(np.concatenate([sc.vref_scale for sc in races]))
    p = S.params_fullscale()
    variants = (dict(), dict(pred_sigma=(0.4, 0.2)), dict(mppi_lambda=2e4))
    for kw in variants:
        runs = []
        for o in (Pm.launch_opts(schedule=Pm.SCHEDULE_LOCKSTEP), Pm.launch_opts(schedule=Pm.SCHEDULE_QUEUE),
                  Pm.launch_opts(block=256, schedule=Pm.SCHEDULE_QUEUE),
                  Pm.launch_opts(block=128, schedule=Pm.SCHEDULE_QUEUE, ctas_per_sm=1)):
            U = dev(U0)
            out = b.plan(p, X0, U, vs, seed=seed, want_hist=True, opts=o, **kw)
            torch.cuda.synchronize()
            assert out["status"].item() == 0, (seed, kw)
            runs.append({k: v.cpu().numpy() for k, v in out.items()} | {"U": U.cpu().numpy()})
        for r in runs[1:]:
            for k in ("xi", "k_star", "U", "xi_hist", "u_hist"):
                np.testing.assert_array_equal(r[k], runs[0][k], err_msg=f"seed {seed} {kw} {k}")


@pytest.mark.parametrize("seed", range(3))
def test_learned_batches_are_identical_across_schedules_and_builds(seed):
    """The learned proposal's features, network and mixed sampling in fuzzed
    batches (horizon 60, the network's): proposals as lock-step phases or as
    queue items, on the 128- and 256-thread builds."""
    from paper_2607_25388_b300.learned import Mlp
    Pm = P()
    rng = np.random.default_rng(100 + seed)
    K, L = int(rng.integers(300, 900)), int(rng.integers(1, 3))
    races = []
    for r in range(int(rng.integers(2, 6))):
        n_v = int(rng.choice([2, 4, 9, 10, 16]))
        sc = S.grid_race(S.fourier_track(7500 + 17 * seed + r, n_points=500), n_v, 60, K, L, 950 + 7 * seed + r)
        sc.ego = int(rng.integers(0, n_v))
        sc.U0 = rng.normal(0.0, [0.8, 0.03], size=(n_v, 60, 2)).astype(np.float32)
        races.append(sc)
    trk = Pm.Track.from_many([sc.track for sc in races])
    b = Pm.Batch(trk, [dict(track_id=r, n_v=sc.X0.shape[0], T=60, ego=sc.ego, race_tag=70 + r)
                       for r, sc in enumerate(races)], K=K, L=L)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    X0 = dev(np.concatenate([sc.X0 for sc in races]))
    U0 = np.concatenate([sc.U0.reshape(-1) for sc in races])
    vs = dev(np.concatenate([sc.vref_scale for sc in races]))
    net = Mlp(60, seed=seed)
    runs = []
    for o in (Pm.launch_opts(block=256, schedule=Pm.SCHEDULE_LOCKSTEP), None,
              Pm.launch_opts(block=256, ctas_per_sm=2, schedule=Pm.SCHEDULE_QUEUE),
              Pm.launch_opts(block=128, samples_per_thread=3, schedule=Pm.SCHEDULE_LOCKSTEP)):
        U = dev(U0)
        out = b.plan(S.params_fullscale(), X0, U, vs, seed=seed, want_hist=True, opts=o, mlp=net, K_prop=K // 2)
        torch.cuda.synchronize()
        assert out["status"].item() == 0
        runs.append({k: v.cpu().numpy() for k, v in out.items()} | {"U": U.cpu().numpy()})
    for r in runs[1:]:
        for k in ("xi", "k_star", "U", "xi_hist", "u_hist"):
            np.testing.assert_array_equal(r[k], runs[0][k], err_msg=f"seed {seed} {k}")


def test_repeated_queue_launches_are_identical():
    """Under the queue schedule the CTA that runs an item changes from launch
    to launch; five launches of one batch (plain and GA-IBR-MPPI) must still
    give the same bits, so no reduction or hand-off depends on timing."""
    Pm = P()
    races, K, L = _batch(11)
    trk = Pm.Track.from_many([sc.track for sc in races])
    b = Pm.Batch(trk, [dict(track_id=r, n_v=sc.X0.shape[0], T=sc.T, ego=sc.ego, race_tag=r)
                       for r, sc in enumerate(races)], K=K, L=L)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    X0 = dev(np.concatenate([sc.X0 for sc in races]))
    U0 = np.concatenate([sc.U0.reshape(-1) for sc in races])
    vs = dev(np.concatenate([sc.vref_scale for sc in races]))
    for kw in (dict(), dict(mppi_lambda=5e3)):
        ref = None
        for _ in range(5):
            U = dev(U0)
            out = b.plan(S.params_fullscale(), X0, U, vs, seed=3, want_hist=True,
                         opts=Pm.launch_opts(schedule=Pm.SCHEDULE_QUEUE), **kw)
            torch.cuda.synchronize()
            got = {k: v.cpu().numpy() for k, v in out.items()} | {"U": U.cpu().numpy()}
            assert got["status"][0] == 0
            if ref is None:
                ref = got
            for k in ("xi", "k_star", "U", "xi_hist", "u_hist"):
                np.testing.assert_array_equal(got[k], ref[k], err_msg=f"{kw} {k}")
