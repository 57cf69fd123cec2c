"""GPU parity of the planning call with perturbed opponent predictions
(robustness study of Table II; sgtp_ibr_plan_perturbed /
sgtp_batch_plan_perturbed) against the FP64 oracle.

Every best response is recomputed by the oracle from the GPU's own inputs
(previous-round trajectories and warm-started controls), with the oracle's
own perturbation of each opponent prediction (orc_perturb_prediction, same
counters), under the rules of tests/parity_util.py: the selected sample
equal unless a near-tie or a near-threshold candidate, its trajectory and
controls to the state tolerance.  The oracle takes each predicted point's
nearest segment in double precision and the GPU in float; where they
differ (a point on the bisector of two segments) the displacement axes
differ by the angle between the segments (about 3 mrad), which moves the
point by under 1e-3 of sigma, far inside the cost tolerance."""
import numpy as np
import pytest

import oracle as O
from paper_2607_25388_b300 import scenario as S
from tests.parity_util import STATE_RTOL, assert_rel_close, selection_ok

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def planner():
    from paper_2607_25388_b300 import planner as P
    return P


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def gpu_plan(sc, params, K, L, seed, sigma, race=0, opts=None):
    P = planner()
    trk = P.Track.from_data(sc.track)
    U = dev(sc.U0.copy())
    out = P.ibr_plan(trk, params, dev(sc.X0), U, dev(sc.vref_scale), sc.T, K, L, ego=sc.ego, seed=seed, race=race,
                     want_hist=True, opts=opts, pred_sigma=sigma)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["U"] = U.cpu().numpy()
    return res


def _race(n_v, T, K, L, seed):
    return S.grid_race(S.fourier_track(seed, n_points=1200), n_v, T, K, L, seed + 1)


def test_zero_sigma_is_the_sgtp_plan_bit_for_bit():
    sc = S.ten_car_race(206, K=1024, T=50, L=2)
    p = S.params_fullscale()
    a = gpu_plan(sc, p, 1024, 2, seed=3, sigma=None)
    b = gpu_plan(sc, p, 1024, 2, seed=3, sigma=(0.0, 0.0))
    for k in ("k_star", "U", "xi", "xi_hist", "u_hist", "status"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("n_v,T,K,L,sigma,seed", [
    (3, 40, 512, 2, (0.4, 0.2), 741),       # the severe setting at full scale
    (4, 33, 300, 1, (1.5, 1.0), 743),       # large noise, ragged K, odd T
])
def test_perturbed_plan_teacher_forced(n_v, T, K, L, sigma, seed):
    sc = _race(n_v, T, K, L, seed)
    p = S.params_fullscale()
    race = 2
    g = gpu_plan(sc, p, K, L, seed=seed, sigma=sigma, race=race)
    assert g["status"][0] == 0
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    n_tail = O.tail_count(p["mu_tail"], T)
    lo = np.float32([p["a_min"], -p["delta_max"]])
    hi = np.float32([p["a_max"], p["delta_max"]])
    nominal = np.stack([O.rollout(p, sc.X0[i], np.clip(sc.U0[i], lo, hi), T) for i in range(n_v)])
    for rnd in range(L + 2):
        agents = [sc.ego] if rnd == L + 1 else range(n_v)
        for i in agents:
            prev = nominal if rnd == 0 else g["xi_hist"][rnd - 1]
            u_nom = sc.U0[i] if rnd == 0 else g["u_hist"][rnd - 1][i]
            others = [j for j in range(n_v) if j != i]
            opp = np.stack([prev[j] for j in others])
            pert = [O.perturb_prediction(ot, prev[j], T, seed, race, i, rnd, j, sigma[0], sigma[1], n_tail)
                    for j in others]
            opp_pos = np.stack([q[0] for q in pert])
            delta = np.stack([q[1] for q in pert])
            o = O.rollout_costs_perturbed(p, ot, sc.X0[i], u_nom, sc.vref_scale[i], opp, opp_pos, delta, T, K=K,
                                          seed=seed, race=race, agent=i, rnd=rnd, game_on=rnd > 0)
            ko, _ = O.select(o["cost"], o["feasible"], o["violation"])
            slot = (L + 1) * n_v if rnd == L + 1 else rnd * n_v + i
            kg = int(g["k_star"][slot])
            what = f"round {rnd} agent {i}"
            assert selection_ok(kg, ko, o["cost"], o["feasible"], o["violation"], o["margins"]), \
                f"{what}: gpu k*={kg} oracle k*={ko}"
            w = O.rollout_costs_perturbed(p, ot, sc.X0[i], u_nom, sc.vref_scale[i], opp, opp_pos, delta, T,
                                          k_list=[kg], seed=seed, race=race, agent=i, rnd=rnd, game_on=rnd > 0,
                                          want_states=True, want_controls=True)
            assert_rel_close(g["xi_hist"][rnd][i], w["states"][0], STATE_RTOL, what + " xi")
            assert_rel_close(g["u_hist"][rnd][i], w["controls"][0], STATE_RTOL, what + " U")


def test_perturbation_changes_the_plan_and_is_shape_invariant():
    P = planner()
    sc = S.ten_car_race(207, K=1500, T=40, L=1)
    p = S.params_fullscale()
    plain = gpu_plan(sc, p, 1500, 1, seed=6, sigma=None)
    ref = gpu_plan(sc, p, 1500, 1, seed=6, sigma=(0.4, 0.2))
    assert not np.array_equal(plain["k_star"], ref["k_star"])
    for block, spt, ctas in ((128, 3, 0), (128, 1, 2), (256, 1, 1)):
        o = P.launch_opts(block=block, samples_per_thread=spt, ctas_per_sm=ctas)
        g = gpu_plan(sc, p, 1500, 1, seed=6, sigma=(0.4, 0.2), opts=o)
        for k in ("k_star", "U", "xi", "xi_hist", "u_hist"):
            np.testing.assert_array_equal(g[k], ref[k], err_msg=f"{k} block {block}")


def test_batch_equals_single_race_plans():
    P = planner()
    p = S.params_fullscale()
    K, L, sigma = 600, 1, (0.4, 0.2)
    races = [_race(3, 25, K, L, 745), _race(4, 31, K, L, 747)]
    trk = P.Track.from_many([sc.track for sc in races])
    b = P.Batch(trk, [dict(track_id=r, n_v=sc.X0.shape[0], T=sc.T, ego=sc.ego, race_tag=r) for r, sc in
                      enumerate(races)], K=K, L=L)
    X0 = dev(np.concatenate([sc.X0 for sc in races]))
    U = dev(np.concatenate([sc.U0.reshape(-1) for sc in races]))
    vs = dev(np.concatenate([sc.vref_scale for sc in races]))
    out = b.plan(p, X0, U, vs, seed=8, pred_sigma=sigma)
    torch.cuda.synchronize()
    assert int(out["status"].cpu()[0]) == 0
    xi_all, ks_all = out["xi"].cpu().numpy(), out["k_star"].cpu().numpy()
    xo = ko = 0
    for r, sc in enumerate(races):
        n_v, T = sc.X0.shape[0], sc.T
        g = gpu_plan(sc, p, K, L, seed=8, sigma=sigma, race=r)
        nx, nk = n_v * (T + 1) * 4, (L + 1) * n_v + 1
        np.testing.assert_array_equal(xi_all[xo:xo + nx], g["xi"].reshape(-1))
        np.testing.assert_array_equal(ks_all[ko:ko + nk], g["k_star"])
        xo, ko = xo + nx, ko + nk


def test_invalid_sigma_is_rejected():
    sc = _race(2, 10, 64, 1, 749)
    p = S.params_fullscale()
    for sigma in ((-0.1, 0.1), (0.1, float("nan")), (float("inf"), 0.0)):
        with pytest.raises(RuntimeError, match="sigma"):
            gpu_plan(sc, p, 64, 1, seed=1, sigma=sigma)
