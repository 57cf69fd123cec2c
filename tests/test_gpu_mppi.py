"""GPU parity of the GA-IBR-MPPI planning call (Sec. IV-A, second ablation;
sgtp_ibr_plan_mppi / sgtp_batch_plan_mppi) against the FP64 oracle.

Tolerance of the path-integral mean.  U_new = sum_k w_k u_k / sum_k w_k with
w_k = exp(-(c_k - c_min)/lambda).  A cost error dc_k changes log w_k by
eps_k = -(dc_k - dc_min)/lambda, and to first order
    |dU_tau| <= sum_k (w_k / W) |eps_k - eps_bar| |u_k,tau - U_tau|
             <= 2 max_k |eps_k| max_k |u_k,tau - U_tau|.
The test measures max_k |dc_k| for the same inputs through the C ABI's
per-candidate path (the plan kernel runs the same candidate code), takes
twice that bound, and adds the float32 rounding of the sums (the tile,
group and rescale sums over K samples: K x 2^-24 relative, written as
1e-4 of the controls' magnitude).  Trajectories: the GPU's xi is the
rollout of its own U_new, compared with the oracle's rollout of the same
controls at the state tolerance.  The reported lowest-cost sample must
match unless the two candidates' oracle costs differ by less than
SELECT_RTOL."""
import numpy as np
import pytest

import oracle as O
from paper_2607_25388_b300 import scenario as S
from tests.parity_util import SELECT_RTOL, STATE_RTOL, assert_rel_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def planner():
    from paper_2607_25388_b300 import planner as P
    return P


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def gpu_plan(sc, params, K, L, seed, lam, race=0, opts=None, sgtp=False):
    P = planner()
    trk = P.Track.from_data(sc.track)
    U = dev(sc.U0.copy())
    out = P.ibr_plan(trk, params, dev(sc.X0), U, dev(sc.vref_scale), sc.T, K, L, ego=sc.ego, seed=seed, race=race,
                     want_hist=True, opts=opts, mppi_lambda=None if sgtp else lam)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["U"] = U.cpu().numpy()
    return res


def _race(n_v, T, K, L, seed):
    return S.grid_race(S.fourier_track(seed, n_points=1200), n_v, T, K, L, seed + 1)


def test_zero_temperature_equals_sgtp_when_every_sample_is_feasible():
    """lambda -> 0 puts all weight on the lowest-cost sample; with every
    sample feasible that is SGTP's selection, and the whole plan must agree
    bit for bit (same controls, re-rolled the same way)."""
    sc = S.ten_car_race(203, K=2048, T=60, L=2)
    p = dict(S.params_fullscale(), m_bd=-1e9, d_col=-1e9)
    a = gpu_plan(sc, p, 2048, 2, seed=5, lam=None, sgtp=True)
    b = gpu_plan(sc, p, 2048, 2, seed=5, lam=1e-30)
    assert a["status"][0] == 0 and b["status"][0] == 0
    for k in ("k_star", "U", "xi", "xi_hist", "u_hist"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def check_mppi_response(sc, params, g, K, L, seed, lam, race, rnd, i, trk, ot, nominal):
    """Recompute response (rnd, i) of a GPU GA-IBR-MPPI plan with the oracle
    from the GPU's own inputs and compare (tolerance in the module doc)."""
    P = planner()
    n_v, T = sc.X0.shape[0], sc.T
    prev_xi = nominal if rnd == 0 else g["xi_hist"][rnd - 1]
    u_nom = sc.U0[i] if rnd == 0 else g["u_hist"][rnd - 1][i]
    opp = np.stack([prev_xi[j] for j in range(n_v) if j != i]) if n_v > 1 else None
    slot = (L + 1) * n_v if rnd == L + 1 else rnd * n_v + i
    what = f"round {rnd} agent {i}"
    o = O.best_response_mppi(params, ot, sc.X0[i], u_nom, sc.vref_scale[i], opp, T, K, lam, seed=seed, race=race,
                             agent=i, rnd=rnd, game_on=rnd > 0, want_costs=True)
    smp = O.rollout_costs(params, ot, sc.X0[i], u_nom, sc.vref_scale[i], opp, T, K=K, seed=seed, race=race,
                          agent=i, rnd=rnd, game_on=rnd > 0, want_controls=True)
    gc = P.rollout_costs(trk, params, dev(np.float32(sc.X0[i])), dev(np.float32(u_nom)), sc.vref_scale[i],
                         None if opp is None else dev(np.float32(opp)), T, K, seed=seed, race=race, agent=i,
                         rnd=rnd, game_on=rnd > 0)["cost"].cpu().numpy().astype(np.float64)
    c = o["costs"]
    dc = float(np.abs(gc - c).max())
    eps = dc / lam
    spread = np.abs(smp["controls"] - o["u_new"][None]).max(axis=0)           # (T, 2)
    tol = 2.0 * 2.0 * eps * spread + 1e-4 * np.maximum(1.0, np.abs(smp["controls"]).max(axis=0))
    err = np.abs(g["u_hist"][rnd][i] - o["u_new"])
    assert (err <= tol).all(), f"{what}: U error {err.max():.3e} above bound (dc {dc:.3e})"
    # the trajectory is the rollout of the GPU's own U_new
    assert_rel_close(g["xi_hist"][rnd][i], O.rollout(params, sc.X0[i], g["u_hist"][rnd][i], T), STATE_RTOL,
                     f"{what} xi")
    kg, ko = int(g["k_star"][slot]), o["k_min"]
    assert kg == ko or abs(c[kg] - c[ko]) <= SELECT_RTOL * max(1.0, abs(c[ko])), \
        f"{what}: lowest-cost sample gpu {kg} oracle {ko}"


def nominal_predictions(sc, params):
    lo = np.float32([params["a_min"], -params["delta_max"]])
    hi = np.float32([params["a_max"], params["delta_max"]])
    return np.stack([O.rollout(params, sc.X0[i], np.clip(sc.U0[i], lo, hi), sc.T) for i in range(sc.X0.shape[0])])


def teacher_forced_mppi(sc, params, g, K, L, seed, lam, race=0):
    """Recompute every response with the oracle from the GPU's own inputs."""
    P = planner()
    trk = P.Track.from_data(sc.track)
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    nominal = nominal_predictions(sc, params)
    for rnd in range(L + 2):
        for i in ([sc.ego] if rnd == L + 1 else range(sc.X0.shape[0])):
            check_mppi_response(sc, params, g, K, L, seed, lam, race, rnd, i, trk, ot, nominal)


@pytest.mark.parametrize("n_v,T,K,L,lam,seed", [
    (3, 30, 600, 2, 2.0e4, 713),      # three tiles, the last one ragged
    (2, 41, 257, 1, 3.0e3, 715),      # odd horizon (a half-used noise block), one sample in the last tile
    (4, 20, 1024, 1, 1.0e6, 717),     # a high temperature: close to the plain sample mean
])
def test_plan_teacher_forced_against_oracle(n_v, T, K, L, lam, seed):
    sc = _race(n_v, T, K, L, seed)
    p = S.params_fullscale()
    g = gpu_plan(sc, p, K, L, seed=seed, lam=lam, race=3)
    assert g["status"][0] == 0
    assert ((g["k_star"] >= 0) & (g["k_star"] < K)).all()
    teacher_forced_mppi(sc, p, g, K, L, seed, lam, race=3)
    np.testing.assert_array_equal(g["U"], g["u_hist"][L + 1])
    np.testing.assert_array_equal(g["xi"][sc.ego], g["xi_hist"][L + 1][sc.ego])


def test_launch_shape_invariance():
    P = planner()
    sc = S.ten_car_race(204, K=1500, T=40, L=1)
    p = S.params_fullscale()
    ref = gpu_plan(sc, p, 1500, 1, seed=2, lam=5e4)
    for block, spt, ctas in ((256, 1, 3), (256, 1, 1), (256, 1, 2), (128, 2, 0), (128, 0, 1), (0, 2, 0)):
        o = P.launch_opts(block=block, samples_per_thread=spt, ctas_per_sm=ctas)
        g = gpu_plan(sc, p, 1500, 1, seed=2, lam=5e4, opts=o)
        for k in ("k_star", "U", "xi", "xi_hist", "u_hist"):
            np.testing.assert_array_equal(g[k], ref[k], err_msg=f"{k} block {block} x {spt} ctas {ctas}")
    for bad in (dict(block=128, samples_per_thread=1), dict(samples_per_thread=3)):
        with pytest.raises(RuntimeError, match="SGTP_E_INVALID"):
            gpu_plan(sc, p, 1500, 1, seed=2, lam=5e4, opts=P.launch_opts(**bad))


def test_batch_equals_single_race_plans():
    P = planner()
    p = S.params_fullscale()
    K, L, lam = 700, 1, 3e4
    races = [_race(3, 25, K, L, 721), _race(5, 33, K, L, 723)]
    trk = P.Track.from_many([sc.track for sc in races])
    b = P.Batch(trk, [dict(track_id=r, n_v=sc.X0.shape[0], T=sc.T, ego=sc.ego, race_tag=r) for r, sc in
                      enumerate(races)], K=K, L=L)
    X0 = dev(np.concatenate([sc.X0 for sc in races]))
    U = dev(np.concatenate([sc.U0.reshape(-1) for sc in races]))
    vs = dev(np.concatenate([sc.vref_scale for sc in races]))
    out = b.plan(p, X0, U, vs, seed=9, mppi_lambda=lam)
    torch.cuda.synchronize()
    assert int(out["status"].cpu()[0]) == 0
    xi_all, ks_all, U_all = out["xi"].cpu().numpy(), out["k_star"].cpu().numpy(), U.cpu().numpy()
    xo = ko = uo = 0
    for r, sc in enumerate(races):
        n_v, T = sc.X0.shape[0], sc.T
        g = gpu_plan(sc, p, K, L, seed=9, lam=lam, race=r)
        nx, nk, nu = n_v * (T + 1) * 4, (L + 1) * n_v + 1, n_v * T * 2
        np.testing.assert_array_equal(xi_all[xo:xo + nx], g["xi"].reshape(-1))
        np.testing.assert_array_equal(ks_all[ko:ko + nk], g["k_star"])
        np.testing.assert_array_equal(U_all[uo:uo + nu], g["U"].reshape(-1))
        xo, ko, uo = xo + nx, ko + nk, uo + nu


def test_invalid_temperature_is_rejected():
    P = planner()
    sc = _race(2, 10, 64, 1, 725)
    p = S.params_fullscale()
    for lam in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(RuntimeError, match="lambda"):
            gpu_plan(sc, p, 64, 1, seed=1, lam=lam)
