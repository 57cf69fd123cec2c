"""GPU parity of the single best-response path (sgtp_rollout_costs,
sgtp_best_response) against the FP64 oracle, element by element, through the
C ABI.  Tolerances: see parity_util."""
import numpy as np
import pytest

import oracle as O
from paper_2607_25388_b300 import scenario as S
from tests.parity_util import (STATE_RTOL, assert_frenet_close, assert_rel_close, check_candidates,
                               selection_ok)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def planner():
    from paper_2607_25388_b300 import planner as P
    return P


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def run_both(td, params, x0, u_nom, vscale, opp, T, K, seed=7, race=3, agent=1, rnd=2, game_on=True,
             k_list=None, want_states=True):
    P = planner()
    trk = P.Track.from_data(td)
    g = P.rollout_costs(trk, params, dev(np.float32(x0)), dev(np.float32(u_nom)), vscale,
                        None if opp is None else dev(np.float32(opp)), T, K, seed=seed, race=race, agent=agent,
                        rnd=rnd, game_on=game_on, want_states=want_states, want_frenet=want_states,
                        want_controls=want_states)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in g.items()}
    ot = O.Track(td.xr, td.wl, td.wr)
    kl = np.arange(K) if k_list is None else np.asarray(k_list)
    o = O.rollout_costs(params, ot, x0, u_nom, vscale, opp, T, k_list=kl, seed=seed, race=race, agent=agent,
                        rnd=rnd, game_on=game_on, want_states=want_states, want_frenet=want_states,
                        want_controls=want_states)
    if k_list is not None:
        g = {k: v[kl] for k, v in g.items()}
    return g, o, trk


def test_track_length_matches_oracle():
    P = planner()
    for td in (S.oval_track(), S.fourier_track(100)):
        info = P.Track.from_data(td).info()
        L = O.track_length(O.Track(td.xr, td.wl, td.wr))
        assert info["N"] == td.N
        assert abs(info["length"] - L) <= 1e-6 * L


def test_oval_single_response_all_candidates():
    """The 1-ego-1-opponent oval workload (K=1024, T=40): every candidate's
    states, Frenet coordinates, controls, cost, flag and violation."""
    sc = S.single_br_oval()
    p = S.params_fullscale()
    g, o, _ = run_both(sc.track, p, sc.X0[0], sc.U0[0], 1.0, sc.opp, sc.T, sc.K, rnd=1)
    assert_rel_close(g["states"], o["states"], STATE_RTOL, "states")
    assert_frenet_close(g["frenet"], o["frenet"], o["states"], sc.track.xr)
    assert_rel_close(g["controls"], o["controls"], STATE_RTOL, "controls")
    nb = check_candidates(g, o, "oval")
    assert nb <= 0.01 * sc.K
    assert 0 < o["feasible"].sum() < sc.K        # the case exercises both branches


@pytest.mark.parametrize("seed,n_opp,T,K", [(101, 0, 1, 33), (102, 1, 2, 64), (103, 3, 7, 257), (104, 9, 33, 300),
                                            (105, 15, 50, 129), (106, 2, 128, 77)])
def test_fuzzed_small_problems(seed, n_opp, T, K):
    """Random Fourier tracks, random agents and opponents, ragged K and odd
    T (one half-used noise block), up to 15 opponents and the maximum T."""
    rng = np.random.default_rng(seed)
    td = S.fourier_track(seed, n_points=int(rng.integers(300, 2500)))
    p = S.params_fullscale()
    L = S.track_length(td)
    s0 = rng.uniform(0, L)
    x, y, psi = S.pose_at(td, s0, rng.uniform(-3, 3))
    x0 = np.float32([x, y, psi, rng.uniform(20, 60)])
    u_nom = np.float32(np.stack([rng.normal(0, 1, T), rng.normal(0, 0.02, T)], 1))
    opp = []
    for j in range(n_opp):
        ox, oy, op = S.pose_at(td, s0 + rng.uniform(-30, 30), rng.uniform(-4, 4))
        opp.append(S.constant_velocity_prediction([ox, oy, op, rng.uniform(20, 60)], T, p["dt"]))
    opp = np.stack(opp) if opp else None
    g, o, _ = run_both(td, p, x0, u_nom, float(np.float32(rng.uniform(0.8, 1.0))), opp, T, K, seed=seed,
                       agent=int(rng.integers(0, 9)), rnd=int(rng.integers(0, 6)), game_on=bool(seed % 2))
    assert_rel_close(g["states"], o["states"], STATE_RTOL, "states")
    assert_frenet_close(g["frenet"], o["frenet"], o["states"], td.xr)
    check_candidates(g, o, f"fuzz{seed}")


def test_zero_noise_makes_every_sample_the_nominal():
    sc = S.single_br_oval(K=300, T=40)
    p = S.params_fullscale()
    p.update(sigma_a=0.0, sigma_delta=0.0)
    P = planner()
    trk = P.Track.from_data(sc.track)
    u = np.float32(np.stack([np.linspace(-3, 3, 40), np.linspace(-0.1, 0.1, 40)], 1))
    g = P.rollout_costs(trk, p, dev(sc.X0[0]), dev(u), 1.0, dev(sc.opp), 40, 300, want_states=True)
    st = g["states"].cpu().numpy()
    assert (st == st[0]).all() and (g["cost"].cpu().numpy() == g["cost"][0].item()).all()
    br = P.best_response(trk, p, dev(sc.X0[0]), dev(u), 1.0, dev(sc.opp), 40, 300)
    assert br["k_star"].item() == 0
    nominal = O.rollout(p, sc.X0[0], u, 40)
    assert_rel_close(st[0], nominal, STATE_RTOL, "nominal")


def test_best_response_selection_and_winner_reroll():
    sc = S.single_br_oval()
    p = S.params_fullscale()
    P = planner()
    trk = P.Track.from_data(sc.track)
    x0, u0, opp = dev(sc.X0[0]), dev(sc.U0[0]), dev(sc.opp)
    br = P.best_response(trk, p, x0, u0, 1.0, opp, sc.T, sc.K, seed=7, race=3, agent=1, rnd=2)
    rc = P.rollout_costs(trk, p, x0, u0, 1.0, opp, sc.T, sc.K, seed=7, race=3, agent=1, rnd=2, want_states=True,
                         want_controls=True)
    torch.cuda.synchronize()
    k = br["k_star"].item()
    # the re-rolled winner is bit-identical to the evaluated candidate
    assert torch.equal(br["xi_star"], rc["states"][k])
    assert torch.equal(br["u_star"], rc["controls"][k])
    # GPU selection = minimum of its own per-candidate keys
    cost, feas, viol = rc["cost"].cpu().numpy(), rc["feasible"].cpu().numpy(), rc["violation"].cpu().numpy()
    order = sorted(range(sc.K), key=lambda i: (0 if feas[i] else 1, cost[i] if feas[i] else viol[i], i))
    assert k == order[0]
    assert br["any_feasible"].item() == int(feas.any())
    # against the oracle's selection
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    o = O.rollout_costs(p, ot, sc.X0[0], sc.U0[0], 1.0, sc.opp, sc.T, K=sc.K, seed=7, race=3, agent=1, rnd=2)
    ko, _ = O.select(o["cost"], o["feasible"], o["violation"])
    assert selection_ok(k, ko, o["cost"], o["feasible"], o["violation"], o["margins"])


def test_fallback_when_no_sample_is_feasible():
    """Ego starts outside the boundary margin: all candidates infeasible,
    the least violation is selected (Sec. III-B)."""
    td = S.oval_track()
    p = S.params_fullscale()
    x, y, psi = S.pose_at(td, 50.0, 4.7)
    x0 = np.float32([x, y, psi, 20.0])
    P = planner()
    trk = P.Track.from_data(td)
    T, K = 20, 512
    br = P.best_response(trk, p, dev(x0), dev(np.zeros((T, 2), np.float32)), 1.0, None, T, K)
    ot = O.Track(td.xr, td.wl, td.wr)
    o = O.rollout_costs(p, ot, x0, np.zeros((T, 2)), 1.0, None, T, K=K)
    assert not o["feasible"].any() and br["any_feasible"].item() == 0
    ko, _ = O.select(o["cost"], o["feasible"], o["violation"])
    assert selection_ok(br["k_star"].item(), ko, o["cost"], o["feasible"], o["violation"], o["margins"])


def test_full_size_ten_car_response_on_sampled_candidates():
    """A 10-car, K=16384, T=60 best response (9 opponents) in the launch
    configuration the plan uses; the oracle computes 192 sampled candidates."""
    sc = S.ten_car_race(200)
    p = S.params_fullscale()
    T, K = sc.T, sc.K
    opp = np.stack([S.constant_velocity_prediction(sc.X0[j], T, p["dt"]) for j in range(1, 10)])
    kl = np.unique(np.concatenate([np.arange(0, 64), np.random.default_rng(0).integers(0, K, 128), [K - 1]]))
    g, o, _ = run_both(sc.track, p, sc.X0[0], sc.U0[0], 1.0, opp, T, K, k_list=kl, seed=11, agent=0, rnd=3)
    assert_rel_close(g["states"], o["states"], STATE_RTOL, "states")
    check_candidates(g, o, "ten-car sample")


def test_vehicles_driving_against_the_track_direction():
    """Ego and opponents heading backwards along the track at 50 m/s: 150 m
    of travel (about 95 segments) against the polyline's direction.  The
    opponents' progress summaries and every candidate's Frenet coordinates
    must still be the globally nearest projections of Sec. II."""
    td = S.fourier_track(707)
    p = S.params_fullscale()
    T, K = 60, 200
    x, y, psi = S.pose_at(td, 900.0, 1.0)
    x0 = np.float32([x, y, psi + np.pi, 50.0])
    rng = np.random.default_rng(707)
    u_nom = np.float32(np.stack([rng.normal(0, 1, T), rng.normal(0, 0.01, T)], 1))
    opp = []
    for ds, d in ((-20.0, -3.0), (15.0, 2.5), (40.0, 0.0)):
        ox, oy, op = S.pose_at(td, 900.0 + ds, d)
        opp.append(S.constant_velocity_prediction([ox, oy, op + np.pi, 50.0], T, p["dt"]))
    g, o, _ = run_both(td, p, x0, u_nom, 1.0, np.stack(opp), T, K, seed=11, rnd=2, game_on=True)
    assert_rel_close(g["states"], o["states"], STATE_RTOL, "states")
    assert_frenet_close(g["frenet"], o["frenet"], o["states"], td.xr)
    check_candidates(g, o, "reversed")


@pytest.mark.parametrize("K", [1024, 20480])
def test_best_response_launch_shapes_select_the_oracle_argmin(K):
    """The standalone response runs its rollouts in 128-thread CTAs while
    K <= 128 x SMs and in 256-thread CTAs above (20480 > 128 x 148): in both
    shapes the selection equals the oracle's argmin over all K candidates
    (Eq. selection) and its sampled candidates match element by element."""
    P = planner()
    sc = S.single_br_oval(K=K)
    p = S.params_fullscale()
    trk = P.Track.from_data(sc.track)
    br = P.best_response(trk, p, dev(sc.X0[0]), dev(sc.U0[0]), 1.0, dev(sc.opp), sc.T, K, seed=5, rnd=1)
    torch.cuda.synchronize()
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    o = O.rollout_costs(p, ot, sc.X0[0], sc.U0[0], 1.0, sc.opp, sc.T, K=K, seed=5, rnd=1)
    ko, _ = O.select(o["cost"], o["feasible"], o["violation"])
    assert selection_ok(br["k_star"].item(), ko, o["cost"], o["feasible"], o["violation"], o["margins"])
    assert br["any_feasible"].item() == int(o["feasible"].any())
    kl = np.unique(np.concatenate([np.arange(0, 32), np.random.default_rng(K).integers(0, K, 96), [K - 1]]))
    g, oo, _ = run_both(sc.track, p, sc.X0[0], sc.U0[0], 1.0, sc.opp, sc.T, K, k_list=kl, seed=5, rnd=1,
                        want_states=False)
    check_candidates(g, oo, f"oval K={K}")
