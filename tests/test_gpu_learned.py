"""GPU parity of the learned proposal: the BF16 tensor-core network
(forward, gradient, Adam) against the FP64 oracle on BF16-rounded tensors,
the mixed best response, and the learned plan (features, in-kernel
proposals and every best response teacher-forced against the oracle).

Tolerances: network outputs and gradients 2e-3 relative (Frobenius); an
Adam step 1e-6 absolute on the parameters; features 1e-4 relative to
max(1, |value|) with the opponent order checked up to 2 mm near-ties;
best responses by the rules of ``tests/parity_util.py``."""
import numpy as np
import pytest

import oracle as O
from oracle import features as OF
from oracle import mlp as OM
from paper_2607_25388_b300 import scenario as S
from tests.parity_util import STATE_RTOL, assert_rel_close, selection_ok

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NET_RTOL = 2e-3
ADAM_ATOL = 1e-6
FEAT_RTOL = 1e-4


def L():
    from paper_2607_25388_b300 import learned
    return learned


def P():
    from paper_2607_25388_b300 import planner
    return planner


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def frob(a, b):
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def feature_batch(B, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, 64)).astype(np.float32)
    x[:, 62] = rng.integers(1, 10, B) / 9.0
    x[:, 63] = rng.integers(0, 2, B)
    return x


@pytest.fixture(scope="module")
def net():
    return L().Mlp(60, seed=3)


def test_init_is_kaiming_uniform_with_zero_biases(net):
    w = net.get_params().astype(np.float64)
    dims = OM.dims_for(60)
    assert w.size == OM.param_count(dims) == net.n_params
    for (W, b), n_in in zip(OM.unpack(w, dims), dims[:-1]):
        bound = np.sqrt(6.0 / n_in)
        assert np.all(b == 0.0) and np.abs(W).max() <= bound
        assert abs(W.std() - bound / np.sqrt(3.0)) < 0.05 * bound     # uniform on [-bound, bound]


@pytest.mark.parametrize("B", [1, 10, 300])
def test_forward_matches_oracle(net, B):
    x = feature_batch(B, B)
    g = net.forward(dev(x)).cpu().numpy()
    o = OM.forward(net.get_params().astype(np.float64), x, OM.dims_for(60))[0]
    assert frob(g, o) <= NET_RTOL


def test_gradient_matches_oracle_per_layer():
    m = L().Mlp(60, seed=11)
    B, T = 777, 60
    x = feature_batch(B, 5)
    tgt = np.random.default_rng(6).standard_normal((B, 2 * T)).astype(np.float32)
    loss, grad = m.train_step(dev(x), dev(tgt), lr=1e-3, apply=False, want_grad=True)
    w = m.get_params().astype(np.float64)
    lo, go, _ = OM.loss_and_grad(w, x, tgt, T)
    assert abs(float(loss.item()) - lo) <= 1e-4 * abs(lo)
    dims = OM.dims_for(T)
    for l, ((gW, gb), (oW, ob)) in enumerate(zip(OM.unpack(grad.cpu().numpy().astype(np.float64), dims),
                                                 OM.unpack(go, dims))):
        assert frob(gW, oW) <= NET_RTOL, f"layer {l} W"
        assert frob(gb, ob) <= NET_RTOL, f"layer {l} b"
    # apply=False leaves the parameters and the step count untouched
    np.testing.assert_array_equal(m.get_params(), w.astype(np.float32))
    assert m.info()["step"] == 0


def test_adam_steps_match_oracle():
    m = L().Mlp(60, seed=12)
    B, T = 512, 60
    rng = np.random.default_rng(7)
    w = m.get_params().astype(np.float64)
    mo = np.zeros_like(w); vo = np.zeros_like(w)
    for step in (1, 2, 3):
        x = feature_batch(B, 100 + step)
        tgt = rng.standard_normal((B, 2 * T)).astype(np.float32)
        _, g = m.train_step(dev(x), dev(tgt), lr=1e-3, apply=True, want_grad=True)
        g = g.cpu().numpy().astype(np.float64)
        w, mo, vo = OM.adam(w, g, mo, vo, step, 1e-3)
        got = m.get_params().astype(np.float64)
        assert np.abs(got - w).max() <= ADAM_ATOL, f"step {step}"
        w = got      # carry the device's FP32 weights (the oracle step is exact up to FP32 rounding)
    assert m.info()["step"] == 3


def test_training_reduces_the_loss_on_a_learnable_target():
    """Targets that are a fixed function of the features: the loss drops."""
    m = L().Mlp(60, seed=13)
    B, T = 4096, 60
    x = feature_batch(B, 21)
    tgt = np.tanh(x[:, :1] * np.linspace(-1, 1, 2 * T)[None, :]).astype(np.float32)
    X, Y = dev(x), dev(tgt)
    first = float(m.train_step(X, Y, lr=1e-3)[0].item())
    for _ in range(200):
        last = m.train_step(X, Y, lr=1e-3)[0]
    assert float(last.item()) < first - 1.0


def test_proposal_matches_oracle(net):
    x = feature_batch(33, 9)
    p = S.params_fullscale()
    sa, sd = float(np.float32(p["sigma_a"])), float(np.float32(p["sigma_delta"]))
    un = np.float32(np.random.default_rng(34).normal(0.0, [1.0, 0.05], (33, 60, 2)))
    g = net.proposal(dev(x), sa, sd, dev(un)).cpu().numpy()
    out = OM.forward(net.get_params().astype(np.float64), x, OM.dims_for(60))[0]
    o = np.stack([OM.proposal(r, 60, sa, sd, u) for r, u in zip(out, un)])
    assert frob(g, o) <= NET_RTOL
    # without nominal controls the means are sigma x mu alone
    g0 = net.proposal(dev(x), sa, sd).cpu().numpy()
    assert frob(g0, np.stack([OM.proposal(r, 60, sa, sd) for r in out])) <= NET_RTOL


def test_save_load_round_trip(tmp_path, net):
    f = tmp_path / "net.bin"
    net.save(str(f))
    m = L().Mlp.load(str(f))
    np.testing.assert_array_equal(m.get_params(), net.get_params())
    x = dev(feature_batch(8, 1))
    np.testing.assert_array_equal(m.forward(x).cpu().numpy(), net.forward(x).cpu().numpy())


# ------------------------------------------------------------------ mixed best response
def _prop(u_nom, p, T, seed):
    rng = np.random.default_rng(seed)
    sa, sd = float(np.float32(p["sigma_a"])), float(np.float32(p["sigma_delta"]))
    pr = np.zeros((T, 4), np.float32)
    pr[:, 0] = u_nom[:, 0] + 2.0 * np.sin(np.arange(T) / 7.0)
    pr[:, 1] = u_nom[:, 1] + 0.02 * np.cos(np.arange(T) / 5.0)
    pr[:, 2] = sa * rng.uniform(0.3, 1.5, T)
    pr[:, 3] = sd * rng.uniform(0.3, 1.5, T)
    return pr


@pytest.mark.parametrize("case", ["oval", "two_car"])
def test_mixed_best_response_matches_oracle(case):
    p = S.params_fullscale()
    if case == "oval":
        sc = S.single_br_oval(K=2048, T=40)
        x0, u, opp, vs, game = sc.X0[0], sc.U0[0], sc.opp, 1.0, True
    else:
        sc = S.two_car_race(301, K=2048, T=50)
        x0, u, vs, game = sc.X0[0], sc.U0[0], 1.0, True
        opp = S.constant_velocity_prediction(sc.X0[1], sc.T, p["dt"])[None]
    T, K, Kp = sc.T, 2048, 900
    pr = _prop(u, p, T, 1)
    trk = P().Track.from_data(sc.track)
    g = P().best_response_mixed(trk, p, dev(x0), dev(u), vs, dev(opp), T, K, dev(pr), Kp, seed=4, agent=2, rnd=1,
                                game_on=game)
    torch.cuda.synchronize()
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    o = O.rollout_costs(p, ot, x0, u, vs, opp, T, K=K, seed=4, agent=2, rnd=1, game_on=game, prop=pr, K_prop=Kp)
    ko, anyf = O.select(o["cost"], o["feasible"], o["violation"])
    kg = int(g["k_star"].item())
    assert selection_ok(kg, ko, o["cost"], o["feasible"], o["violation"], o["margins"])
    assert bool(g["any_feasible"].item()) == bool(anyf)
    w = O.rollout_costs(p, ot, x0, u, vs, opp, T, k_list=[kg], seed=4, agent=2, rnd=1, game_on=game, prop=pr,
                        K_prop=Kp, want_states=True, want_controls=True)
    assert_rel_close(g["xi_star"].cpu().numpy(), w["states"][0], STATE_RTOL, "xi*")
    assert_rel_close(g["u_star"].cpu().numpy(), w["controls"][0], STATE_RTOL, "u*")
    want = w["cost"][0] if anyf else w["violation"][0]
    assert abs(float(g["cost"].item()) - want) <= 1e-4 * max(1.0, abs(want))


def test_mixed_with_zero_proposal_samples_equals_plain_best_response():
    p = S.params_fullscale()
    sc = S.two_car_race(302, K=4096, T=50)
    opp = dev(S.constant_velocity_prediction(sc.X0[1], sc.T, p["dt"])[None])
    trk = P().Track.from_data(sc.track)
    x0, u = dev(sc.X0[0]), dev(sc.U0[0])
    pr = dev(_prop(sc.U0[0], p, sc.T, 2))
    a = P().best_response(trk, p, x0, u, 1.0, opp, sc.T, 4096, seed=9, rnd=1)
    b = P().best_response_mixed(trk, p, x0, u, 1.0, opp, sc.T, 4096, pr, 0, seed=9, rnd=1)
    for k in ("k_star", "u_star", "xi_star", "any_feasible"):
        assert torch.equal(a[k], b[k]), k


# ------------------------------------------------------------------ learned plan
def _gpu_learned_plan(sc, p, K, Kp, Lr, seed, mlp, trk=None):
    trk = trk or P().Track.from_data(sc.track)
    U = dev(sc.U0.copy())
    out = P().ibr_plan(trk, p, dev(sc.X0), U, dev(sc.vref_scale), sc.T, K, Lr, ego=sc.ego, seed=seed,
                       want_hist=True, mlp=mlp, K_prop=Kp, want_features=True, want_prop=True)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["U"] = U.cpu().numpy()
    return res


def test_learned_plan_with_zero_proposal_samples_equals_plain_plan(net):
    sc = S.ten_car_race(203, K=2048, T=60, L=2)
    p = S.params_fullscale()
    trk = P().Track.from_data(sc.track)
    a = _gpu_learned_plan(sc, p, 2048, 0, 2, 5, net, trk)
    U = dev(sc.U0.copy())
    b = P().ibr_plan(trk, p, dev(sc.X0), U, dev(sc.vref_scale), sc.T, 2048, 2, ego=sc.ego, seed=5, want_hist=True)
    for k in ("xi", "k_star", "xi_hist", "u_hist"):
        np.testing.assert_array_equal(a[k], b[k].cpu().numpy())


def _check_features(sc, p, g, Lr, i, rnd, prev_xi):
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    n_v, T = sc.X0.shape[0], sc.T
    gains = np.array([OF.progress_gain(ot, prev_xi[j]) for j in range(n_v)])
    fo = OF.features(ot, sc.X0.astype(np.float64), gains, i, T, float(np.float32(p["dt"])), rnd > 0)
    fg = g["features"][rnd, i].astype(np.float64)
    # opponent slots: match rows; equal floors of 1000 |Delta s| may order differently only at near-ties
    keys = OF.order_keys(ot, sc.X0.astype(np.float64), i)
    head = np.r_[0:4, 62:64]
    assert_rel_close(fg[head], fo[head], FEAT_RTOL, f"features r{rnd} a{i}")
    # curvature ahead: a point within 2 mm of a waypoint may fall in either adjacent segment
    sj, Lap, lens = OF.arc_lengths(ot)
    s_i = O.frenet(ot, sc.X0[i:i + 1, :2].astype(np.float64))[0][0]
    xr = ot.xr
    for q, ahead in enumerate((0.0, 20.0, 40.0, 80.0)):
        sm = np.fmod(s_i + ahead, Lap)
        j = min(max(int(np.searchsorted(sj, sm, side="right")) - 1, 0), ot.N - 1)
        cands = {j}
        if sm - sj[j] < 2e-3:
            cands.add((j - 1) % ot.N)
        if sj[j + 1] - sm < 2e-3:
            cands.add((j + 1) % ot.N)
        kap = [100.0 * np.angle(np.exp(1j * (xr[(c + 1) % ot.N, 2] - xr[c, 2]))) / lens[c] for c in cands]
        assert min(abs(fg[4 + q] - k) / max(1.0, abs(k)) for k in kap) <= FEAT_RTOL, f"curvature r{rnd} a{i} q{q}"
    rows_g = fg[8:62].reshape(9, 6)
    rows_o = fo[8:62].reshape(9, 6)
    kv = np.sort(np.array(list(keys.values())))
    near_tie = kv.size > 1 and np.min(np.diff(np.floor(kv))) <= 2.0
    if not near_tie:
        assert_rel_close(rows_g, rows_o, FEAT_RTOL, f"opponent features r{rnd} a{i}")
    else:
        for r in rows_o:
            d = np.abs(rows_g - r[None]).max(axis=1) / np.maximum(1.0, np.abs(r).max())
            assert d.min() <= FEAT_RTOL, f"opponent row missing r{rnd} a{i}"


@pytest.mark.parametrize("case", ["two_car", "ten_car"])
def test_learned_plan_teacher_forced(net, case):
    p = S.params_fullscale()
    if case == "two_car":
        sc, K, Kp, Lr, n_check = S.two_car_race(311, K=1024, T=60, L=2), 1024, 512, 2, None
    else:
        sc, K, Kp, Lr, n_check = S.ten_car_race(212, K=512, T=60, L=2), 512, 256, 2, 14
    g = _gpu_learned_plan(sc, p, K, Kp, Lr, 6, net)
    assert g["status"][0] == 0
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    n_v, T = sc.X0.shape[0], sc.T
    lo = np.float32([p["a_min"], -p["delta_max"]])
    hi = np.float32([p["a_max"], p["delta_max"]])
    nominal = np.stack([O.rollout(p, sc.X0[i], np.clip(sc.U0[i], lo, hi), T) for i in range(n_v)])
    sa, sd = float(np.float32(p["sigma_a"])), float(np.float32(p["sigma_delta"]))
    w = net.get_params().astype(np.float64)
    checked = 0
    for rnd in range(Lr + 2):
        agents = [sc.ego] if rnd == Lr + 1 else range(n_v)
        for i in agents:
            if n_check is not None and checked >= n_check:
                return
            prev_xi = nominal if rnd == 0 else g["xi_hist"][rnd - 1]
            _check_features(sc, p, g, Lr, i, rnd, prev_xi)
            # the in-kernel network on the kernel's own features
            out = OM.forward(w, g["features"][rnd, i][None], OM.dims_for(T))[0][0]
            u_nom = sc.U0[i] if rnd == 0 else g["u_hist"][rnd - 1][i]
            po = OM.proposal(out, T, sa, sd, u_nom)
            pg = g["prop"][rnd, i]
            assert frob(pg, po) <= NET_RTOL, f"proposal r{rnd} a{i}"
            # the response itself, teacher-forced on the kernel's proposal
            opp = np.stack([prev_xi[j] for j in range(n_v) if j != i]) if n_v > 1 else None
            slot = (Lr + 1) * n_v if rnd == Lr + 1 else rnd * n_v + i
            kg = int(g["k_star"][slot])
            o = O.rollout_costs(p, ot, sc.X0[i], u_nom, sc.vref_scale[i], opp, T, K=K, seed=6, agent=i, rnd=rnd,
                                game_on=rnd > 0, prop=pg, K_prop=Kp)
            ko, _ = O.select(o["cost"], o["feasible"], o["violation"])
            assert selection_ok(kg, ko, o["cost"], o["feasible"], o["violation"], o["margins"]), \
                f"round {rnd} agent {i}: gpu k*={kg} oracle k*={ko}"
            ww = O.rollout_costs(p, ot, sc.X0[i], u_nom, sc.vref_scale[i], opp, T, k_list=[kg], seed=6, agent=i,
                                 rnd=rnd, game_on=rnd > 0, prop=pg, K_prop=Kp, want_states=True, want_controls=True)
            assert_rel_close(g["xi_hist"][rnd][i], ww["states"][0], STATE_RTOL, f"xi r{rnd} a{i}")
            assert_rel_close(g["u_hist"][rnd][i], ww["controls"][0], STATE_RTOL, f"U r{rnd} a{i}")
            checked += 1


@pytest.mark.parametrize("schedule", [0, 1, 2])
def test_learned_batch_equals_learned_single_plans(net, schedule):
    """Two ten-car races planned in one learned batch launch give exactly the
    learned single-race plans (proposal phase included), under the default,
    lock-step and queue schedules."""
    p = S.params_fullscale()
    races = [S.ten_car_race(221 + r, K=512, T=60, L=1) for r in range(2)]
    trk = P().Track.from_many([sc.track for sc in races])
    b = P().Batch(trk, [dict(track_id=r, n_v=10, T=60, ego=0, race_tag=r) for r in range(2)], K=512, L=1)
    X0 = dev(np.concatenate([sc.X0 for sc in races]))
    U = dev(np.concatenate([sc.U0.reshape(-1) for sc in races]))
    vs = dev(np.concatenate([sc.vref_scale for sc in races]))
    out = b.plan(p, X0, U, vs, seed=4, mlp=net, K_prop=200, opts=P().launch_opts(schedule=schedule))
    torch.cuda.synchronize()
    assert out["status"].item() == 0
    xi_all, ks_all = out["xi"].cpu().numpy(), out["k_star"].cpu().numpy()
    for r, sc in enumerate(races):
        Ur = dev(sc.U0.copy())
        single = P().ibr_plan(P().Track.from_data(sc.track), p, dev(sc.X0), Ur, dev(sc.vref_scale), 60, 512, 1, ego=0,
                              seed=4, race=r, mlp=net, K_prop=200)
        torch.cuda.synchronize()
        nx, nk = 10 * 61 * 4, 2 * 10 + 1
        np.testing.assert_array_equal(xi_all[r * nx:(r + 1) * nx], single["xi"].cpu().numpy().reshape(-1))
        np.testing.assert_array_equal(ks_all[r * nk:(r + 1) * nk], single["k_star"].cpu().numpy())


@pytest.mark.parametrize("shape", [(128, 1, 0, 0), (128, 2, 1, 0), (256, 1, 2, 0), (0, 0, 0, 2), (128, 3, 0, 2),
                                   (256, 1, 2, 2)])
def test_learned_plan_is_identical_for_every_block_size(net, shape):
    """Features (incl. the zeroed slots of absent opponents), proposals and
    selections do not depend on the CTA size or the schedule."""
    p = S.params_fullscale()
    sc = S.two_car_race(331, K=1024, T=60, L=2)
    trk = P().Track.from_data(sc.track)

    def run(opts):
        U = dev(sc.U0.copy())
        out = P().ibr_plan(trk, p, dev(sc.X0), U, dev(sc.vref_scale), sc.T, 1024, 2, ego=sc.ego, seed=2,
                           want_hist=True, mlp=net, K_prop=300, want_features=True, want_prop=True, opts=opts)
        torch.cuda.synchronize()
        return {k: v.cpu().numpy() for k, v in out.items()}

    a = run(None)
    b = run(P().launch_opts(block=shape[0], samples_per_thread=shape[1], ctas_per_sm=shape[2], schedule=shape[3]))
    assert np.all(a["features"][:, :, 14:62] == 0.0)       # one opponent: slots 1..8 are zero
    for k in ("features", "prop", "xi", "k_star", "u_hist"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
