"""Pins of the oracle's learned-proposal pieces (network, loss, Adam,
features, proposal sampling) against what the mathematics fixes: finite
differences, closed forms, the round-to-nearest-even definition, geometry of
the oval track, and the plain sampler as a special case of the mixed one."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import features as OF
from oracle import mlp as OM
from paper_2607_25388_b300 import scenario as S


# ------------------------------------------------------------------ BF16 rounding
def test_bf16_round_to_nearest_even_on_exact_binary_values():
    one = 1.0
    cases = {
        one: one,
        one + 2.0 ** -8: one,                       # halfway, 1.0 is even -> down
        one + 3 * 2.0 ** -8: one + 2.0 ** -6,       # halfway, 1+2^-6 is even -> up
        one + 2.0 ** -8 + 2.0 ** -20: one + 2.0 ** -7,   # above halfway -> up
        -(one + 2.0 ** -9): -one,                   # below halfway -> toward |x| smaller
        1.5 * 2.0 ** 100: 1.5 * 2.0 ** 100,         # exactly representable
        0.0: 0.0,
    }
    for x, want in cases.items():
        assert OM.bf16_round(np.array([x]))[0] == want, x


def test_bf16_round_agrees_with_torch_conversion():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.uniform(-6, 6, 20000),
                        np.float32(1.0) + np.arange(-300, 300) * 2.0 ** -16])
    t = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(OM.bf16_round(x), t)


# ------------------------------------------------------------------ loss
def test_nll_closed_forms():
    T = 3
    tgt = np.array([[0.5, -1.0, 2.0, 0.0, 1.0, -0.5]])
    out = np.zeros((1, 4 * T))
    out[0, :2 * T] = tgt[0]                     # mu = target, logsig = 0
    loss, d = OM.nll(out, tgt, T)
    n = 2 * T
    assert loss == 0.0
    assert np.all(d[0, :n] == 0.0) and np.allclose(d[0, n:], 1.0 / n)
    # mu = 0, logsig = log 2 everywhere: 0.5 (t / 2)^2 + log 2 per element
    out = np.zeros((1, 4 * T)); out[0, n:] = math.log(2.0)
    loss, d = OM.nll(out, tgt, T)
    want = np.mean(0.5 * (tgt[0] / 2.0) ** 2 + math.log(2.0))
    assert abs(loss - want) < 1e-15
    assert np.allclose(d[0, :n], -(tgt[0] / 2.0) / 2.0 / n)
    assert np.allclose(d[0, n:], (1.0 - (tgt[0] / 2.0) ** 2) / n)
    # clamped logsig: value at the clamp, zero gradient
    out = np.zeros((1, 4 * T)); out[0, n:] = 3.0
    loss, d = OM.nll(out, np.zeros((1, n)), T)
    assert abs(loss - 2.0) < 1e-15 and np.all(d[0, n:] == 0.0)


# ------------------------------------------------------------------ gradient
def test_backward_matches_central_finite_differences_fp64():
    T = 2
    dims = [5, 7, 6, 4, 4 * T]
    rng = np.random.default_rng(1)
    w = rng.standard_normal(OM.param_count(dims)) * 0.5
    x = rng.standard_normal((9, dims[0]))
    tgt = rng.standard_normal((9, 2 * T))
    loss, g, _ = OM.loss_and_grad(w, x, tgt, T, dims, bf16=False)
    h = 1e-6
    fd = np.zeros_like(w)
    for k in range(w.size):
        wp = w.copy(); wp[k] += h
        wm = w.copy(); wm[k] -= h
        fd[k] = (OM.loss_and_grad(wp, x, tgt, T, dims, bf16=False)[0] -
                 OM.loss_and_grad(wm, x, tgt, T, dims, bf16=False)[0]) / (2 * h)
    scale = np.abs(fd).max()
    assert np.abs(g - fd).max() <= 1e-7 * scale + 1e-10
    # every parameter takes part (no dropped term): each layer's block is non-zero
    for W, b in OM.unpack(g, dims):
        assert np.abs(W).max() > 0 and np.abs(b).max() > 0


def test_bf16_network_is_close_to_fp64_network():
    T = 60
    dims = OM.dims_for(T)
    rng = np.random.default_rng(2)
    w = np.concatenate([np.concatenate([rng.uniform(-1, 1, (o, i)).ravel() * math.sqrt(6.0 / i), np.zeros(o)])
                        for i, o in zip(dims[:-1], dims[1:])])
    x = rng.standard_normal((16, 64))
    o64 = OM.forward(w, x, dims, bf16=False)[0]
    o16 = OM.forward(w, x, dims, bf16=True)[0]
    rel = np.linalg.norm(o16 - o64) / np.linalg.norm(o64)
    assert 1e-4 < rel < 3e-2     # rounding is applied, and stays at BF16's scale


# ------------------------------------------------------------------ Adam
def test_adam_first_steps_closed_form():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    w = np.array([1.0, 1.0, 1.0, 1.0])
    m = np.zeros(4); v = np.zeros(4)
    lr = 1e-3
    w1, m, v = OM.adam(w, g, m, v, 1, lr)
    # bias-corrected moments equal g and g^2 after the first step
    assert np.allclose(w1, w - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    w2, m, v = OM.adam(w1, g, m, v, 2, lr)
    assert np.allclose(w2, w1 - lr * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_proposal_units():
    T = 4
    row = np.concatenate([np.full(T, 2.0), np.full(T, -1.0), np.full(T, 0.0), np.full(T, -9.0)])
    P = OM.proposal(row, T, 1.0, 0.05)
    assert np.allclose(P[:, 0], 2.0) and np.allclose(P[:, 1], -0.05)
    assert np.allclose(P[:, 2], 1.0) and np.allclose(P[:, 3], 0.05 * math.exp(-5.0))
    # a residual around the nominal controls: mu = 0, logsig = 0 is the plain sampler N(U-bar, sigma^2)
    un = np.stack([np.linspace(-1, 1, T), np.linspace(0.1, -0.1, T)], axis=1)
    P = OM.proposal(np.zeros(4 * T), T, 1.0, 0.05, un)
    assert np.allclose(P[:, :2], un) and np.allclose(P[:, 2], 1.0) and np.allclose(P[:, 3], 0.05)
    P = OM.proposal(row, T, 1.0, 0.05, un)
    assert np.allclose(P[:, 0], un[:, 0] + 2.0) and np.allclose(P[:, 1], un[:, 1] - 0.05)


# ------------------------------------------------------------------ features
def _oval():
    td = S.oval_track()
    return td, O.Track(td.xr, td.wl, td.wr)


def test_features_closed_forms_on_the_oval():
    td, tr = _oval()
    T, dt = 60, 0.05
    # ego on the lower straight at s = 150, 1 m left, heading 0.1 rad
    X = np.array([[150.0, 1.0, 0.1, 30.0],
                  [170.0, -2.0, 0.0, 35.0],     # 20 m ahead
                  [140.0, 3.0, -0.2, 25.0],     # 10 m behind
                  [60.0, 0.0, 0.0, 40.0]])      # 90 m behind
    gains = np.array([0.0, 100.0, 70.0, 130.0])
    f = OF.features(tr, X, gains, 0, T, dt, True)
    assert abs(f[0] - 0.2) < 1e-9
    assert abs(f[1] - math.sin(0.1)) < 1e-6 and abs(f[2] - math.cos(0.1)) < 1e-6
    assert f[3] == 0.5
    # curvature: straight at s+0, s+20, s+40; semicircle (R = 50) at s+80
    assert np.all(np.abs(f[4:7]) < 1e-4)
    assert abs(f[7] - 100.0 / 50.0) < 2e-3
    # opponents by |Delta s|: 10 m behind, 20 m ahead, 90 m behind
    want = [[1, -10 / 40, 3 / 5, -5 / 10, -0.2 - 0.1, (70 - 30 * T * dt) / 40],
            [1, 20 / 40, -2 / 5, 5 / 10, -0.1, (100 - 30 * T * dt) / 40],
            [1, -90 / 40, 0.0, 10 / 10, -0.1, (130 - 30 * T * dt) / 40]]
    assert np.allclose(f[8:26].reshape(3, 6), want, atol=1e-9)
    assert np.all(f[26:62] == 0.0)
    assert abs(f[62] - 3 / 9) < 1e-15 and f[63] == 1.0
    assert OF.features(tr, X, gains, 0, T, dt, False)[63] == 0.0


def test_features_progress_wraps_across_the_start_line():
    td, tr = _oval()
    L = OF.arc_lengths(tr)[1]
    # ego 5 m of arc before the start line (end of the left semicircle), the
    # opponent 5 m past it: Delta s = +10 across the wrap, -10 seen from it
    X = np.zeros((2, 4))
    X[:, 3] = 30.0
    X[0, :2] = [-50.0 * math.sin(5.0 / 50.0), 50.0 - 50.0 * math.cos(5.0 / 50.0)]
    X[1, :2] = [5.0, 0.0]
    s, _, _ = O.frenet(tr, X[:, :2])
    assert s[0] > L - 6.0 and abs(s[1] - 5.0) < 1e-9
    f0 = OF.features(tr, X, np.zeros(2), 0, 60, 0.05, False)
    f1 = OF.features(tr, X, np.zeros(2), 1, 60, 0.05, False)
    assert abs(f0[9] * 40.0 - (s[1] + L - s[0])) < 1e-9 and 9.9 < f0[9] * 40.0 < 10.1
    assert abs(f1[9] + f0[9]) < 1e-12


def test_progress_gain_along_a_straight_and_across_the_wrap():
    td, tr = _oval()
    L = OF.arc_lengths(tr)[1]
    st = np.array([[x, 0.0, 0.0, 20.0] for x in np.arange(100.0, 121.0)])
    assert abs(OF.progress_gain(tr, st) - 20.0) < 1e-9
    # around the end of the left semicircle into the straight: arc 5 m, then 5 m of straight
    a = np.linspace(math.pi - 0.1, math.pi, 11)
    arc = np.stack([-50.0 * np.sin(a), 50.0 + 50.0 * np.cos(a), np.zeros(11), np.full(11, 20.0)], axis=1)
    line = np.array([[x, 0.0, 0.0, 20.0] for x in np.arange(1.0, 6.0)])
    g = OF.progress_gain(tr, np.concatenate([arc, line]))
    assert 9.9 < g < 10.1


# ------------------------------------------------------------------ mixed sampler
@pytest.fixture(scope="module")
def br_case():
    sc = S.single_br_oval()
    p = S.params_fullscale()
    tr = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    return sc, p, tr


def test_mixed_with_no_proposal_samples_is_the_plain_response(br_case):
    sc, p, tr = br_case
    T, K = sc.T, 256
    a = O.best_response(p, tr, sc.X0[0], sc.U0[0], 1.0, sc.opp, T, K, seed=5, want_costs=True)
    prop = np.tile([0.0, 0.0, 1.0, 0.05], (T, 1))
    b = O.best_response(p, tr, sc.X0[0], sc.U0[0], 1.0, sc.opp, T, K, seed=5, want_costs=True, prop=prop,
                        K_prop=0)
    assert a["k_star"] == b["k_star"] and np.array_equal(a["costs"], b["costs"])


def test_mixed_sampler_with_the_plain_distribution_uses_stream_one(br_case):
    """A proposal equal to the plain distribution (mean U-bar, sigma) for all
    K samples is the plain sampler on noise stream 1."""
    sc, p, tr = br_case
    T, K = sc.T, 256
    f32 = lambda v: float(np.float32(v))
    prop = np.stack([np.asarray(sc.U0[0])[:, 0], np.asarray(sc.U0[0])[:, 1],
                     np.full(T, f32(p["sigma_a"])), np.full(T, f32(p["sigma_delta"]))], axis=1)
    a = O.best_response(p, tr, sc.X0[0], sc.U0[0], 1.0, sc.opp, T, K, seed=5, stream=1, want_costs=True)
    b = O.best_response(p, tr, sc.X0[0], sc.U0[0], 1.0, sc.opp, T, K, seed=5, want_costs=True, prop=prop,
                        K_prop=K)
    c = O.best_response(p, tr, sc.X0[0], sc.U0[0], 1.0, sc.opp, T, K, seed=5, want_costs=True)
    assert np.array_equal(a["costs"], b["costs"]) and a["k_star"] == b["k_star"]
    assert not np.array_equal(a["costs"], c["costs"])
    # a split budget takes the first K_prop costs from stream 1, the rest from stream 0
    d = O.best_response(p, tr, sc.X0[0], sc.U0[0], 1.0, sc.opp, T, K, seed=5, want_costs=True, prop=prop,
                        K_prop=100)
    assert np.array_equal(d["costs"][:100], a["costs"][:100])
    assert np.array_equal(d["costs"][100:], c["costs"][100:])


def test_mixed_sampler_clips_and_centres_on_the_proposal(br_case):
    sc, p, tr = br_case
    T = sc.T
    # a near-deterministic proposal far from U-bar: every proposal sample's
    # controls sit at the (clipped) proposal mean
    prop = np.tile([3.0, 0.01, 1e-9, 1e-9], (T, 1))
    r = O.best_response(p, tr, sc.X0[0], sc.U0[0], 1.0, sc.opp, T, 8, seed=1, prop=prop, K_prop=8)
    assert np.allclose(r["u_star"][:, 0], 3.0, atol=1e-6) and np.allclose(r["u_star"][:, 1], 0.01, atol=1e-6)
    prop[:, 0] = 50.0
    r = O.best_response(p, tr, sc.X0[0], sc.U0[0], 1.0, sc.opp, T, 8, seed=1, prop=prop, K_prop=8)
    assert np.allclose(r["u_star"][:, 0], float(np.float32(p["a_max"])))
