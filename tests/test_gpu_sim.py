"""GPU parity of the closed-loop trial step (sgtp_sim_reset / sgtp_sim_step)
against the FP64 oracle (oracle/sim.py), teacher-forced per control period:
each GPU step is recomputed by the oracle from the GPU's own inputs (states,
warm starts, plans and trial records before the step).

Rules (tests/parity_util.py): states to STATE_RTOL; Frenet progress and
offsets to STATE_RTOL of the position magnitude; the warm-start shift is a
copy, so exact; the integer fields (steps, alive, contact kind, close-run
counters) exactly, except in a step where the oracle's decision arguments
came within the guard band (GUARD_DIST m, GUARD_PROG m of longitudinal
distance) of a threshold; the ego's speed and control-difference sums to
1e-4 relative (absolute 1e-5 for the latter: pure-pursuit controls are
differences of nearly equal numbers).  Also: replaying a plan's controls
reproduces its trajectory bit for bit (same dynamics code), and whole trials
of all three planners run to their end."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from oracle import sim as OS
from paper_2607_25388_b300 import scenario as S
from tests.parity_util import GUARD_DIST, GUARD_PROG, STATE_RTOL, assert_rel_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _trials(tracker, n_apply, K=256, T=30, L=1, n=4, max_steps=60, mppi_lambda=None, params=None):
    from paper_2607_25388_b300 import sim as SM
    scs = [S.trial_race(S.fourier_track(731 + r, n_points=1500), 3, T, K, L, 900 + r, s0=100.0 * r)
           for r in range(n)]
    p = params or S.params_fullscale()
    sp = SM.sim_params(n_apply=n_apply, max_steps=max_steps, tracker=tracker, pp_preview=4)
    return SM.Trials(scs, p, K, L, sp, mppi_lambda=mppi_lambda), scs, p, sp


def _records(tr):
    from paper_2607_25388_b300._lib import SimRace
    raw = tr.state.cpu().numpy().tobytes()
    return (SimRace * len(tr.scenarios)).from_buffer_copy(raw)


def _as_oracle(rec, n_v):
    return dict(alive=rec.alive, steps=rec.steps, ego_collision=rec.ego_collision,
                close_segments=rec.close_segments, close_steps=rec.close_steps,
                ego_speed_sum=float(rec.ego_speed_sum), ego_du2_sum=float(rec.ego_du2_sum),
                progress=np.array(rec.progress[:n_v], np.float64), rel0=np.array(rec.rel0[:n_v], np.float64),
                d=np.array(rec.d[:n_v], np.float64), s_raw=np.array(rec.s_raw[:n_v], np.float64),
                close_run=np.array(rec.close_run[:n_v], np.int64), u_prev=np.array(rec.u_prev[:], np.float64))


def _sp_dict(sp):
    return {f: getattr(sp, f) for f, _ in sp._fields_}


def _slices(scs):
    a = u = x = 0
    out = []
    for sc in scs:
        n_v, T = sc.X0.shape[0], sc.T
        out.append((a, u, x))
        a, u, x = a + n_v, u + n_v * T * 2, x + n_v * (T + 1) * 4
    return out


def _frenet_close(g, o, scale, what):
    err = np.abs(np.asarray(g, np.float64) - np.asarray(o, np.float64)) / max(1.0, scale)
    assert err.max() <= STATE_RTOL, f"{what}: scaled error {err.max():.3e}"


def test_reset_matches_oracle():
    tr, scs, p, sp = _trials(0, 2)
    tr.reset()
    torch.cuda.synchronize()
    for rec, sc in zip(_records(tr), scs):
        ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
        o = OS.reset(ot, sc.X0.astype(np.float64), sc.ego)
        n_v = sc.X0.shape[0]
        scale = float(np.abs(sc.track.xr[:, :2]).max())
        assert rec.alive == 1 and rec.steps == 0 and rec.ego_collision == 0
        _frenet_close(rec.s_raw[:n_v], o["s_raw"], max(scale, OS.track_len(ot)), "s")
        _frenet_close(rec.d[:n_v], o["d"], scale, "d")
        _frenet_close(rec.rel0[:n_v], o["rel0"], max(scale, OS.track_len(ot)), "rel0")


def check_trial_step(p, ot, spd, sc, sl, X0, U0, xi, rec0, rec1, X1, U1, what):
    """Compare one trial's GPU step (rec0 -> rec1, X0/U0 -> X1/U1) with the
    oracle's step from the same inputs; returns whether the continuous
    fields were compared (not after a contact decided within the guard)."""
    n_v, T = sc.X0.shape[0], sc.T
    a, u, x = sl
    mg = []
    Xo, Uo, so = OS.step(p, ot, spd, X0[a:a + n_v], U0[u:u + n_v * T * 2].reshape(n_v, T, 2),
                         xi[x:x + n_v * (T + 1) * 4].reshape(n_v, T + 1, 4), sc.ego, _as_oracle(rec0, n_v), margins=mg)
    near = any(m[0] <= GUARD_DIST or m[1] <= GUARD_DIST or m[2] <= GUARD_PROG or m[3] <= GUARD_DIST for m in mg)
    g = rec1
    if not near:
        assert (g.alive, g.steps, g.ego_collision) == (so["alive"], so["steps"], so["ego_collision"]), what
        assert (g.close_segments, g.close_steps) == (so["close_segments"], so["close_steps"]), what
        assert list(g.close_run[:n_v]) == [int(v) for v in so["close_run"]], what
    if g.steps != so["steps"]:
        return False                 # a contact decided differently within the guard band
    assert_rel_close(X1[a:a + n_v], Xo, STATE_RTOL, what + " X")
    np.testing.assert_array_equal(U1[u:u + n_v * T * 2].reshape(n_v, T, 2), Uo.astype(np.float32), err_msg=what + " U")
    scale = max(float(np.abs(sc.track.xr[:, :2]).max()), OS.track_len(ot))
    _frenet_close(g.progress[:n_v], so["progress"], scale, what + " progress")
    _frenet_close(g.s_raw[:n_v], so["s_raw"], scale, what + " s")
    _frenet_close(g.d[:n_v], so["d"], scale, what + " d")
    assert abs(g.ego_speed_sum - so["ego_speed_sum"]) <= 1e-4 * max(1.0, abs(so["ego_speed_sum"])), what
    assert abs(g.ego_du2_sum - so["ego_du2_sum"]) <= 1e-4 * abs(so["ego_du2_sum"]) + 1e-5, what
    return True


def _run_checked(tr, scs, p, sp, periods, trials):
    spd = _sp_dict(sp)
    sl = _slices(scs)
    tracks = {r: O.Track(scs[r].track.xr, scs[r].track.wl, scs[r].track.wr) for r in trials}
    checked = 0
    for period in range(periods):
        tr.plan()
        torch.cuda.synchronize()
        X0, U0, xi = tr.X.cpu().numpy(), tr.U.cpu().numpy(), tr.out["xi"].cpu().numpy()
        before = _records(tr)
        tr.sim_step()
        tr.k += 1
        torch.cuda.synchronize()
        X1, U1 = tr.X.cpu().numpy(), tr.U.cpu().numpy()
        after = _records(tr)
        for r in trials:
            if not before[r].alive:
                assert after[r].steps == before[r].steps
                continue
            checked += check_trial_step(p, tracks[r], spd, scs[r], sl[r], X0, U0, xi, before[r], after[r], X1, U1,
                                        f"period {period} trial {r}")
    return checked


@pytest.mark.parametrize("tracker,n_apply", [(0, 3), (1, 2)])
def test_sim_step_teacher_forced(tracker, n_apply):
    tr, scs, p, sp = _trials(tracker, n_apply)
    tr.reset()
    assert _run_checked(tr, scs, p, sp, 10, range(len(scs))) >= 20


def test_full_trial_set_sampled_trials():
    """The 42-trial set of the closed-loop results (7 tracks x 6 starts, the
    ego behind two opponents, K = 4096, T = 60, L = 2, pure pursuit, one
    control step per plan): eight sampled trials teacher-forced over the
    first 12 control periods."""
    from paper_2607_25388_b300 import sim as SM
    p = S.params_fullscale()
    scs = S.trial_set(7, 6, 3, 60, 4096, 2)
    sp = SM.sim_params(n_apply=1, max_steps=1000, tracker=SM.TRACK_PURE_PURSUIT)
    tr = SM.Trials(scs, p, 4096, 2, sp)
    tr.reset()
    trials = sorted(np.random.default_rng(5).choice(len(scs), 8, replace=False).tolist())
    assert _run_checked(tr, scs, p, sp, 12, trials) >= 60


def test_replaying_the_plan_controls_reproduces_its_trajectory():
    T = 30
    tr, scs, p, sp = _trials(0, T, T=T, max_steps=1000)
    tr.reset()
    tr.plan()
    torch.cuda.synchronize()
    xi = tr.out["xi"].cpu().numpy()
    tr.sim_step()
    torch.cuda.synchronize()
    X1 = tr.X.cpu().numpy()
    recs = _records(tr)
    sl = _slices(scs)
    n_full = 0
    for r, sc in enumerate(scs):
        if recs[r].steps != T:
            continue             # ended by a contact before the plan's end
        n_v = sc.X0.shape[0]
        a, _, x = sl[r]
        np.testing.assert_array_equal(X1[a:a + n_v], xi[x:x + n_v * (T + 1) * 4].reshape(n_v, T + 1, 4)[:, T])
        n_full += 1
    assert n_full >= 1


@pytest.mark.parametrize("variant", ["sgtp", "no_game_cost", "mppi"])
def test_whole_trials_run_to_their_end(variant):
    from paper_2607_25388_b300 import sim as SM
    p = S.params_fullscale()
    lam = None
    if variant == "no_game_cost":
        p = dict(p, w_game=0.0)
    if variant == "mppi":
        lam = 1.0e4
    tr, scs, p, sp = _trials(1, 2, K=512, T=40, L=1, n=6, max_steps=80, mppi_lambda=lam, params=p)
    tr.reset()
    times = tr.run()
    res = tr.results()
    assert all(r["alive"] == 0 for r in res)
    assert all(1 <= r["steps"] <= 80 for r in res)
    assert all(r["steps"] == 80 or r["ego_collision"] in (1, 2) for r in res)
    m = SM.trial_metrics(res, dt=p["dt"], limit_s=80 * p["dt"])
    assert 0.0 <= m["wins"] <= 1.0 and 0.0 <= m["fpr"] <= 1.0 and m["v_ego"] > 0
    assert np.isfinite(m["d_mean"]) and len(times) >= 1
