"""The static-scratch best response (sgtp_best_response_noalloc) against the
workspace entry point (sgtp_best_response) and the oracle: two calls in a
row on different problems through the one library-held scratch, each
identical bit for bit to the workspace call (both run the same kernels on
the same inputs), the first also checked against the FP64 oracle's
selection and re-rolled winner; and the largest problem the ABI accepts
(15 opponents, T = 128), which must fit the scratch.  Kept in its own file,
collected last, so that it runs after every other test as well as alone."""
import numpy as np
import pytest

import oracle as O
from paper_2607_25388_b300 import scenario as S
from tests.parity_util import STATE_RTOL, assert_rel_close, selection_ok

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _pair(P, trk, p, x0, u0, opp, T, K, seed, rnd):
    args = (trk, p, dev(x0), dev(u0), 1.0, dev(opp), T, K)
    a = P.best_response(*args, seed=seed, rnd=rnd, game_on=rnd > 0)
    b = P.best_response_noalloc(*args, seed=seed, rnd=rnd, game_on=rnd > 0)
    torch.cuda.synchronize()
    for k in ("k_star", "any_feasible", "xi_star", "u_star"):
        assert torch.equal(a[k], b[k]), k
    return b


def test_noalloc_matches_workspace_entry_point_on_two_calls_in_a_row():
    from paper_2607_25388_b300 import planner as P
    p = S.params_fullscale()
    sc = S.ten_car_race(401, K=4096, T=60, L=1)          # 9 opponents, T = 60
    opp = np.stack([S.constant_velocity_prediction(sc.X0[j], sc.T, p["dt"]) for j in range(1, 10)])
    sc2 = S.two_car_race(402, K=2048, T=40)               # 1 opponent, T = 40
    opp2 = S.constant_velocity_prediction(sc2.X0[1], sc2.T, p["dt"])[None]
    b = _pair(P, P.Track.from_data(sc.track), p, sc.X0[0], sc.U0[0], opp, 60, 4096, 3, 1)
    _pair(P, P.Track.from_data(sc2.track), p, sc2.X0[0], sc2.U0[0], opp2, 40, 2048, 8, 0)
    # the first call against the oracle: its selection over all 4096 samples and the winner
    ot = O.Track(sc.track.xr, sc.track.wl, sc.track.wr)
    o = O.rollout_costs(p, ot, sc.X0[0], sc.U0[0], 1.0, opp, 60, K=4096, seed=3, rnd=1, game_on=True)
    ko, _ = O.select(o["cost"], o["feasible"], o["violation"])
    kg = int(b["k_star"].item())
    assert selection_ok(kg, ko, o["cost"], o["feasible"], o["violation"], o["margins"]), (kg, ko)
    w = O.rollout_costs(p, ot, sc.X0[0], sc.U0[0], 1.0, opp, 60, k_list=[kg], seed=3, rnd=1, game_on=True,
                        want_states=True, want_controls=True)
    assert_rel_close(b["xi_star"].cpu().numpy(), w["states"][0], STATE_RTOL, "xi*")
    assert_rel_close(b["u_star"].cpu().numpy(), w["controls"][0], STATE_RTOL, "u*")


def test_noalloc_holds_the_largest_problem_the_abi_accepts():
    from paper_2607_25388_b300 import planner as P
    p = S.params_fullscale()
    sc = S.ten_car_race(403, K=256, T=128, L=1)
    X0 = np.concatenate([sc.X0, sc.X0[:6] + np.float32([0.0, 0.0, 0.0, 1.0])])      # 16 vehicles
    opp = np.stack([S.constant_velocity_prediction(X0[j], 128, p["dt"]) for j in range(1, 16)])
    U0 = np.zeros((128, 2), np.float32)
    _pair(P, P.Track.from_data(sc.track), p, X0[0], U0, opp, 128, 256, 5, 2)


def test_noalloc_rejects_out_of_range_sizes_before_launch():
    from paper_2607_25388_b300 import _lib
    L = _lib.lib()
    n0 = L.sgtp_launch_count()
    P = _lib.make_params(S.params_fullscale())
    import ctypes as C
    vp = C.c_void_p
    for n_opp, T in ((16, 60), (3, 129), (3, 0)):
        st = L.sgtp_best_response_noalloc(vp(16), 0, C.byref(P), vp(16), vp(16), 1.0, vp(16), n_opp, T, 64, 0, 0, 0,
                                          0, 1, vp(16), vp(16), vp(16), vp(16), None)
        assert st == 1
    assert L.sgtp_launch_count() == n0
