"""The static-scratch best response (sgtp_best_response_noalloc) against the
workspace entry point (sgtp_best_response): two calls in a row on different
problems through the one library-held scratch, each equal to the workspace
call within the parity tolerances (same selected index, states and
controls within STATE_RTOL).  Kept in its own file, collected last, so that
it runs after every other test as well as alone."""
import numpy as np
import pytest

from paper_2607_25388_b300 import scenario as S
from tests.parity_util import STATE_RTOL, assert_rel_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_workspace_entry_point_on_two_calls_in_a_row():
    from paper_2607_25388_b300 import planner as P
    p = S.params_fullscale()
    cases = []
    sc = S.ten_car_race(401, K=4096, T=60, L=1)          # 9 opponents, T = 60
    opp = np.stack([S.constant_velocity_prediction(sc.X0[j], sc.T, p["dt"]) for j in range(1, 10)])
    cases.append((sc, opp, 4096, 3, 1))
    sc2 = S.two_car_race(402, K=2048, T=40)               # 1 opponent, T = 40
    opp2 = S.constant_velocity_prediction(sc2.X0[1], sc2.T, p["dt"])[None]
    cases.append((sc2, opp2, 2048, 8, 0))
    for n, (sc, opp, K, seed, rnd) in enumerate(cases):
        trk = P.Track.from_data(sc.track)
        args = (trk, p, dev(sc.X0[0]), dev(sc.U0[0]), 1.0, dev(opp), sc.T, K)
        a = P.best_response(*args, seed=seed, rnd=rnd, game_on=rnd > 0)
        b = P.best_response_noalloc(*args, seed=seed, rnd=rnd, game_on=rnd > 0)
        torch.cuda.synchronize()
        assert int(a["k_star"].item()) == int(b["k_star"].item()), f"call {n}"
        assert int(a["any_feasible"].item()) == int(b["any_feasible"].item()), f"call {n}"
        assert_rel_close(b["xi_star"].cpu().numpy(), a["xi_star"].cpu().numpy(), STATE_RTOL, f"xi* call {n}")
        assert_rel_close(b["u_star"].cpu().numpy(), a["u_star"].cpu().numpy(), STATE_RTOL, f"u* call {n}")


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
