"""Host-side allocation-failure injection (sgtp_debug_fail_alloc): any one
device allocation made by track creation, batch creation, network creation
or training-scratch growth can fail.  The entry point then returns
SGTP_E_NOMEM without launching anything, releases what it had allocated
(device free memory returns to its level), and the library works again
once the hook is disarmed.  Nothing on the device fails."""
import pytest

from paper_2607_25388_b300 import scenario as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib():
    from paper_2607_25388_b300 import _lib as L
    return L.lib()


def _fails_at_every_allocation(make, n_max):
    """Arm the hook for allocation 1, 2, ... until the call succeeds; return
    the number of allocations the call makes."""
    L = _lib()
    try:
        for n in range(1, n_max + 1):
            L.sgtp_debug_fail_alloc(n)
            launches = L.sgtp_launch_count()
            try:
                obj = make()
            except RuntimeError as e:
                assert "SGTP_E_NOMEM" in str(e), str(e)
                assert L.sgtp_launch_count() == launches
                continue
            L.sgtp_debug_fail_alloc(0)
            return n - 1, obj
        raise AssertionError("the call kept failing")
    finally:
        L.sgtp_debug_fail_alloc(0)


def test_track_batch_and_network_creation_fail_cleanly():
    from paper_2607_25388_b300 import learned as LR, planner as P
    import gc
    sc = S.ten_car_race(601, K=256, T=30, L=1)
    p = S.params_fullscale()
    X0, U0, vs = torch.as_tensor(sc.X0).cuda(), torch.as_tensor(sc.U0.reshape(-1)).cuda(), \
        torch.as_tensor(sc.vref_scale).cuda()

    def plan_once(trk):
        b = P.Batch(trk, [dict(track_id=0, n_v=10, T=30, ego=0, race_tag=0)], K=256, L=1)
        out = b.plan(p, X0, U0.clone(), vs, seed=1)
        torch.cuda.synchronize()
        return out["status"].item()

    # warm-up: the kernels' code is loaded on first use and stays resident
    assert plan_once(P.Track.from_data(sc.track)) == 0
    LR.Mlp(60, seed=1).reserve(1024)
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0 = torch.cuda.mem_get_info()[0]
    n_trk, trk = _fails_at_every_allocation(lambda: P.Track.from_data(sc.track), 40)
    assert n_trk >= 10                                  # every track array is its own allocation
    n_b, b = _fails_at_every_allocation(
        lambda: P.Batch(trk, [dict(track_id=0, n_v=10, T=30, ego=0, race_tag=0)], K=256, L=1), 5)
    assert n_b >= 1
    n_m, net = _fails_at_every_allocation(lambda: LR.Mlp(60, seed=1), 20)
    assert n_m >= 5
    n_r, _ = _fails_at_every_allocation(lambda: net.reserve(1024), 30)
    assert n_r >= 10
    # the surviving objects work
    out = b.plan(p, X0, U0.clone(), vs, seed=1)
    torch.cuda.synchronize()
    assert out["status"].item() == 0
    del out, b, trk, net
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    # nothing leaked by the failed attempts (driver allocation granularity allowed)
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)
