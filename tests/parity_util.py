"""Shared helpers of the GPU parity tests: comparison rules against the
FP64 oracle.

Tolerances (written here once and used by every parity test):

* states: |gpu - oracle| <= STATE_RTOL * max(1, |oracle|) with STATE_RTOL =
  1e-4 (relative; absolute below magnitude 1).
* Frenet progress s and offset d: |gpu - oracle| <= STATE_RTOL * max(1, |p|,
  |s|) where |p| is the size of the state's position.  s and d are
  1-Lipschitz functions of the position (away from the polyline's medial
  axis), so their error is bounded by the position error, which the state
  tolerance bounds relative to the coordinates, not to d itself.
* cost: same rule with COST_RTOL = 1e-4, for candidates not near a threshold.
* violation nu: a sum of clearance shortfalls in metres, i.e. of differences
  of 1-Lipschitz functions of positions, so it inherits the position
  tolerance: |gpu - oracle| <= STATE_RTOL * max(1, |nu|, position scale)
  with the track's coordinate magnitude as the position scale.
* feasibility flags: exact, except candidates whose oracle indicator
  arguments lie within a guard band of their threshold (boundary clearance
  within GUARD_DIST of m_bd, obstacle clearance within GUARD_DIST of d_col,
  |Delta s| within GUARD_PROG of s_contest / s_role).  The bands bound the
  float32 rounding of coordinates up to a few km (ulp 2.4e-4 m at 3 km)
  accumulated over at most 128 steps.
* selected index: equal, unless the oracle costs (or violations) of the two
  picks differ by less than SELECT_RTOL = 1e-5 relative, or either pick is
  near a threshold.
"""
import numpy as np

STATE_RTOL = 1e-4
COST_RTOL = 1e-4
SELECT_RTOL = 1e-5
GUARD_DIST = 2e-3
GUARD_PROG = 2e-2


def assert_rel_close(gpu, ref, rtol, what, mask=None):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    err = np.abs(gpu - ref) / np.maximum(1.0, np.abs(ref))
    if mask is not None:
        err = err[mask]
    worst = float(err.max()) if err.size else 0.0
    assert worst <= rtol, f"{what}: worst relative error {worst:.3e} > {rtol:.1e}"
    return worst


def assert_frenet_close(gpu_fr, ref_fr, ref_states, what="frenet"):
    g = np.asarray(gpu_fr, dtype=np.float64)
    r = np.asarray(ref_fr, dtype=np.float64)
    st = np.asarray(ref_states, dtype=np.float64)
    scale = np.maximum(1.0, np.maximum(np.abs(st[..., :2]).max(-1), np.abs(r[..., 0])))
    err = np.abs(g - r) / scale[..., None]
    worst = float(err.max()) if err.size else 0.0
    assert worst <= STATE_RTOL, f"{what}: worst scaled error {worst:.3e} > {STATE_RTOL:.1e}"
    return worst


def borderline(margins):
    """Candidates whose oracle indicator arguments sit within the guard band."""
    m = np.asarray(margins)
    return (m[:, 0] <= GUARD_DIST) | (m[:, 1] <= GUARD_DIST) | (m[:, 2] <= GUARD_PROG)


def check_candidates(gpu, orc, what="", pos_scale=1.0):
    """Element-wise comparison of per-candidate outputs; returns the number
    of borderline candidates excluded from the exact checks.  pos_scale is
    the coordinate magnitude of the track (metres)."""
    bl = borderline(orc["margins"])
    ok = ~bl
    feas_g = np.asarray(gpu["feasible"]).astype(bool)
    feas_o = np.asarray(orc["feasible"]).astype(bool)
    bad = np.nonzero((feas_g != feas_o) & ok)[0]
    assert bad.size == 0, f"{what}: feasibility differs at k={bad[:10]} (of {bad.size})"
    assert_rel_close(np.asarray(gpu["cost"])[ok], orc["cost"][ok], COST_RTOL, f"{what} cost")
    vg = np.asarray(gpu["violation"], dtype=np.float64)[ok]
    vo = np.asarray(orc["violation"], dtype=np.float64)[ok]
    err = np.abs(vg - vo) / np.maximum(max(1.0, pos_scale), np.abs(vo))
    worst = float(err.max()) if err.size else 0.0
    assert worst <= STATE_RTOL, f"{what} violation: worst scaled error {worst:.3e} > {STATE_RTOL:.1e}"
    return int(bl.sum())


def selection_ok(k_gpu, k_orc, orc_cost, orc_feas, orc_viol, orc_margins=None):
    """Selected index equal, or an allowed near-tie (see module docstring)."""
    if k_gpu == k_orc:
        return True
    if orc_margins is not None:
        bl = borderline(orc_margins)
        if bl[k_gpu] or bl[k_orc]:
            return True
    fg, fo = bool(orc_feas[k_gpu]), bool(orc_feas[k_orc])
    if fg != fo:
        return False
    vg = orc_cost[k_gpu] if fo else orc_viol[k_gpu]
    vo = orc_cost[k_orc] if fo else orc_viol[k_orc]
    return abs(vg - vo) <= SELECT_RTOL * max(1.0, abs(vo))
