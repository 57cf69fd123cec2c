"""Shared helpers of the GPU parity tests: comparison rules against the
FP64 oracle.

Tolerances (written here once and used by every parity test):

* states: |gpu - oracle| <= STATE_RTOL * max(1, |oracle|) with STATE_RTOL =
  1e-4 (relative; absolute below magnitude 1).
* Frenet offset d and violation nu: absolute, FRENET_ABS = VIOL_ABS = 2e-3 m,
  the feasibility guard band.  Measured worst over the parity workloads:
  d 5.4e-4 m, nu 5.0e-4 m (positions 5.7e-4 m after 128 steps), so the bound
  has a margin of about four.
* Frenet progress s: |gpu - oracle| <= FRENET_ABS (measured 3.8e-4 m),
  except at a near-tie of the projection (two feet on the polyline nearly
  equidistant from the state; Sec. II does not single one out beyond the
  lowest-index rule, which an FP32 evaluation cannot resolve inside its
  rounding): there the GPU's foot point, the polyline point at its s, must
  lie at the oracle's distance |d| within FRENET_ABS -- the unique part of
  the result is the distance, and the GPU's s must be a nearest point.
* cost: |gpu - oracle| <= COST_RTOL * max(1, |oracle|), COST_RTOL = 1e-4,
  for candidates not near a threshold.
* feasibility flags: exact, except candidates whose oracle indicator
  arguments lie within a guard band of their threshold (boundary clearance
  within GUARD_DIST of m_bd, obstacle clearance within GUARD_DIST of d_col,
  |Delta s| within GUARD_PROG of s_contest / s_role).  The bands bound the
  float32 rounding of coordinates up to a few km (ulp 2.4e-4 m at 3 km)
  accumulated over at most 128 steps.
* selected index: equal, unless the oracle costs (or violations) of the two
  picks differ by less than SELECT_RTOL = 1e-5 relative, or either pick is
  near a threshold.

Every check records its worst error in WORST; the test session prints them.
"""
import numpy as np

STATE_RTOL = 1e-4
COST_RTOL = 1e-4
SELECT_RTOL = 1e-5
GUARD_DIST = 2e-3
GUARD_PROG = 2e-2
FRENET_ABS = 2e-3
VIOL_ABS = 2e-3

WORST = {}


def _note(what, value):
    WORST[what] = max(WORST.get(what, 0.0), float(value))


def assert_rel_close(gpu, ref, rtol, what, mask=None):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    err = np.abs(gpu - ref) / np.maximum(1.0, np.abs(ref))
    if mask is not None:
        err = err[mask]
    worst = float(err.max()) if err.size else 0.0
    _note(f"relative {what.split()[0]}", worst)
    assert worst <= rtol, f"{what}: worst relative error {worst:.3e} > {rtol:.1e}"
    return worst


def polyline_point(xr, s):
    """Point of the closed polyline through the waypoints xr[:, :2] at arc
    length s (modulo the length), in float64."""
    P = np.asarray(xr, dtype=np.float64)[:, :2]
    Q = np.roll(P, -1, axis=0)
    seg = np.linalg.norm(Q - P, axis=1)
    cum = np.concatenate([[0.0], np.cumsum(seg)])
    s = np.mod(np.asarray(s, dtype=np.float64), cum[-1])
    j = np.clip(np.searchsorted(cum, s, side="right") - 1, 0, len(P) - 1)
    u = (s - cum[j]) / seg[j]
    return P[j] + u[..., None] * (Q[j] - P[j])


def assert_frenet_close(gpu_fr, ref_fr, ref_states, track_xr, what="frenet"):
    """Frenet (s, d) per state against the oracle (rules in the module
    docstring); returns (worst |ds| outside near-ties, worst |dd|, near-ties)."""
    g = np.asarray(gpu_fr, dtype=np.float64)
    r = np.asarray(ref_fr, dtype=np.float64)
    st = np.asarray(ref_states, dtype=np.float64)
    dd = np.abs(g[..., 1] - r[..., 1])
    worst_d = float(dd.max()) if dd.size else 0.0
    assert worst_d <= FRENET_ABS, f"{what}: worst |d| error {worst_d:.3e} m > {FRENET_ABS:.1e}"
    ds = np.abs(g[..., 0] - r[..., 0])
    far = ds > FRENET_ABS
    n_tie = int(far.sum())
    if n_tie:
        foot = polyline_point(track_xr, g[..., 0][far])
        dist = np.linalg.norm(st[..., :2][far] - foot, axis=-1)
        gap = np.abs(dist - np.abs(r[..., 1][far]))
        assert gap.max() <= FRENET_ABS, \
            f"{what}: {n_tie} states with |s| error above {FRENET_ABS} m whose GPU foot point is not nearest " \
            f"(worst distance gap {gap.max():.3e} m, worst |ds| {ds.max():.3e} m)"
    worst_s = float(ds[~far].max()) if (~far).any() else 0.0
    _note("frenet |ds| (m)", worst_s)
    _note("frenet |dd| (m)", worst_d)
    _note("frenet s near-ties", n_tie)
    return worst_s, worst_d, n_tie


def borderline(margins):
    """Candidates whose oracle indicator arguments sit within the guard band."""
    m = np.asarray(margins)
    return (m[:, 0] <= GUARD_DIST) | (m[:, 1] <= GUARD_DIST) | (m[:, 2] <= GUARD_PROG)


def check_candidates(gpu, orc, what=""):
    """Element-wise comparison of per-candidate outputs; returns the number
    of borderline candidates excluded from the exact checks."""
    bl = borderline(orc["margins"])
    ok = ~bl
    feas_g = np.asarray(gpu["feasible"]).astype(bool)
    feas_o = np.asarray(orc["feasible"]).astype(bool)
    bad = np.nonzero((feas_g != feas_o) & ok)[0]
    assert bad.size == 0, f"{what}: feasibility differs at k={bad[:10]} (of {bad.size})"
    assert_rel_close(np.asarray(gpu["cost"])[ok], orc["cost"][ok], COST_RTOL, f"{what} cost")
    vg = np.asarray(gpu["violation"], dtype=np.float64)[ok]
    vo = np.asarray(orc["violation"], dtype=np.float64)[ok]
    err = np.abs(vg - vo)
    worst = float(err.max()) if err.size else 0.0
    _note("violation (m)", worst)
    assert worst <= VIOL_ABS, f"{what} violation: worst error {worst:.3e} m > {VIOL_ABS:.1e}"
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
