"""Algorithmic work of the best-response path, counted from its definition.

One rollout-step is one (candidate k, step tau) pair.  Its floating-point
operations are counted from the method's definition (Sec. II sampling and
dynamics, Eq. ctrack, Sec. III-B checks, Eq. Dmin), one per add, subtract,
multiply, divide, min/max, compare, square root, logarithm or trigonometric
function; an FMA counts as two.  The Frenet projection is counted as three
point-to-segment evaluations (the nearest segment and the two neighbours that
certify it as the local minimum) plus the signed offset and progress.

Per step (n = opponents):
  noise        12   two uniforms (2 each), ln, x(-2), sqrt, 2*pi*u, cos, sin, 2 products
  controls      8   two sigma*z, two additions to U-bar, two clips (min+max)
  control cost  6   a^2, delta^2, two weights, two sums
  smoothness    8   two differences, two squares, two weights... (tau >= 1)
  dynamics     16   cos, sin, dt*v, two products, two sums, tan, product, /L, sum, dt*a, sum, clamp(2)
  Frenet       61   3 x 16 per segment evaluation, sqrt, cross product (3), sign, s_j + t*len (2), unwrap (7)
  tracking     17   four errors (heading wrap 4 extra), four squares, four weights, sums
  boundary      8   two width interpolations (4), w+d, w-d, two minima
  tail offset   0.3 one sum over the tail share (mu_tail = 0.3) of the steps
  opponents    6n   per opponent: dx, dy, dx^2 + dy^2 (3), minimum
Terminal work per candidate: 10 + 26 n (progress gap, indicators, alpha-
weighted gain, blocking ratio, sqrt, safety square, sums, checks).
"""
from __future__ import annotations

STEP_BASE = 12 + 8 + 6 + 8 + 16 + 61 + 17 + 8 + 0.3
STEP_PER_OPP = 6.0
TERM_BASE = 10.0
TERM_PER_OPP = 26.0

SMS = 148
FP32_LANES_PER_SM = 128
MAX_SM_MHZ = 2032.0


def flops_per_step(n_opp: int) -> float:
    return STEP_BASE + STEP_PER_OPP * n_opp


def flops_best_response(K: int, T: int, n_opp: int) -> float:
    return K * (T * flops_per_step(n_opp) + TERM_BASE + TERM_PER_OPP * n_opp)


def flops_plan(n_v: int, K: int, T: int, L: int) -> float:
    """(L+1) Jacobi rounds of n_v responses plus the extra ego response,
    each against n_v - 1 opponents."""
    n_br = (L + 1) * n_v + 1
    return n_br * flops_best_response(K, T, n_v - 1)


def rollout_steps_plan(n_v: int, K: int, T: int, L: int) -> int:
    return ((L + 1) * n_v + 1) * K * T


def kernel_source_digest() -> str:
    """SHA-256 over the CUDA sources and ABI headers, so that a DRAM traffic
    figure taken by ncu can be tied to the exact kernel it measured."""
    import hashlib
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    files = []
    for d, exts in ((os.path.join(here, "csrc"), (".cu", ".cuh", ".hpp")),
                    (os.path.join(os.path.dirname(here), "include"), (".h",))):
        files += sorted(os.path.join(d, f) for f in os.listdir(d) if f.endswith(exts))
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(profile_md: str):
    """(bytes per launch, source digest) from a profile summary's
    `traffic_bytes_per_launch:` and `source_sha256:` lines, or None."""
    import os
    import re
    if not os.path.exists(profile_md):
        return None
    txt = open(profile_md).read()
    t = re.search(r"^traffic_bytes_per_launch:\s*([0-9]+)", txt, re.M)
    d = re.search(r"^source_sha256:\s*([0-9a-f]{64})", txt, re.M)
    if not (t and d):
        return None
    return int(t.group(1)), d.group(1)


def fp32_peak_tflops(sm_mhz: float = MAX_SM_MHZ, sms: int = SMS) -> float:
    """SMs x 128 FP32 lanes x 2 (FMA) x clock."""
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
