"""Algorithmic work of the best-response path, counted from its definition.

One rollout-step is one (candidate k, step tau) pair.  The FP32 work of a
step follows the method's definition (Sec. II sampling and dynamics,
Eq. ctrack, Sec. III-B checks, Eq. Dmin) with the projection taken as the
incremental nearest-segment search of about 2.5 segment evaluations per
step: 72 FP32 operations for noise scaling, controls, control costs,
dynamics, projection, tracking and boundary terms, plus 5 per opponent
(two differences, the squared distance, its minimum).  The terminal game
terms (Eqs. c_contest, c_long, c_block, c_safety) cost 25 FP32 operations
and one square root per opponent and candidate.  An FMA counts as two
operations.  The Philox integer work and the special-function evaluations
(logarithm, square root, sine, cosine of the noise and the dynamics) are
not counted as FP32 operations, so the fraction of the FP32 peak is a
lower bound of the arithmetic the kernel issues.

Per rollout-step: 72 + 5 n_opp; per candidate: 26 n_opp.  Ten-car plan
(n_opp = 9, T = 60): 117 + 234 / 60 = 120.9 per rollout-step.
"""
from __future__ import annotations

STEP_BASE = 72.0
STEP_PER_OPP = 5.0
TERM_BASE = 0.0
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
    """SHA-256 over the sources the plan kernel is compiled from (its
    translation unit sgtp_plan.cu, every CUDA header and the ABI headers),
    so that a DRAM traffic figure taken by ncu can be tied to the exact
    kernel it measured."""
    import hashlib
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    files = [os.path.join(here, "csrc", "sgtp_plan.cu")]
    for d, exts in ((os.path.join(here, "csrc"), (".cuh", ".hpp")),
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
    """Nominal FP32 peak from unit counts: SMs x 128 FP32 lanes x 2 (FMA) x clock."""
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def measure_fma_peak(reps: int = 5, iters: int = 20000):
    """FP32 FMA throughput of the current device measured with the library's
    own probe (sgtp_fma_probe: independent FMA chains, scalar and packed
    f32x2, four 256-thread CTAs per SM), CUDA events on the launching
    stream, best of `reps` launches of each form.  Returns (TFLOP/s, form)."""
    import ctypes

    import torch

    from . import _lib
    L = _lib.lib()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sink = torch.zeros(sms * 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    best = (0.0, "")
    for packed in (0, 1):
        for r in range(reps + 1):
            fl = ctypes.c_double()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st = L.sgtp_fma_probe(4, iters, packed, ctypes.c_void_p(sink.data_ptr()),
                                  ctypes.c_void_p(stream.cuda_stream), ctypes.byref(fl))
            b.record(stream)
            torch.cuda.synchronize()
            if st != 0:
                raise RuntimeError(f"sgtp_fma_probe failed: {L.sgtp_last_error().decode()}")
            if r == 0:
                continue                      # first launch warms the clocks
            tf = fl.value / (a.elapsed_time(b) / 1e3) / 1e12
            if tf > best[0]:
                best = (tf, "fma.rn.f32x2" if packed else "fma.rn.f32")
    return best
