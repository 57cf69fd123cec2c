"""CPU-side checks of the C ABI: the library builds for sm_103a, loads,
exports every symbol the headers under include/ declare, and rejects
invalid arguments before launching anything (no GPU needed for any of
this)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2607_25388_b300 import _lib, scenario as S
from paper_2607_25388_b300.planner import Track

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    inc = os.path.join(ROOT, "include")
    for name in sorted(os.listdir(inc)):
        if name.endswith(".h"):
            txt = open(os.path.join(inc, name)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            syms |= set(re.findall(r"\b(sgtp_[a-z_0-9]+)\s*\(", txt))
    return sorted(syms)


def test_library_exports_every_declared_symbol():
    L = _lib.lib()
    syms = declared_symbols()
    assert len(syms) >= 25
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing
    assert set(_lib.EXPORTS) == set(syms)
    assert b"sm_103a" in L.sgtp_version()


def test_build_targets_sm_103a_only():
    from paper_2607_25388_b300 import build
    flags = " ".join(build.NVCC_FLAGS)
    assert "arch=compute_103a,code=sm_103a" in flags and "sm_100" not in flags


def test_workspace_sizes():
    L = _lib.lib()
    assert L.sgtp_br_workspace_bytes(9, 60) >= 256
    assert L.sgtp_br_workspace_bytes(-1, 60) == 0
    assert L.sgtp_plan_workspace_bytes(10, 60, 5) > L.sgtp_plan_workspace_bytes(2, 60, 5)
    assert L.sgtp_plan_workspace_bytes(0, 60, 5) == 0
    # GA-IBR-MPPI adds one row of 2T+2 floats per 256-sample tile per vehicle
    base = L.sgtp_plan_workspace_bytes(10, 60, 5)
    assert L.sgtp_plan_mppi_workspace_bytes(10, 60, 5, 16384) >= base + 10 * 64 * 122 * 4
    assert L.sgtp_plan_mppi_workspace_bytes(10, 60, 5, 0) == 0


def _params():
    return _lib.make_params(S.params_fullscale())


def test_invalid_arguments_are_rejected_without_launch():
    L = _lib.lib()
    P = _params()
    n0 = L.sgtp_launch_count()
    vp = C.c_void_p
    # NULL track
    st = L.sgtp_rollout_costs(None, 0, C.byref(P), vp(16), vp(16), 1.0, None, 0, 10, 10, 0, 0, 0, 0, 1,
                              vp(16), vp(16), vp(16), None, None, None, vp(256), 4096, None)
    assert st == 1 and b"track" in L.sgtp_last_error()
    st = L.sgtp_ibr_plan(None, 0, C.byref(P), 2, vp(16), vp(16), vp(16), 10, 10, 1, 0, 0, 0, vp(16), vp(16), None,
                         None, vp(16), None, vp(256), 1 << 20, None)
    assert st == 1
    # track with too few points / zero-length segment
    h = C.c_void_p()
    xr = np.zeros((2, 4), np.float32); w = np.ones(2, np.float32)
    assert L.sgtp_track_create(xr.ctypes.data, w.ctypes.data, w.ctypes.data, 2, None, C.byref(h)) == 1
    xr = np.zeros((5, 4), np.float32); w = np.ones(5, np.float32)
    assert L.sgtp_track_create(xr.ctypes.data, w.ctypes.data, w.ctypes.data, 5, None, C.byref(h)) == 1
    assert b"zero-length" in L.sgtp_last_error()
    # learned proposal: invalid sizes and NULL handles
    assert L.sgtp_mlp_param_count(0) == 0 and L.sgtp_mlp_param_count(129) == 0
    assert L.sgtp_mlp_param_count(60) == 64 * 256 + 256 + 2 * (256 * 256 + 256) + 240 * 256 + 240
    m = C.c_void_p()
    assert L.sgtp_mlp_create(0, 0, None, C.byref(m)) == 1 and not m.value
    assert L.sgtp_mlp_reserve(None, 16) == 1
    assert L.sgtp_mlp_forward(None, vp(16), 4, vp(16), None) == 1
    assert L.sgtp_ibr_plan_learned(None, 0, C.byref(P), 2, vp(16), vp(16), vp(16), 10, 10, 1, 0, 0, 0, None, 0,
                                   vp(16), vp(16), None, None, None, None, vp(16), None, vp(256), 1 << 20, None) == 1
    # GA-IBR-MPPI: the temperature must be finite and > 0
    for lam in (0.0, -2.0, float("inf"), float("nan")):
        st = L.sgtp_ibr_plan_mppi(None, 0, C.byref(P), 2, vp(16), vp(16), vp(16), 10, 10, 1, 0, 0, 0, lam, vp(16),
                                  vp(16), None, None, vp(16), None, vp(256), 1 << 20, None)
        assert st == 1 and b"lambda" in L.sgtp_last_error()
        assert L.sgtp_batch_plan_mppi(None, C.byref(P), lam, None, None, None, 0, None, None, None, None, None,
                                      None, None, 0, None) == 1
    assert L.sgtp_ibr_plan_mppi(None, 0, C.byref(P), 2, vp(16), vp(16), vp(16), 10, 10, 1, 0, 0, 0, 1.0, vp(16),
                                vp(16), None, None, vp(16), None, vp(256), 1 << 20, None) == 1
    assert b"track" in L.sgtp_last_error()
    # closed-loop simulation: NULL batch
    sp = _lib.SimParams(1, 10, 0, 5, 4.5, 0.0, 5.0, 2.5)
    assert L.sgtp_sim_reset(None, vp(16), vp(256), None) == 1 and b"batch" in L.sgtp_last_error()
    assert L.sgtp_sim_step(None, C.byref(P), C.byref(sp), vp(16), vp(16), vp(16), vp(256), None) == 1
    # bad params
    bad = _params(); bad.dt = -1.0
    assert L.sgtp_batch_plan(None, C.byref(bad), None, None, None, 0, None, None, None, None, None, None, None, 0,
                             None) == 1
    assert L.sgtp_launch_count() == n0


def test_tail_count_rule_matches_oracle():
    import oracle as O
    for mu in (0.3, 0.25, 0.1, 0.5, 1.0, 0.01):
        for H in (1, 4, 12, 30, 50, 60, 80, 128):
            # host rule of the library restated from include/sgtp.h's reading
            v = float(np.float32(mu)) * H - 1e-4
            n = min(H, max(1, int(np.ceil(v))))
            assert O.tail_count(mu, H) == n


def test_sim_structs_match_the_header(tmp_path):
    """Sizes and offsets of sgtp_sim_params / sgtp_sim_race as a C compiler
    lays them out from include/sgtp.h equal the binding's mirrors."""
    import os
    import subprocess
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "probe.c"
    fields = [f for f, _ in _lib.SimRace._fields_]
    body = "".join(f'printf("%zu ", offsetof(sgtp_sim_race, {f}));' for f in fields)
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "sgtp.h"\nint main(void){'
                   'printf("%zu %zu ", sizeof(sgtp_sim_params), sizeof(sgtp_sim_race));' + body + 'return 0;}\n')
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got[0] == C.sizeof(_lib.SimParams) and got[1] == C.sizeof(_lib.SimRace)
    assert got[2:] == [getattr(_lib.SimRace, f).offset for f in fields]
