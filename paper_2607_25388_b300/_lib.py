"""ctypes declarations of the C ABI in ``include/sgtp.h`` (argument
marshalling only; every step of the path runs in the CUDA library)."""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

PARAM_FIELDS = [
    "dt", "wheelbase", "a_min", "a_max", "delta_max", "v_min", "v_max", "sigma_a", "sigma_delta",
    "Q", "R", "S", "w_game", "w_contest", "w_long", "w_block", "w_safety",
    "s_contest", "s_role", "mu_tail", "g_safe", "eps_alpha", "m_bd", "d_col",
]

MAX_AGENTS = 16
MAX_T = 128
DEBUG_SKIP_BARRIER_ARRIVAL = 1
DEBUG_SKIP_WINNER_SIGNAL = 2

STATUS = {0: "SGTP_OK", 1: "SGTP_E_INVALID", 2: "SGTP_E_CUDA", 3: "SGTP_E_NOMEM", 4: "SGTP_E_TIMEOUT",
          5: "SGTP_E_DEVICE", 6: "SGTP_E_UNSUPPORTED"}


class Params(C.Structure):
    _fields_ = [
        ("dt", C.c_float), ("wheelbase", C.c_float), ("a_min", C.c_float), ("a_max", C.c_float),
        ("delta_max", C.c_float), ("v_min", C.c_float), ("v_max", C.c_float),
        ("sigma_a", C.c_float), ("sigma_delta", C.c_float),
        ("Q", C.c_float * 4), ("R", C.c_float * 2), ("S", C.c_float * 2),
        ("w_game", C.c_float), ("w_contest", C.c_float), ("w_long", C.c_float), ("w_block", C.c_float),
        ("w_safety", C.c_float), ("s_contest", C.c_float), ("s_role", C.c_float), ("mu_tail", C.c_float),
        ("g_safe", C.c_float), ("eps_alpha", C.c_float), ("m_bd", C.c_float), ("d_col", C.c_float),
    ]


class LaunchOpts(C.Structure):
    _fields_ = [("block", C.c_int32), ("samples_per_thread", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("window", C.c_int32), ("wait_timeout_ns", C.c_int64), ("debug_flags", C.c_int32),
                ("schedule", C.c_int32), ("trace_ns", C.c_void_p)]


class Race(C.Structure):
    _fields_ = [("track_id", C.c_int32), ("n_v", C.c_int32), ("T", C.c_int32), ("ego", C.c_int32),
                ("race_tag", C.c_uint32)]


class SimParams(C.Structure):
    _fields_ = [("n_apply", C.c_int32), ("max_steps", C.c_int32), ("tracker", C.c_int32), ("pp_preview", C.c_int32),
                ("contact_dist", C.c_float), ("wall_margin", C.c_float), ("close_ds", C.c_float),
                ("close_dd", C.c_float)]


MAX_AGENTS = 16


class SimRace(C.Structure):
    """Mirror of sgtp_sim_race (include/sgtp.h)."""
    _fields_ = [("alive", C.c_int32), ("steps", C.c_int32), ("ego_collision", C.c_int32),
                ("close_segments", C.c_int32), ("close_steps", C.c_int32), ("ego_speed_sum", C.c_float),
                ("ego_du2_sum", C.c_float), ("pad0", C.c_int32),
                ("progress", C.c_float * MAX_AGENTS), ("rel0", C.c_float * MAX_AGENTS), ("d", C.c_float * MAX_AGENTS),
                ("s_raw", C.c_float * MAX_AGENTS), ("close_run", C.c_int32 * MAX_AGENTS),
                ("u_prev", C.c_float * 2), ("pad1", C.c_int32 * 2)]


def make_params(d: dict) -> Params:
    P = Params()
    for f in PARAM_FIELDS:
        v = d[f]
        if f in ("Q", "R", "S"):
            arr = getattr(P, f)
            for i, x in enumerate(v):
                arr[i] = float(x)
        else:
            setattr(P, f, float(v))
    return P


def lib():
    """Load libsgtp.so (building it with nvcc when missing or stale).  Raises
    if the library cannot be built or loaded: there is no other path."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            vp, sz, i32, u32, u64, f32 = C.c_void_p, C.c_size_t, C.c_int32, C.c_uint32, C.c_uint64, C.c_float
            L.sgtp_track_create.argtypes = [vp, vp, vp, i32, vp, C.POINTER(vp)]
            L.sgtp_track_create_many.argtypes = [vp, vp, vp, vp, i32, vp, C.POINTER(vp)]
            L.sgtp_track_destroy.argtypes = [vp]
            L.sgtp_track_destroy.restype = None
            L.sgtp_track_info.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(f32)]
            L.sgtp_br_workspace_bytes.argtypes = [i32, i32]
            L.sgtp_br_workspace_bytes.restype = sz
            L.sgtp_rollout_costs.argtypes = [vp, i32, C.POINTER(Params), vp, vp, f32, vp, i32, i32, i32, u64, u32,
                                             u32, u32, i32, vp, vp, vp, vp, vp, vp, vp, sz, vp]
            L.sgtp_best_response.argtypes = [vp, i32, C.POINTER(Params), vp, vp, f32, vp, i32, i32, i32, u64, u32,
                                             u32, u32, i32, vp, vp, vp, vp, vp, sz, vp]
            L.sgtp_best_response_noalloc.argtypes = [vp, i32, C.POINTER(Params), vp, vp, f32, vp, i32, i32, i32,
                                                     u64, u32, u32, u32, i32, vp, vp, vp, vp, vp]
            L.sgtp_sync_status.argtypes = [vp, vp, C.POINTER(i32)]
            L.sgtp_last_error.restype = C.c_char_p
            L.sgtp_version.restype = C.c_char_p
            L.sgtp_launch_count.restype = C.c_int64
            L.sgtp_debug_fail_alloc.argtypes = [i32]
            L.sgtp_debug_fail_alloc.restype = None
            L.sgtp_fma_probe.argtypes = [i32, i32, i32, vp, vp, C.POINTER(C.c_double)]
            L.sgtp_philox_words.argtypes = [u64, u32, u32, u32, u32, i32, vp, vp, vp]
            L.sgtp_noise_normals.argtypes = [u64, u32, u32, u32, u32, u32, i32, i32, vp, vp]
            if hasattr(L, "sgtp_plan_workspace_bytes"):
                L.sgtp_plan_workspace_bytes.argtypes = [i32, i32, i32]
                L.sgtp_plan_workspace_bytes.restype = sz
                L.sgtp_ibr_plan.argtypes = [vp, i32, C.POINTER(Params), i32, vp, vp, vp, i32, i32, i32, i32, u64,
                                            u32, vp, vp, vp, vp, vp, C.POINTER(LaunchOpts), vp, sz, vp]
                L.sgtp_batch_create.argtypes = [vp, C.POINTER(Race), i32, i32, i32, C.POINTER(vp)]
                L.sgtp_batch_destroy.argtypes = [vp]
                L.sgtp_batch_destroy.restype = None
                L.sgtp_batch_sizes.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                               C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(sz)]
                L.sgtp_batch_plan.argtypes = [vp, C.POINTER(Params), vp, vp, vp, u64, vp, vp, vp, vp, vp,
                                              C.POINTER(LaunchOpts), vp, sz, vp]
            L.sgtp_plan_mppi_workspace_bytes.argtypes = [i32, i32, i32, i32]
            L.sgtp_plan_mppi_workspace_bytes.restype = sz
            L.sgtp_ibr_plan_mppi.argtypes = [vp, i32, C.POINTER(Params), i32, vp, vp, vp, i32, i32, i32, i32, u64,
                                             u32, f32, vp, vp, vp, vp, vp, C.POINTER(LaunchOpts), vp, sz, vp]
            L.sgtp_batch_mppi_workspace_bytes.argtypes = [vp, C.POINTER(sz)]
            L.sgtp_batch_plan_mppi.argtypes = [vp, C.POINTER(Params), f32, vp, vp, vp, u64, vp, vp, vp, vp, vp,
                                               C.POINTER(LaunchOpts), vp, sz, vp]
            L.sgtp_ibr_plan_perturbed.argtypes = [vp, i32, C.POINTER(Params), i32, vp, vp, vp, i32, i32, i32, i32,
                                                  u64, u32, f32, f32, vp, vp, vp, vp, vp, C.POINTER(LaunchOpts), vp,
                                                  sz, vp]
            L.sgtp_batch_plan_perturbed.argtypes = [vp, C.POINTER(Params), f32, f32, vp, vp, vp, u64, vp, vp, vp, vp,
                                                    vp, C.POINTER(LaunchOpts), vp, sz, vp]
            L.sgtp_sim_reset.argtypes = [vp, vp, vp, vp]
            L.sgtp_sim_step.argtypes = [vp, C.POINTER(Params), C.POINTER(SimParams), vp, vp, vp, vp, vp]
            L.sgtp_graph_capture_plan.argtypes = [vp, i32, C.POINTER(Params), i32, vp, vp, vp, i32, i32, i32, i32,
                                                  u64, u32, vp, vp, vp, vp, vp, C.POINTER(LaunchOpts), vp, sz,
                                                  C.POINTER(vp)]
            L.sgtp_graph_capture_batch.argtypes = [vp, C.POINTER(Params), vp, vp, vp, u64, vp, vp, vp, vp, vp,
                                                   C.POINTER(LaunchOpts), vp, sz, C.POINTER(vp)]
            L.sgtp_graph_set_seed.argtypes = [vp, u64]
            L.sgtp_graph_launch.argtypes = [vp, vp]
            L.sgtp_graph_destroy.argtypes = [vp]
            L.sgtp_graph_destroy.restype = None
            # learned proposal (include/sgtp_mlp.h)
            L.sgtp_mlp_param_count.argtypes = [i32]
            L.sgtp_mlp_param_count.restype = sz
            L.sgtp_mlp_create.argtypes = [i32, u64, vp, C.POINTER(vp)]
            L.sgtp_mlp_destroy.argtypes = [vp]
            L.sgtp_mlp_destroy.restype = None
            L.sgtp_mlp_reserve.argtypes = [vp, i32]
            L.sgtp_mlp_forward.argtypes = [vp, vp, i32, vp, vp]
            L.sgtp_mlp_proposal.argtypes = [vp, vp, vp, i32, f32, f32, vp, vp]
            L.sgtp_mlp_train_step.argtypes = [vp, vp, vp, i32, f32, vp, vp, i32, vp]
            L.sgtp_mlp_get_params.argtypes = [vp, vp]
            L.sgtp_mlp_set_params.argtypes = [vp, vp]
            L.sgtp_mlp_info.argtypes = [vp, C.POINTER(i32), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                        C.POINTER(vp)]
            L.sgtp_best_response_mixed.argtypes = [vp, i32, C.POINTER(Params), vp, vp, f32, vp, i32, i32, i32,
                                                   u64, u32, u32, u32, i32, vp, i32, vp, vp, vp, vp, vp, vp, sz,
                                                   vp]
            L.sgtp_batch_plan_learned.argtypes = [vp, C.POINTER(Params), vp, i32, vp, vp, vp, u64, vp, vp, vp, vp,
                                                  vp, vp, vp, C.POINTER(LaunchOpts), vp, sz, vp]
            L.sgtp_ibr_plan_learned.argtypes = [vp, i32, C.POINTER(Params), i32, vp, vp, vp, i32, i32, i32, i32,
                                                u64, u32, vp, i32, vp, vp, vp, vp, vp, vp, vp,
                                                C.POINTER(LaunchOpts), vp, sz, vp]
            _lib = L
    return _lib


def check(status: int, what: str = ""):
    if status != 0:
        msg = lib().sgtp_last_error().decode(errors="replace")
        raise RuntimeError(f"{what}: {STATUS.get(status, status)}: {msg}")


# every symbol include/*.h declares (checked by the CPU test-suite)
EXPORTS = [
    "sgtp_track_create", "sgtp_track_create_many", "sgtp_track_destroy", "sgtp_track_info",
    "sgtp_br_workspace_bytes", "sgtp_rollout_costs", "sgtp_best_response", "sgtp_best_response_noalloc",
    "sgtp_batch_create", "sgtp_batch_destroy", "sgtp_batch_sizes", "sgtp_batch_plan",
    "sgtp_plan_workspace_bytes", "sgtp_ibr_plan",
    "sgtp_graph_capture_plan", "sgtp_graph_capture_batch", "sgtp_graph_set_seed", "sgtp_graph_launch",
    "sgtp_graph_destroy",
    "sgtp_sync_status", "sgtp_last_error", "sgtp_version", "sgtp_launch_count",
    "sgtp_mlp_param_count", "sgtp_mlp_create", "sgtp_mlp_destroy", "sgtp_mlp_reserve", "sgtp_mlp_forward",
    "sgtp_mlp_proposal", "sgtp_mlp_train_step", "sgtp_mlp_get_params", "sgtp_mlp_set_params", "sgtp_mlp_info",
    "sgtp_best_response_mixed", "sgtp_ibr_plan_learned", "sgtp_batch_plan_learned",
    "sgtp_plan_mppi_workspace_bytes", "sgtp_ibr_plan_mppi", "sgtp_batch_mppi_workspace_bytes",
    "sgtp_batch_plan_mppi", "sgtp_sim_reset", "sgtp_sim_step", "sgtp_ibr_plan_perturbed", "sgtp_batch_plan_perturbed",
    "sgtp_fma_probe", "sgtp_philox_words", "sgtp_noise_normals", "sgtp_debug_fail_alloc",
]


def lib_path() -> str:
    return os.path.abspath(_build.LIB)
