"""ctypes declarations of the C ABI in ``include/finrl_gb300.h``.

Loading fails loudly when ``libfinrl_gb300.so`` has not been built: there is
no CPU fallback for anything the library computes.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfinrl_gb300.so")

FR_OK, FR_EINVAL, FR_ENOMEM, FR_EBUSY, FR_ETIMEDOUT, FR_ECUDA, FR_ENOTREADY, FR_ENOTFOUND = (
    0, -1, -2, -3, -4, -5, -6, -7)
FR_ECANCELED = -8
TASK_STOCK, TASK_CRYPTO = 0, 1
ACT_I32_SHARES, ACT_F32_UNIT, ACT_U8_DISCRETE = 0, 1, 2
PREC_FP32, PREC_BF16, PREC_FP8, PREC_BF16X3, PREC_FP16 = 0, 1, 2, 3, 4
COMBINE_MEAN, COMBINE_VOTE = 0, 1
HEAD_Q, HEAD_DUELING = 0, 1
PATH_AUTO, PATH_UNFUSED = 0, 1
BUY_ASCENDING, BUY_LARGEST_FIRST = 0, 1
FAULT_ALLOC, FAULT_SUBMIT, FAULT_POLL = 1, 2, 3

i32, i64, u32, u64, f64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
vp, cp = C.c_void_p, C.c_char_p
size_t = C.c_size_t


class MarketDesc(C.Structure):
    _fields_ = [("task", i32), ("n_days", i32), ("n_assets", i32), ("n_ind", i32),
                ("close", vp), ("ind", vp), ("n_seconds", i64), ("mid", vp),
                ("spread", vp), ("fac", vp), ("high", vp), ("low", vp)]


class TuneReport(C.Structure):
    _fields_ = [("n", i32), ("chosen", i32), ("cached", i32), ("path", i32 * 8), ("packed", i32 * 8),
                ("stages", i32 * 8), ("tiled", i32 * 8), ("ms", C.c_float * 8)]


class EnvDesc(C.Structure):
    _fields_ = [("task", i32), ("n_envs", i32), ("n_assets", vp), ("window", vp),
                ("start", vp), ("bps", vp), ("init_cash", i64), ("hmax", i32),
                ("fee_bps", i32), ("pmax", i32), ("auto_reset", i32), ("buy_order", i32)]


class Action(C.Structure):
    _fields_ = [("kind", i32), ("data", vp)]


class StepOut(C.Structure):
    _fields_ = [("rew", vp), ("rew_f32", vp), ("done", vp), ("obs", vp)]


class EnsembleDesc(C.Structure):
    _fields_ = [("n_agents", i32), ("n_layers", i32), ("dims", vp), ("params", vp),
                ("weights", vp), ("precision", i32), ("combine", i32), ("out_act", i32), ("heads", vp)]


class Traj(C.Structure):
    _fields_ = [("obs", vp), ("obs_ld", i32), ("act", vp), ("rew", vp), ("rew_f32", vp),
                ("done", vp)]


class Explore(C.Structure):
    _fields_ = [("kind", i32), ("sigma", C.c_float), ("eps", C.c_float), ("seed", u64)]


EXPLORE_NONE, EXPLORE_GAUSSIAN, EXPLORE_EPS_GREEDY = 0, 1, 2


class ServerDesc(C.Structure):
    _fields_ = [("market", vp), ("ens", vp), ("capacity", i32), ("chunk_steps", i32),
                ("init_cash", i64), ("hmax", i32), ("fee_bps", i32), ("pmax", i32), ("hbm_budget", u64)]


class Request(C.Structure):
    _fields_ = [("n_envs", i32), ("window", i32), ("start", i32), ("start_stride", i32),
                ("n_assets", i32), ("bps_range", i32), ("seed", u64), ("want_traj", i32),
                ("metrics", vp), ("timeout_s", f64), ("task", i32), ("ens", vp)]


class Result(C.Structure):
    _fields_ = [("status", i32), ("n_envs", i32), ("queue_s", f64), ("latency_s", f64),
                ("task", i32), ("traj_steps", i32), ("traj_bytes", u64)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", u64), ("completed", u64), ("queued", u64), ("running", u64),
                ("env_steps", f64), ("pool_steps", f64), ("busy_s", f64), ("failed", u64),
                ("canceled", u64), ("timed_out", u64), ("bytes_reserved", u64), ("bytes_peak", u64),
                ("budget", u64), ("pools", u64)]


# name -> (restype, argtypes); every symbol the header declares
SIGNATURES = {
    "fr_last_error": (cp, []),
    "fr_version": (cp, []),
    "fr_ctx_create": (i32, [i32, u64, vp]),
    "fr_ctx_destroy": (None, [vp]),
    "fr_ctx_bytes_in_use": (u64, [vp]),
    "fr_ctx_sm_count": (i32, [vp]),
    "fr_market_create": (i32, [vp, vp, vp]),
    "fr_market_destroy": (None, [vp]),
    "env_create": (i32, [vp, vp, vp, vp]),
    "env_destroy": (None, [vp]),
    "env_dims": (i32, [vp, vp, vp, vp]),
    "env_reset": (i32, [vp, vp]),
    "env_step": (i32, [vp, vp, vp, vp]),
    "env_observe": (i32, [vp, vp, i32, vp]),
    "env_get_state": (i32, [vp, vp, vp, vp, vp, vp]),
    "env_metrics": (i32, [vp, vp, vp]),
    "env_snapshot": (i32, [vp, vp, size_t, vp]),
    "env_restore": (i32, [vp, vp, size_t]),
    "env_error_count": (i32, [vp, vp]),
    "ensemble_create": (i32, [vp, vp, vp]),
    "ensemble_destroy": (None, [vp]),
    "ensemble_forward": (i32, [vp, vp, i32, vp, vp]),
    "ensemble_act": (i32, [vp, vp, i32, vp, vp]),
    "ensemble_device_errors": (i32, [vp, vp]),
    "rollout": (i32, [vp, vp, i32, vp, vp, vp]),
    "env_set_rollout_path": (i32, [vp, i32]),
    "ensemble_act_noalloc": (i32, [vp, vp, i32, vp, vp]),
    "env_set_kernel_timing": (i32, [vp, i32]),
    "env_last_kernel_ms": (i32, [vp, vp]),
    "env_last_launch_shape": (i32, [vp, vp, vp]),
    "env_set_exploration": (i32, [vp, vp]),
    "trajectory_metrics": (i32, [vp, vp, i32, i32, i64, f64, f64, vp, vp]),
    "ensemble_set_weights": (i32, [vp, vp]),
    "ensemble_validate": (i32, [vp, vp, i32, f64, vp, vp, vp]),
    "env_set_tile_packing": (i32, [vp, i32]),
    "env_set_table_cache": (i32, [vp, i32]),
    "env_set_rollout_split": (i32, [vp, i32]),
    "env_tile_packing_efficiency": (i32, [vp, vp]),
    "fr_server_create": (i32, [vp, vp, vp]),
    "fr_server_destroy": (None, [vp]),
    "backtest_submit": (i32, [vp, vp, vp]),
    "backtest_poll": (i32, [vp, u64, vp, vp]),
    "backtest_cancel": (i32, [vp, u64]),
    "fr_server_add_pool": (i32, [vp, vp, vp, i32, i32]),
    "backtest_fetch_traj": (i32, [vp, u64, vp, vp]),
    "backtest_release": (i32, [vp, u64]),
    "fr_server_stats_get": (i32, [vp, vp]),
    "fr_fault_inject": (i32, [i32, i32, i32]),
    "fr_wait_selftest": (i32, [vp, i32, vp, vp]),
    "fr_market_copy_indicators": (i32, [vp, vp]),
    "market_indicators": (i32, [vp, vp, vp, i32, i32, vp, vp]),
    "env_perturb": (i32, [vp, u64, i32, vp]),
    "ensemble_set_act_scales": (i32, [vp, vp]),
    "ensemble_get_act_scales": (i32, [vp, vp]),
    "ensemble_calibrate_sync": (i32, [vp, vp, i32, vp]),
    "ensemble_q": (i32, [vp, vp, i32, vp, vp]),
    "ensemble_q_targets": (i32, [vp, vp, vp, vp, vp, i32, C.c_float, i32, vp, vp]),
    "env_autotune": (i32, [vp, vp, i32, i32, vp, vp]),
    "env_tune_clear": (i32, [vp]),
    "env_tune_set": (i32, [vp, i32, i32, i32, i32]),
    "replay_create": (i32, [vp, vp, i64, vp]),
    "replay_destroy": (None, [vp]),
    "replay_push": (i32, [vp, vp, vp, i32, vp, vp, vp]),
    "replay_sample": (i32, [vp, i32, u64, u64, vp, vp, vp, vp, vp, vp, vp]),
    "replay_size_sync": (i32, [vp, vp, vp, vp, vp]),
}

_lock = threading.Lock()
_lib = None


def load():
    """Load the CUDA library (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is not built; run paper_2501_10709_gb300.build.build() "
                "(this package has no CPU fallback)")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class FrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def check(rc: int, what: str = ""):
    if rc != FR_OK:
        msg = load().fr_last_error().decode(errors="replace")
        raise FrError(rc, f"{what}: {msg}" if what else msg)
