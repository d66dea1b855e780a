"""GB300 sampling library for the FinRL stock and crypto trading environments.

A thin Python binding over the C ABI of ``libfinrl_gb300.so`` (declared in
``include/finrl_gb300.h``): every function here only marshals arguments --
numpy arrays for host tables, torch CUDA tensors for device buffers, the
current torch stream -- and calls the library function of the same name.
All computation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (ACT_F32_UNIT, ACT_I32_SHARES, ACT_U8_DISCRETE, BUY_ASCENDING, BUY_LARGEST_FIRST,
                   COMBINE_MEAN, FAULT_ALLOC, FAULT_POLL, FAULT_SUBMIT, HEAD_DUELING, HEAD_Q,
                   COMBINE_VOTE, PATH_AUTO, PATH_UNFUSED, PREC_BF16, PREC_BF16X3, PREC_FP16, PREC_FP8,
                   PREC_FP32, TASK_CRYPTO, TASK_STOCK, FrError)

__all__ = [
    "fr_ctx_create", "fr_market_create", "env_create", "env_reset", "env_step",
    "env_observe", "env_get_state", "env_metrics", "env_snapshot", "env_restore",
    "env_error_count", "env_dims", "ensemble_create", "ensemble_forward",
    "ensemble_act", "ensemble_act_noalloc", "ensemble_device_errors", "rollout", "env_set_rollout_path", "env_set_kernel_timing", "env_last_kernel_ms", "env_last_launch_shape", "env_set_tile_packing", "env_set_table_cache", "env_set_rollout_split",
    "env_tile_packing_efficiency", "ensemble_set_weights", "ensemble_validate", "trajectory_metrics", "env_set_exploration",
    "EXPLORE_NONE", "EXPLORE_GAUSSIAN", "EXPLORE_EPS_GREEDY", "Server", "fr_server_create", "backtest_submit",
    "backtest_poll", "backtest_cancel", "fr_server_stats", "fr_server_add_pool", "backtest_fetch_traj",
    "backtest_release", "FrError", "lib", "market_indicators", "fr_market_indicators",
    "env_perturb", "ensemble_set_act_scales", "ensemble_get_act_scales", "ensemble_calibrate_sync",
    "Replay", "replay_create", "replay_push", "replay_sample", "replay_size", "ensemble_q", "ensemble_q_targets",
    "HEAD_Q", "HEAD_DUELING", "env_autotune", "env_tune_clear", "env_tune_set",
    "PATH_AUTO", "PATH_UNFUSED", "BUY_ASCENDING", "BUY_LARGEST_FIRST",
    "fr_fault_inject", "FAULT_ALLOC", "FAULT_SUBMIT", "FAULT_POLL", "fr_wait_selftest",
    "ACT_I32_SHARES", "ACT_F32_UNIT", "ACT_U8_DISCRETE", "PREC_FP32", "PREC_BF16",
    "PREC_FP8", "PREC_BF16X3", "PREC_FP16", "COMBINE_MEAN", "COMBINE_VOTE", "TASK_STOCK", "TASK_CRYPTO",
]


def lib():
    return _lib.load()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t, dtype=None, numel=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")
    return t.data_ptr()


def _hptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _Handle:
    _destroy = None

    def __init__(self, ptr, keep=()):
        self.ptr = ptr
        self._keep = keep

    def close(self):
        if self.ptr:
            getattr(lib(), self._destroy)(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return self.ptr


class Ctx(_Handle):
    _destroy = "fr_ctx_destroy"

    @property
    def bytes_in_use(self) -> int:
        return int(lib().fr_ctx_bytes_in_use(self.ptr))

    @property
    def sm_count(self) -> int:
        return int(lib().fr_ctx_sm_count(self.ptr))


class Market(_Handle):
    _destroy = "fr_market_destroy"


class Env(_Handle):
    _destroy = "env_destroy"


class Ensemble(_Handle):
    _destroy = "ensemble_destroy"


def fr_ctx_create(device: int = 0, hbm_budget_bytes: int = 0) -> Ctx:
    out = C.c_void_p()
    _lib.check(lib().fr_ctx_create(int(device), int(hbm_budget_bytes), C.byref(out)), "fr_ctx_create")
    return Ctx(out.value)


def fr_market_create(ctx: Ctx, market, *, device_indicators: bool = False) -> Market:
    """market: an object with close/high/low and optionally an indicator
    table ind (stock), or mid/spread/fac (crypto).  A stock market without
    ind, or with device_indicators, gets its 8 indicators computed on the
    device from close/high/low (market_indicators)."""
    d = _lib.MarketDesc()
    keep = []
    if hasattr(market, "close"):
        device_indicators = device_indicators or getattr(market, "ind", None) is None
        close = np.ascontiguousarray(market.close, np.int64)
        d.task, d.n_days, d.n_assets = TASK_STOCK, close.shape[0], close.shape[1]
        d.close = _hptr(close)
        keep.append(close)
        if device_indicators:
            high = np.ascontiguousarray(market.high, np.int64)
            low = np.ascontiguousarray(market.low, np.int64)
            keep += [high, low]
            d.n_ind, d.high, d.low = 8, _hptr(high), _hptr(low)
        else:
            ind = np.ascontiguousarray(market.ind, np.float32)
            keep.append(ind)
            d.n_ind, d.ind = ind.shape[1], _hptr(ind)
    else:
        mid = np.ascontiguousarray(market.mid, np.int64)
        spread = np.ascontiguousarray(market.spread, np.uint8)
        fac = np.ascontiguousarray(market.fac, np.float32)
        keep += [mid, spread, fac]
        d.task, d.n_seconds = TASK_CRYPTO, mid.size
        d.mid, d.spread, d.fac = _hptr(mid), _hptr(spread), _hptr(fac)
    out = C.c_void_p()
    _lib.check(lib().fr_market_create(ctx, C.byref(d), C.byref(out)), "fr_market_create")
    m = Market(out.value, keep=(ctx,))
    m.task = d.task
    if d.task == TASK_STOCK:
        m.shape_ind = (d.n_days, d.n_ind, d.n_assets)
    return m


def fr_market_indicators(market: Market) -> np.ndarray:
    """A stock market's resident indicator table, float32 [n_days][n_ind][K]."""
    out = np.empty(market.shape_ind, np.float32)
    _lib.check(lib().fr_market_copy_indicators(market, _hptr(out)), "fr_market_copy_indicators")
    return out


def market_indicators(close, high, low, out=None, stream=None):
    """The 8 technical indicators from device int64 close/high/low [T][K]
    -> float32 [T][8][K] on the device."""
    import torch
    T, K = close.shape
    if out is None:
        out = torch.empty(T, 8, K, dtype=torch.float32, device=close.device)
    _lib.check(lib().market_indicators(_dptr(close, torch.int64, T * K, "close"),
                                       _dptr(high, torch.int64, T * K, "high"),
                                       _dptr(low, torch.int64, T * K, "low"), int(T), int(K),
                                       _dptr(out, torch.float32, T * 8 * K, "out"), _stream(stream)),
               "market_indicators")
    return out


def env_perturb(env: Env, seed: int, bps_range: int = 100, stream=None):
    """Draw the env batch's per-env, per-asset price perturbations on the
    device (uniform in [-bps_range, bps_range] basis points, SplitMix64)."""
    _lib.check(lib().env_perturb(env, C.c_uint64(int(seed) & (2**64 - 1)), int(bps_range), _stream(stream)),
               "env_perturb")


def env_create(ctx: Ctx, market: Market, *, start, window, n_assets=None, bps=None,
               init_cash: int = 100_000_000, hmax: int = 100, fee_bps: int = 10,
               pmax: int = 10, auto_reset: bool = False, buy_order: int = 0) -> Env:
    """buy_order (stock): BUY_ASCENDING fills a step's buys in ascending asset
    order, BUY_LARGEST_FIRST largest requested count first (equal counts in
    ascending asset order)."""
    start = np.ascontiguousarray(start, np.int32)
    window = np.ascontiguousarray(np.broadcast_to(window, start.shape), np.int32)
    na = None if n_assets is None else np.ascontiguousarray(np.broadcast_to(n_assets, start.shape), np.int32)
    b = None if bps is None else np.ascontiguousarray(bps, np.int16)
    d = _lib.EnvDesc(task=market.task, n_envs=start.size, n_assets=_hptr(na), window=_hptr(window),
                     start=_hptr(start), bps=_hptr(b), init_cash=int(init_cash), hmax=int(hmax),
                     fee_bps=int(fee_bps), pmax=int(pmax), auto_reset=int(bool(auto_reset)),
                     buy_order=int(buy_order))
    out = C.c_void_p()
    _lib.check(lib().env_create(ctx, C.byref(d), market, C.byref(out)), "env_create")
    env = Env(out.value, keep=(ctx, market))
    env.N, env.D, env.K = env_dims(env)
    env.task = market.task
    return env


def env_dims(env: Env):
    n, d, k = C.c_int32(), C.c_int32(), C.c_int32()
    _lib.check(lib().env_dims(env, C.byref(n), C.byref(d), C.byref(k)), "env_dims")
    return n.value, d.value, k.value


def env_reset(env: Env, stream=None):
    _lib.check(lib().env_reset(env, _stream(stream)), "env_reset")


def env_step(env: Env, action, kind: int, *, rew=None, rew_f32=None, done=None, obs=None,
             stream=None):
    import torch
    a = _lib.Action(kind=int(kind), data=_dptr(action, name="action"))
    o = _lib.StepOut(rew=_dptr(rew, torch.int64, env.N, "rew"),
                     rew_f32=_dptr(rew_f32, torch.float32, env.N, "rew_f32"),
                     done=_dptr(done, torch.uint8, env.N, "done"),
                     obs=_dptr(obs, torch.float32, env.N * env.D, "obs"))
    _lib.check(lib().env_step(env, C.byref(a), C.byref(o), _stream(stream)), "env_step")


def env_observe(env: Env, obs, ld: int | None = None, stream=None):
    import torch
    ld = ld or env.D
    _lib.check(lib().env_observe(env, _dptr(obs, torch.float32, env.N * ld, "obs"), int(ld),
                                 _stream(stream)), "env_observe")


def env_get_state(env: Env, cash=None, hold=None, steps=None, done=None, stream=None):
    import torch
    _lib.check(lib().env_get_state(env, _dptr(cash, torch.int64, env.N, "cash"),
                                   _dptr(hold, torch.int32, env.N * env.K, "hold"),
                                   _dptr(steps, torch.int32, env.N, "steps"),
                                   _dptr(done, torch.uint8, env.N, "done"), _stream(stream)),
               "env_get_state")


def env_metrics(env: Env, metrics, stream=None):
    import torch
    _lib.check(lib().env_metrics(env, _dptr(metrics, torch.float64, env.N * 3, "metrics"),
                                 _stream(stream)), "env_metrics")


def env_snapshot(env: Env) -> bytes:
    n = C.c_size_t()
    _lib.check(lib().env_snapshot(env, None, 0, C.byref(n)), "env_snapshot")
    buf = C.create_string_buffer(n.value)
    _lib.check(lib().env_snapshot(env, buf, n.value, C.byref(n)), "env_snapshot")
    return buf.raw[:n.value]


def env_restore(env: Env, blob):
    """blob: the bytes env_snapshot returned, or a contiguous CPU uint8
    tensor holding them (page-locked memory copies to the device faster)."""
    if not isinstance(blob, bytes):
        import torch
        if (not isinstance(blob, torch.Tensor) or blob.device.type != "cpu" or blob.dtype != torch.uint8
                or not blob.is_contiguous()):
            raise ValueError("env_restore: the snapshot must be bytes or a contiguous CPU uint8 tensor")
        _lib.check(lib().env_restore(env, C.c_void_p(blob.data_ptr()), blob.numel()), "env_restore")
        return
    _lib.check(lib().env_restore(env, blob, len(blob)), "env_restore")


def env_set_rollout_path(env: Env, path: int):
    _lib.check(lib().env_set_rollout_path(env, int(path)), "env_set_rollout_path")


def env_set_rollout_split(env: Env, on: bool):
    _lib.check(lib().env_set_rollout_split(env, 1 if on else 0), "env_set_rollout_split")


def env_set_table_cache(env: Env, on: bool):
    """Keep the fused stock kernel's indicator table across rollouts (on, the
    default) or rebuild it in every rollout (off)."""
    _lib.check(lib().env_set_table_cache(env, 1 if on else 0), "env_set_table_cache")


def env_set_tile_packing(env: Env, on: bool):
    _lib.check(lib().env_set_tile_packing(env, 1 if on else 0), "env_set_tile_packing")


def env_tile_packing_efficiency(env: Env) -> float:
    e = C.c_float()
    _lib.check(lib().env_tile_packing_efficiency(env, C.byref(e)), "env_tile_packing_efficiency")
    return e.value


def env_set_kernel_timing(env: Env, on: bool):
    _lib.check(lib().env_set_kernel_timing(env, 1 if on else 0), "env_set_kernel_timing")


def env_last_kernel_ms(env: Env) -> float:
    ms = C.c_float()
    _lib.check(lib().env_last_kernel_ms(env, C.byref(ms)), "env_last_kernel_ms")
    return ms.value


def env_last_launch_shape(env: Env) -> tuple:
    """(thread blocks, envs per tile) of the env's last fused stock rollout."""
    ctas, tile = C.c_int32(), C.c_int32()
    _lib.check(lib().env_last_launch_shape(env, C.byref(ctas), C.byref(tile)), "env_last_launch_shape")
    return ctas.value, tile.value


def env_error_count(env: Env) -> int:
    c = C.c_uint64()
    _lib.check(lib().env_error_count(env, C.byref(c)), "env_error_count")
    return c.value


def ensemble_create(ctx: Ctx, dims, params, *, weights=None, precision: int = PREC_FP32,
                    combine: int = COMBINE_MEAN, out_act: int = 1, heads=None) -> Ensemble:
    """heads: per-agent HEAD_Q / HEAD_DUELING (VOTE ensembles), None = all HEAD_Q."""
    dims = np.ascontiguousarray(dims, np.int32)
    params = np.ascontiguousarray(params, np.float32)
    w = None if weights is None else np.ascontiguousarray(weights, np.float32)
    hd = None if heads is None else np.ascontiguousarray(heads, np.int32)
    d = _lib.EnsembleDesc(n_agents=params.shape[0], n_layers=dims.size - 1, dims=_hptr(dims),
                          params=_hptr(params), weights=_hptr(w), precision=int(precision),
                          combine=int(combine), out_act=int(out_act), heads=_hptr(hd))
    out = C.c_void_p()
    _lib.check(lib().ensemble_create(ctx, C.byref(d), C.byref(out)), "ensemble_create")
    e = Ensemble(out.value, keep=(ctx,))
    e.M, e.dims, e.combine, e.precision = params.shape[0], tuple(int(x) for x in dims), combine, precision
    e.heads = [HEAD_Q] * e.M if hd is None else [int(x) for x in hd]
    e.n_act = e.dims[-1] - (1 if HEAD_DUELING in e.heads else 0)
    return e


def ensemble_q(ens: Ensemble, obs, q=None, stream=None):
    """Per-agent Q-values after the heads, device float [M][n][n_act]."""
    import torch
    n = obs.shape[0]
    if q is None:
        q = torch.empty(ens.M, n, ens.n_act, device=obs.device)
    _lib.check(lib().ensemble_q(ens, _dptr(obs, torch.float32, n * ens.dims[0], "obs"), n,
                                _dptr(q, torch.float32, ens.M * n * ens.n_act, "q"), _stream(stream)), "ensemble_q")
    return q


def ensemble_q_targets(online: Ensemble, target: Ensemble, next_obs, rew, done=None, *, gamma: float = 0.99,
                       double_q: bool = True, y=None, stream=None):
    """DQN (double_q False) or Double DQN learning targets [M][n] from replay samples."""
    import torch
    n = next_obs.shape[0]
    if y is None:
        y = torch.empty(online.M, n, device=next_obs.device)
    _lib.check(lib().ensemble_q_targets(online, target, _dptr(next_obs, torch.float32, n * online.dims[0], "next_obs"),
                                        _dptr(rew, torch.float32, n, "rew"), _dptr(done, torch.uint8, n, "done"),
                                        n, float(gamma), 1 if double_q else 0,
                                        _dptr(y, torch.float32, online.M * n, "y"), _stream(stream)),
               "ensemble_q_targets")
    return y


def ensemble_set_act_scales(ens: Ensemble, scales):
    """FP8 ensembles: static activation scales, host float [M][L]."""
    sc = np.ascontiguousarray(scales, np.float32).reshape(ens.M, len(ens.dims) - 1)
    _lib.check(lib().ensemble_set_act_scales(ens, _hptr(sc)), "ensemble_set_act_scales")


def ensemble_get_act_scales(ens: Ensemble) -> np.ndarray:
    out = np.empty((ens.M, len(ens.dims) - 1), np.float32)
    _lib.check(lib().ensemble_get_act_scales(ens, _hptr(out)), "ensemble_get_act_scales")
    return out


def ensemble_calibrate_sync(ens: Ensemble, obs, stream=None) -> np.ndarray:
    """FP8 ensembles: activation scales max |x| / 448 per agent and layer over
    the calibration batch obs (device [n][dims[0]]); returns them."""
    import torch
    n = obs.shape[0]
    _lib.check(lib().ensemble_calibrate_sync(ens, _dptr(obs, torch.float32, n * ens.dims[0], "obs"), n,
                                             _stream(stream)), "ensemble_calibrate_sync")
    return ensemble_get_act_scales(ens)


def ensemble_forward(ens: Ensemble, obs, y, stream=None):
    import torch
    n = obs.shape[0]
    _lib.check(lib().ensemble_forward(ens, _dptr(obs, torch.float32, n * ens.dims[0], "obs"), n,
                                      _dptr(y, torch.float32, ens.M * n * ens.dims[-1], "y"),
                                      _stream(stream)), "ensemble_forward")


def ensemble_act(ens: Ensemble, obs, act, stream=None):
    import torch
    n = obs.shape[0]
    want = (torch.float32, n * ens.dims[-1]) if ens.combine == COMBINE_MEAN else (torch.uint8, n)
    _lib.check(lib().ensemble_act(ens, _dptr(obs, torch.float32, n * ens.dims[0], "obs"), n,
                                  _dptr(act, *want, "act"), _stream(stream)), "ensemble_act")


def ensemble_act_noalloc(ens: Ensemble, obs, act, stream=None):
    """ensemble_act on the library's fixed scratch array (no allocation).
    For callers that cannot allocate device memory while they run; calls that
    overlap on the GPU share the scratch and must be serialised."""
    import torch
    n = obs.shape[0]
    want = (torch.float32, n * ens.dims[-1]) if ens.combine == COMBINE_MEAN else (torch.uint8, n)
    _lib.check(lib().ensemble_act_noalloc(ens, _dptr(obs, torch.float32, n * ens.dims[0], "obs"), n,
                                          _dptr(act, *want, "act"), _stream(stream)),
               "ensemble_act_noalloc")


def ensemble_device_errors(ens: Ensemble) -> int:
    f = C.c_uint32()
    _lib.check(lib().ensemble_device_errors(ens, C.byref(f)), "ensemble_device_errors")
    return f.value


def rollout(env: Env, ens: Ensemble, T: int, *, traj: dict | None = None, metrics=None,
            stream=None):
    """traj: optional dict of device tensors obs [T][N][ld], act, rew, rew_f32, done."""
    import torch
    tp = C.byref(_traj_struct(env, T, traj)) if traj else None
    _lib.check(lib().rollout(env, ens, int(T), tp,
                             _dptr(metrics, torch.float64, env.N * 3, "metrics"),
                             _stream(stream)), "rollout")


# ---------------------------------------------------------------- autotuner
def env_autotune(env: Env, ens: Ensemble, T_probe: int = 16, *, force: bool = False, stream=None) -> dict:
    """Time the launch configurations for this env / ensemble pair on the
    env's own state (restored afterwards) and keep the fastest; returns the
    report: candidates (path, packed, stages, tiled, ms), chosen, cached."""
    r = _lib.TuneReport()
    _lib.check(lib().env_autotune(env, ens, int(T_probe), 1 if force else 0, C.byref(r), _stream(stream)),
               "env_autotune")
    cands = [dict(path=r.path[i], packed=r.packed[i], stages=r.stages[i], tiled=r.tiled[i], ms=r.ms[i])
             for i in range(r.n)]
    return {"candidates": cands, "chosen": r.chosen, "cached": bool(r.cached)}


def env_tune_set(env: Env, path: int, packed: bool = True, stages: int = 0, tiled: bool = True):
    """Pin one launch configuration (see env_autotune's candidates)."""
    _lib.check(lib().env_tune_set(env, int(path), 1 if packed else 0, int(stages), 1 if tiled else 0),
               "env_tune_set")


def env_tune_clear(env: Env):
    _lib.check(lib().env_tune_clear(env), "env_tune_clear")


# ------------------------------------------------------------ replay buffer
class Replay(_Handle):
    """Device-resident FIFO replay buffer of transitions (s, a, r, s', done)."""
    _destroy = "replay_destroy"


def replay_create(ctx: Ctx, env: Env, capacity: int) -> Replay:
    out = C.c_void_p()
    _lib.check(lib().replay_create(ctx, env, int(capacity), C.byref(out)), "replay_create")
    rb = Replay(out.value, keep=(ctx,))
    rb.D, rb.K, rb.task, rb.capacity = env.D, env.K, env.task, int(capacity)
    return rb


def _traj_struct(env, T, traj):
    import torch
    t = _lib.Traj()
    ob = traj.get("obs")
    ld = int(traj.get("obs_ld", ob.shape[-1] if ob is not None else 0))
    t.obs = _dptr(ob, torch.float32, T * env.N * max(ld, 1), "traj obs")
    t.obs_ld = ld
    act = traj.get("act")
    if act is not None:
        if env.task == TASK_STOCK:
            t.act = _dptr(act, torch.float32, T * env.N * env.K, "traj act")
        else:
            t.act = _dptr(act, torch.uint8, T * env.N, "traj act")
    t.rew = _dptr(traj.get("rew"), torch.int64, T * env.N, "traj rew")
    t.rew_f32 = _dptr(traj.get("rew_f32"), torch.float32, T * env.N, "traj rew_f32")
    t.done = _dptr(traj.get("done"), torch.uint8, T * env.N, "traj done")
    return t


def replay_push(rb: Replay, env: Env, traj: dict, T: int, last_obs, live0=None, stream=None):
    """Append the real steps of a T-step trajectory (obs, act, rew_f32, done);
    last_obs: the observation after the rollout, live0: uint8 [N] or None."""
    import torch
    t = _traj_struct(env, T, traj)
    ld = t.obs_ld or env.D
    _lib.check(lib().replay_push(rb, env, C.byref(t), int(T), _dptr(last_obs, torch.float32, env.N * ld, "last_obs"),
                                 _dptr(live0, torch.uint8, env.N, "live0"), _stream(stream)), "replay_push")


def replay_sample(rb: Replay, B: int, seed: int, counter: int = 0, out: dict | None = None, stream=None) -> dict:
    """B uniform draws with replacement: dict of device tensors obs, act,
    rew, next_obs, done, index."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    if out is None:
        out = {"obs": torch.empty(B, rb.D, device=dev), "next_obs": torch.empty(B, rb.D, device=dev),
               "act": (torch.empty(B, rb.K, device=dev) if rb.task == TASK_STOCK
                       else torch.empty(B, dtype=torch.uint8, device=dev)),
               "rew": torch.empty(B, device=dev), "done": torch.empty(B, dtype=torch.uint8, device=dev),
               "index": torch.empty(B, dtype=torch.int64, device=dev)}
    act = out.get("act")
    a_ptr = None if act is None else (_dptr(act, torch.float32, B * rb.K, "act") if rb.task == TASK_STOCK
                                      else _dptr(act, torch.uint8, B, "act"))
    _lib.check(lib().replay_sample(rb, int(B), C.c_uint64(int(seed) & (2**64 - 1)),
                                   C.c_uint64(int(counter) & (2**64 - 1)),
                                   _dptr(out.get("obs"), torch.float32, B * rb.D, "obs"), a_ptr,
                                   _dptr(out.get("rew"), torch.float32, B, "rew"),
                                   _dptr(out.get("next_obs"), torch.float32, B * rb.D, "next_obs"),
                                   _dptr(out.get("done"), torch.uint8, B, "done"),
                                   _dptr(out.get("index"), torch.int64, B, "index"), _stream(stream)),
               "replay_sample")
    return out


def replay_size(rb: Replay, stream=None):
    """(size, pushed, error bits) after the stream's work so far."""
    size, pushed, err = C.c_int64(), C.c_int64(), C.c_uint32()
    _lib.check(lib().replay_size_sync(rb, C.byref(size), C.byref(pushed), C.byref(err), _stream(stream)),
               "replay_size_sync")
    return size.value, pushed.value, err.value


# ------------------------------------------------------------------ serving
class Server(_Handle):
    """Backtest server (continuous batching over pools of env slots)."""
    _destroy = "fr_server_destroy"

    def __init__(self, ptr, keep=(), task=0):
        super().__init__(ptr, keep)
        self.task = task              # the first pool's task (requests default to it)
        self._pending = {}            # ticket -> host metrics buffer the worker writes
        self._shape = {}              # ticket -> (task, n_envs, window, D, K) of kept trajectories

    def close(self):
        super().close()
        self._pending.clear()


def fr_server_create(ctx: Ctx, market: Market, ens: Ensemble, *, capacity: int, chunk_steps: int = 32,
                     init_cash: int = 100_000_000, hmax: int = 100, fee_bps: int = 10,
                     pmax: int = 10, hbm_budget: int = 0) -> Server:
    d = _lib.ServerDesc(market.ptr, ens.ptr, int(capacity), int(chunk_steps), int(init_cash), int(hmax),
                        int(fee_bps), int(pmax), int(hbm_budget))
    out = C.c_void_p()
    _lib.check(lib().fr_server_create(ctx, C.byref(d), C.byref(out)), "fr_server_create")
    return Server(out.value, keep=(ctx, market, ens), task=market.task)


def fr_server_add_pool(srv: Server, market: Market, ens: Ensemble, *, capacity: int, chunk_steps: int = 32):
    """Another pool (market, ensemble) in the same server, e.g. crypto beside stock."""
    _lib.check(lib().fr_server_add_pool(srv, market.ptr, ens.ptr, int(capacity), int(chunk_steps)),
               "fr_server_add_pool")
    srv._keep = tuple(srv._keep) + (market, ens)


def backtest_submit(srv: Server, *, n_envs: int, window: int, start: int, start_stride: int = 0,
                    n_assets: int = 0, bps_range: int = 0, seed: int = 0, timeout_s: float = 0.0,
                    task: int = None, ens: Ensemble = None, want_traj: bool = False) -> int:
    met = np.zeros((int(n_envs), 3), dtype=np.float64)
    task = srv.task if task is None else int(task)
    r = _lib.Request(int(n_envs), int(window), int(start), int(start_stride), int(n_assets),
                     int(bps_range), int(seed) & (2**64 - 1), 1 if want_traj else 0, met.ctypes.data_as(C.c_void_p),
                     float(timeout_s), task, ens.ptr if ens is not None else None)
    t = C.c_uint64()
    _lib.check(lib().backtest_submit(srv, C.byref(r), C.byref(t)), "backtest_submit")
    srv._pending[t.value] = met
    return t.value


def backtest_poll(srv: Server, ticket: int):
    """None while queued or running; else a dict with the request's result
    (status, n_envs, queue_s, latency_s, task, traj_steps, traj_bytes,
    metrics [n_envs][3]).  A kept trajectory (traj_steps > 0) is then
    fetched with backtest_fetch_traj or dropped with backtest_release."""
    res = _lib.Result()
    done = C.c_int32()
    rc = lib().backtest_poll(srv, C.c_uint64(int(ticket)), C.byref(res), C.byref(done))
    if rc == _lib.FR_ENOTREADY:
        return None
    _lib.check(rc, "backtest_poll")
    met = srv._pending.pop(int(ticket))
    if res.traj_steps:
        srv._shape[int(ticket)] = (res.task, res.n_envs, res.traj_steps)
    return {"status": res.status, "n_envs": res.n_envs, "queue_s": res.queue_s,
            "latency_s": res.latency_s, "task": res.task, "traj_steps": res.traj_steps,
            "traj_bytes": res.traj_bytes, "metrics": met}


def backtest_fetch_traj(srv: Server, ticket: int, *, D: int, K: int = 30, device="cuda", stream=None) -> dict:
    """The kept trajectory of a completed request as tensors on `device`
    (obs [T][n][D], act [T][n][K] float (stock) or [T][n] uint8 (crypto), rew
    int64 [T][n], done uint8 [T][n]); the server's copy is freed."""
    import torch
    task, n, T = srv._shape.pop(int(ticket))
    out = {"obs": torch.empty(T, n, D, device=device),
           "act": (torch.empty(T, n, K, device=device) if task == _lib.TASK_STOCK
                   else torch.empty(T, n, dtype=torch.uint8, device=device)),
           "rew": torch.empty(T, n, dtype=torch.int64, device=device),
           "done": torch.empty(T, n, dtype=torch.uint8, device=device)}
    tr = _lib.Traj(out["obs"].data_ptr(), D, out["act"].data_ptr(), out["rew"].data_ptr(), None,
                   out["done"].data_ptr())
    _lib.check(lib().backtest_fetch_traj(srv, C.c_uint64(int(ticket)), C.byref(tr), _stream(stream)),
               "backtest_fetch_traj")
    return out


def backtest_release(srv: Server, ticket: int):
    """Drop a completed request's kept trajectory without copying it."""
    srv._shape.pop(int(ticket), None)
    _lib.check(lib().backtest_release(srv, C.c_uint64(int(ticket))), "backtest_release")


def backtest_cancel(srv: Server, ticket: int):
    """Cancel a queued or running request (its poll then reports status
    FR_ECANCELED); no effect on a complete one."""
    _lib.check(lib().backtest_cancel(srv, C.c_uint64(int(ticket))), "backtest_cancel")


def fr_server_stats(srv: Server) -> dict:
    st = _lib.ServerStats()
    _lib.check(lib().fr_server_stats_get(srv, C.byref(st)), "fr_server_stats_get")
    return {k: getattr(st, k) for k, _ in st._fields_}


def fr_fault_inject(kind: int, skip: int = 0, count: int = 1):
    """Host fault injection for tests: of the next events of `kind`
    (FAULT_ALLOC, FAULT_SUBMIT, FAULT_POLL) the first `skip` proceed and the
    `count` after them fail with the error the real failure returns;
    count 0 disarms the kind."""
    _lib.check(lib().fr_fault_inject(int(kind), int(skip), int(count)), "fr_fault_inject")


def fr_wait_selftest(ctx: Ctx, limit_us: int = 50_000) -> dict:
    """Run the device check of the bounded waits: returns status
    (FR_ETIMEDOUT is the designed outcome), the error bits the waits set and
    the ns each of the two abandoned waits took."""
    flags = C.c_uint32()
    w = (C.c_uint64 * 2)()
    rc = lib().fr_wait_selftest(ctx, int(limit_us), C.byref(flags), w)
    if rc not in (_lib.FR_OK, _lib.FR_ETIMEDOUT):
        _lib.check(rc, "fr_wait_selftest")
    return {"status": rc, "flags": flags.value, "waited_ns": (w[0], w[1])}


# ------------------------------------------------------ ensemble weighting
def ensemble_set_weights(ens: Ensemble, weights):
    w = np.ascontiguousarray(weights, np.float32)
    _lib.check(lib().ensemble_set_weights(ens, _hptr(w)), "ensemble_set_weights")


def ensemble_validate(ens: Ensemble, env: Env, T: int, threshold: float = 0.0, stream=None):
    """Sec. 5.2.1 Sharpe-softmax weights from a validation window; returns
    (sharpe[M] float64, weights[M] float32) and sets the ensemble's weights."""
    M = ens.M
    S = np.zeros(M, np.float64)
    w = np.zeros(M, np.float32)
    _lib.check(lib().ensemble_validate(ens, env, int(T), float(threshold), _hptr(S), _hptr(w), _stream(stream)),
               "ensemble_validate")
    return S, w


def trajectory_metrics(rew, done=None, *, v0: int = 100_000_000, ann: float = 252.0, gamma: float = 0.99,
                       out=None, stream=None):
    """rew [T][N] int64 (device), done [T][N] uint8 or None -> [N][11] float64
    (cumulative return, Sharpe, MDD, annual return, annual volatility, RoMaD,
    Sortino, Calmar, Omega, discounted return, periods)."""
    import torch
    T, N = rew.shape
    if out is None:
        out = torch.empty(N, 11, dtype=torch.float64, device=rew.device)
    _lib.check(lib().trajectory_metrics(_dptr(rew, torch.int64, T * N, "rew"),
                                        _dptr(done, torch.uint8, T * N, "done"), int(T), int(N), int(v0),
                                        float(ann), float(gamma), _dptr(out, torch.float64, N * 11, "out"),
                                        _stream(stream)), "trajectory_metrics")
    return out


EXPLORE_NONE, EXPLORE_GAUSSIAN, EXPLORE_EPS_GREEDY = _lib.EXPLORE_NONE, _lib.EXPLORE_GAUSSIAN, _lib.EXPLORE_EPS_GREEDY


def env_set_exploration(env: Env, kind: int = EXPLORE_NONE, *, sigma: float = 0.0, eps: float = 0.0,
                        seed: int = 0):
    """Exploring rollouts: Gaussian noise on stock actions or epsilon-greedy on
    crypto votes, Philox4x32-10 draws keyed by seed (kind EXPLORE_NONE: off)."""
    x = _lib.Explore(int(kind), float(sigma), float(eps), int(seed) & (2**64 - 1))
    _lib.check(lib().env_set_exploration(env, C.byref(x)), "env_set_exploration")
