"""CPU oracle for the trading environments and ensemble rules -- TEST INFRASTRUCTURE.

This package wraps ``finrl_oracle.c``: a plain, slow fp64 / int64 restatement
of the paper's MDP (Sec. 3.1), its reset/step/reward operations (Sec. 4.2.2),
the two ensemble rules (Sec. 5.2.1 weighted average, Sec. 5.2.2 majority vote)
and the episode metrics (Sharpe equation of Sec. 5.2.1, Sec. 6.1 metric list).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library, and the
CUDA library never imports it.

The shared library is compiled on first use with gcc (``-O2 -fopenmp
-ffp-contract=off``) into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes as C
import hashlib
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "finrl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_lib = None

STOCK_ANNUALISATION = 252.0
CRYPTO_ANNUALISATION = 1.0


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent); returns its path."""
    with open(_SRC, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, f"libfinrl_oracle_{tag}.so")
    if force or not os.path.exists(out):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        i32, i64, f64 = C.c_int32, C.c_int64, C.c_double
        vp = C.c_void_p
        lib.orc_perturb.argtypes = [i64, i32]
        lib.orc_perturb.restype = i64
        lib.orc_fee.argtypes = [i64, i32]
        lib.orc_fee.restype = i64
        lib.orc_buy_cost.argtypes = [i64, i64, i32]
        lib.orc_buy_cost.restype = i64
        lib.orc_buy_max.argtypes = [i64, i64, i32]
        lib.orc_buy_max.restype = i64
        lib.orc_discretise.argtypes = [f64, i32]
        lib.orc_discretise.restype = i32
        lib.orc_discretise_many.argtypes = [vp, i64, i32, vp]
        lib.orc_buy_max_many.argtypes = [vp, vp, vp, i64, vp]
        lib.orc_perturb_many.argtypes = [vp, vp, i64, vp]
        lib.orc_net_param_count.argtypes = [i32, vp]
        lib.orc_net_param_count.restype = i64
        lib.orc_net_forward.argtypes = [i32, vp, vp, i32, vp, i32, i32, vp, i32]
        lib.orc_ensemble_mean.argtypes = [i32, i32, vp, vp, vp]
        lib.orc_argmax.argtypes = [vp, i32]
        lib.orc_argmax.restype = i32
        lib.orc_vote.argtypes = [i32, vp]
        lib.orc_vote.restype = i32
        lib.orc_metrics_series.argtypes = [i32, vp, f64, vp]
        lib.orc_stock_run.argtypes = [i32, i32, i32, vp, vp,
                                      i32, vp, vp, vp, vp,
                                      i64, i32, i32, i32, i32, i32,
                                      vp, vp, i32, i32, vp, vp, vp,
                                      vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, i32]
        lib.orc_stock_run.restype = i32
        lib.orc_crypto_run.argtypes = [i32, vp, vp, vp, i32, vp, vp, i64, i32,
                                       i32, i32, i32, vp, i32, i32, vp, vp,
                                       vp, vp, vp, vp, vp, vp, vp, vp, vp, i32]
        lib.orc_crypto_run.restype = i32
        lib.orc_max_threads.restype = i32
        _lib = lib
        return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


def max_threads() -> int:
    return int(_load().orc_max_threads())


# ------------------------------------------------------------ scalar rules

def perturb(close: int, bps: int) -> int:
    return int(_load().orc_perturb(int(close), int(bps)))


def fee(notional: int, fee_bps: int) -> int:
    return int(_load().orc_fee(int(notional), int(fee_bps)))


def buy_cost(n: int, p: int, fee_bps: int) -> int:
    return int(_load().orc_buy_cost(int(n), int(p), int(fee_bps)))


def buy_max(cash: int, p: int, fee_bps: int) -> int:
    return int(_load().orc_buy_max(int(cash), int(p), int(fee_bps)))


def discretise(a: float, hmax: int) -> int:
    return int(_load().orc_discretise(float(a), int(hmax)))


def discretise_many(a: np.ndarray, hmax: int) -> np.ndarray:
    a = _c(a, np.float32).ravel()
    out = np.empty(a.size, np.int32)
    _load().orc_discretise_many(_p(a), a.size, int(hmax), _p(out))
    return out


def buy_max_many(cash, p, fee_bps) -> np.ndarray:
    cash = _c(cash, np.int64).ravel()
    p = _c(np.broadcast_to(p, cash.shape), np.int64)
    f = _c(np.broadcast_to(fee_bps, cash.shape), np.int32)
    out = np.empty(cash.size, np.int64)
    _load().orc_buy_max_many(_p(cash), _p(p), _p(f), cash.size, _p(out))
    return out


def perturb_many(close, bps) -> np.ndarray:
    close = _c(close, np.int64)
    b = _c(np.broadcast_to(bps, close.shape), np.int32)
    out = np.empty(close.shape, np.int64)
    _load().orc_perturb_many(_p(close), _p(b), close.size, _p(out))
    return out


# ------------------------------------------------------------------ networks

def net_param_count(dims) -> int:
    d = _c(dims, np.int32)
    return int(_load().orc_net_param_count(len(d) - 1, _p(d)))


def net_forward(dims, params: np.ndarray, x: np.ndarray, out_act: int,
                nthreads: int = 0) -> np.ndarray:
    """fp64 forward of one actor.  params: packed fp32 (W_l[out][in], b_l)."""
    d = _c(dims, np.int32)
    params = _c(params, np.float32)
    x = _c(x, np.float32)
    n, ldx = x.shape
    y = np.empty((n, int(d[-1])), np.float64)
    _load().orc_net_forward(len(d) - 1, _p(d), _p(params), int(out_act), _p(x),
                            ldx, n, _p(y), nthreads or max_threads())
    return y


# ------------------------------------------------- DQN-family heads, targets
def head_q(y, head: int, n_act: int) -> np.ndarray:
    """Q-values [..., n_act] from network outputs (float64).  A plain head
    (DQN, Double DQN) reads the first n_act outputs; a dueling head (Wang et
    al., ICML 2016) splits them into V = y_0 and A = y_1 .. y_n_act and
    returns V + A_a - mean_b A_b."""
    y = np.asarray(y, np.float64)
    if head == 0:
        return y[..., :n_act]
    A = y[..., 1:1 + n_act]
    return y[..., :1] + A - A.mean(axis=-1, keepdims=True)


def q_targets(dims, params_online, params_target, heads, next_obs, rew, done, gamma: float,
              double_q: bool) -> np.ndarray:
    """[M][n] float64 learning targets r + (done ? 0 : gamma Q_target(s', a*)):
    a* = argmax Q_online(s') for Double DQN (van Hasselt et al., AAAI 2016),
    argmax Q_target(s') for DQN (Mnih et al., Nature 2015); lowest index on
    ties; Q-values from the fp64 forward through each agent's head."""
    n_act = dims[-1] - (1 if 1 in list(heads) else 0)
    rew = np.asarray(rew, np.float64)
    done = np.zeros(rew.shape, bool) if done is None else np.asarray(done).astype(bool)
    out = []
    for j in range(len(heads)):
        qt = head_q(net_forward(dims, params_target[j], next_obs, 0), heads[j], n_act)
        qs = head_q(net_forward(dims, params_online[j], next_obs, 0), heads[j], n_act) if double_q else qt
        a = qs.argmax(axis=-1)                       # first maximum: lowest index on ties
        out.append(rew + np.where(done, 0.0, gamma * qt[np.arange(len(a)), a]))
    return np.array(out)


# ------------------------------------------------------- FP8 E4M3 actors
# The FP8 option of the actors has no counterpart in the paper (its agents
# run in fp32); these follow the format definition and the library's stated
# quantisation rule, in plain numpy.
E4M3_MAX = 448.0


def e4m3_round(x) -> np.ndarray:
    """Nearest E4M3 value of each element, ties to even, saturating at +-448.

    E4M3 (OCP 8-bit floating point): sign, 4 exponent bits (bias 7), 3
    fraction bits; normal binades 2^-6 .. 2^8 with 8 values each, subnormals
    in steps of 2^-9, largest finite 448, no infinities.  A binade 2^e holds
    multiples of 2^(e-3); below 2^-6 the step stays 2^-9.  Exact in float64."""
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    _, ex = np.frexp(a)                         # a = m 2^ex, 1/2 <= m < 1
    step = np.ldexp(1.0, np.maximum(ex - 1, -6) - 3)
    q = np.minimum(np.rint(a / step) * step, E4M3_MAX)   # rint: ties to even
    return np.copysign(q, x)


def _layers(dims, params):
    """(W_l float32 [out][in], b_l float32 [out]) from packed parameters."""
    params = np.asarray(params, np.float32)
    out, off = [], 0
    for fin, fout in zip(dims[:-1], dims[1:]):
        W = params[off:off + fin * fout].reshape(fout, fin)
        off += fin * fout
        out.append((W, params[off:off + fout]))
        off += fout
    return out


def fp8_weights(W):
    """Per-output-channel E4M3 weights: scale sw[n] = max_k |W[n][k]| / 448
    (1 for a zero row), codes of W[n][k] * (1 / sw[n]); float32 arithmetic.
    Returns (code values float64 [out][in], sw float32 [out])."""
    W = np.asarray(W, np.float32)
    amax = np.abs(W).max(axis=1)
    sw = np.where(amax > 0, amax / np.float32(E4M3_MAX), np.float32(1.0)).astype(np.float32)
    inv = (np.float32(1.0) / sw).astype(np.float32)
    return e4m3_round(W * inv[:, None]), sw


def fp8_forward(dims, params, act_scales, x, out_act: int) -> np.ndarray:
    """One agent's FP8 forward: each layer's input quantised with its static
    scale (codes of x * (1 / sx), float32), the E4M3 dot products summed
    exactly, dequantised by sx * sw[n] (float32 product), bias added in
    float64; ReLU between layers (the next layer quantises the float32 value
    of the activation), tanh or identity on the output.  float64 [n][out]."""
    h = np.asarray(x, np.float32)
    layers = _layers(dims, params)
    for l, (W, b) in enumerate(layers):
        sx = np.float32(act_scales[l])
        qx = e4m3_round(h * (np.float32(1.0) / sx))
        qw, sw = fp8_weights(W)
        acc = qx @ qw.T                      # exact: E4M3 products and sums fit in float64
        y = acc * (sx * sw).astype(np.float64) + b.astype(np.float64)
        if l + 1 < len(layers):
            h = np.maximum(y, 0.0).astype(np.float32)
        else:
            return np.tanh(y) if out_act else y


def fp8_forward_exact_tail(dims, params, act_scales, x, out_act: int, n_quant: int) -> np.ndarray:
    """fp8_forward with the first layer's inputs from column n_quant on taken
    exactly: layer 1 is dequant(codes of x[:, :n_quant] * (1 / sx) . the
    E4M3 weight codes of those columns) + W1[:, n_quant:] x[:, n_quant:]
    (float64) + b1, the weight scales sw[n] those of the whole row (as
    fp8_weights); the later layers as fp8_forward.  The model of an FP8 actor
    whose action-independent inputs (a stock state's indicator block) enter
    through a precomputed float table.  float64 [n][out]."""
    x = np.asarray(x, np.float32)
    layers = _layers(dims, params)
    W, b = layers[0]
    sx = np.float32(act_scales[0])
    qw, sw = fp8_weights(W)
    qx = e4m3_round(x[:, :n_quant] * (np.float32(1.0) / sx))
    acc = qx @ qw[:, :n_quant].T
    y = acc * (sx * sw).astype(np.float64) + x[:, n_quant:].astype(np.float64) @ W[:, n_quant:].astype(np.float64).T \
        + b.astype(np.float64)
    if len(layers) == 1:
        return np.tanh(y) if out_act else y
    h = np.maximum(y, 0.0).astype(np.float32)
    for l, (W, b) in enumerate(layers[1:], start=1):
        sx = np.float32(act_scales[l])
        qx = e4m3_round(h * (np.float32(1.0) / sx))
        qw, sw = fp8_weights(W)
        y = (qx @ qw.T) * (sx * sw).astype(np.float64) + b.astype(np.float64)
        if l + 1 < len(layers):
            h = np.maximum(y, 0.0).astype(np.float32)
        else:
            return np.tanh(y) if out_act else y


def fp8_calibrate(dims, params, obs) -> np.ndarray:
    """One agent's activation scales [L] float32: max |x_l| / 448 over the
    batch (1 where it is 0), x_l the input of layer l through the fp64
    forward of the fp32 master weights."""
    h = np.asarray(obs, np.float64)
    out = []
    layers = _layers(dims, params)
    for l, (W, b) in enumerate(layers):
        amax = np.float32(np.abs(h).max())
        out.append(amax / np.float32(E4M3_MAX) if amax > 0 else np.float32(1.0))
        if l + 1 < len(layers):
            h = np.maximum(h @ W.astype(np.float64).T + b.astype(np.float64), 0.0)
    return np.array(out, np.float32)


def ensemble_mean(a: np.ndarray, w=None) -> np.ndarray:
    """a[M][K] fp64 -> anchored weighted mean [K]."""
    a = _c(a, np.float64)
    M, K = a.shape
    w = _c(w, np.float64)
    out = np.empty(K, np.float64)
    _load().orc_ensemble_mean(M, K, _p(a), _p(w), _p(out))
    return out


def argmax(q) -> int:
    q = _c(q, np.float64)
    return int(_load().orc_argmax(_p(q), q.size))


def vote(ballots) -> int:
    b = _c(ballots, np.uint8)
    return int(_load().orc_vote(b.size, _p(b)))


def metrics_series(v, ann: float) -> np.ndarray:
    v = _c(v, np.int64)
    out = np.empty(3, np.float64)
    _load().orc_metrics_series(v.size, _p(v), float(ann), _p(out))
    return out


TRAJ_METRICS = ("cumulative_return", "sharpe", "max_drawdown", "annual_return", "annual_volatility", "romad",
                "sortino", "calmar", "omega", "discounted_return", "periods")


def trajectory_metrics(rew, done, v0: int, ann: float, gamma: float) -> np.ndarray:
    """rew[T][N] int64, done[T][N] uint8 or None -> [N][11] (TRAJ_METRICS)."""
    rew = _c(rew, np.int64)
    T, N = rew.shape
    d = None if done is None else _c(done, np.uint8)
    out = np.empty((N, 11), np.float64)
    _load().orc_trajectory_metrics(T, N, _p(rew), _p(d), C.c_int64(int(v0)), C.c_double(float(ann)),
                                   C.c_double(float(gamma)), _p(out))
    return out


def philox4x32_10(ctr, key) -> tuple:
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    _load().orc_philox4x32_10(c, k, o)
    return tuple(o)


def uniform24(x: int) -> float:
    f = _load().orc_uniform24
    f.restype = C.c_double
    return f(C.c_uint32(int(x)))


def explore_normal(seed: int, e: int, g: int, k: int) -> float:
    f = _load().orc_explore_normal
    f.restype = C.c_double
    return f(C.c_uint64(int(seed)), C.c_uint32(int(e)), C.c_uint32(int(g)), C.c_uint32(int(k)))


def explore_greedy(seed: int, e: int, g: int, eps: float, action: int) -> int:
    f = _load().orc_explore_greedy
    f.restype = C.c_int32
    return int(f(C.c_uint64(int(seed)), C.c_uint32(int(e)), C.c_uint32(int(g)), C.c_double(float(eps)),
                 C.c_int32(int(action))))


def splitmix64(x: int) -> int:
    f = _load().orc_splitmix64
    f.restype = C.c_uint64
    return int(f(C.c_uint64(int(x) & (2**64 - 1))))


class ReplayRef:
    """The replay buffer of Sec. 3.2 restated plainly: a list of transitions
    in push order, of which the last `capacity` are the contents.

    A trajectory's rows are taken in (t, env) order; a row is a real step
    unless its env was done before it (done[t-1][e]; not live at t = 0),
    with auto-reset every row is; s' is obs[t+1][e], or the observation after
    the rollout at the last row.  A sample draw b takes position
    floor(x * size / 2^32) of the contents (0 = oldest), x the first word of
    Philox4x32-10 with counter (b, counter low, counter high, 3) and key
    (seed low, seed high)."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        self.items = []

    def push(self, obs, act, rew_f32, done, last_obs, live0=None, auto_reset=False):
        T, N = done.shape
        for t in range(T):
            for e in range(N):
                if auto_reset:
                    real = True
                elif t == 0:
                    real = live0 is None or bool(live0[e])
                else:
                    real = done[t - 1, e] == 0
                if not real:
                    continue
                nxt = obs[t + 1, e] if t + 1 < T else last_obs[e]
                self.items.append((obs[t, e], act[t, e], rew_f32[t, e], nxt, done[t, e]))

    def contents(self):
        return self.items[max(0, len(self.items) - self.capacity):]

    def sample_positions(self, B: int, seed: int, counter: int):
        size = len(self.contents())
        key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
        out = []
        for b in range(B):
            x = philox4x32_10([b, counter & 0xFFFFFFFF, (counter >> 32) & 0xFFFFFFFF, 3], key)[0]
            out.append((x * size) >> 32 if size else -1)
        return out


def market_table(market) -> np.ndarray:
    """A stock market's indicator table: its own ``ind`` when set, else the
    8 indicators from its close / high / low."""
    ind = getattr(market, "ind", None)
    return indicators(market.close, market.high, market.low) if ind is None else ind


def perturb_bps(seed: int, e: int, k: int, R: int) -> int:
    f = _load().orc_perturb_bps
    f.restype = C.c_int32
    return int(f(C.c_uint64(int(seed) & (2**64 - 1)), C.c_uint32(int(e)), C.c_uint32(int(k)), C.c_int32(int(R))))


def indicators(close, high, low) -> np.ndarray:
    """int64 [T][K] close/high/low -> float32 [T][8][K] (Sec. 6.1 indicators)."""
    c, h, lo = _c(close, np.int64), _c(high, np.int64), _c(low, np.int64)
    T, K = c.shape
    out = np.empty((T, 8, K), np.float32)
    _load().orc_indicators(T, K, _p(c), _p(h), _p(lo), _p(out))
    return out


# ------------------------------------------------------------------ rollouts

def sharpe_softmax_weights(sharpe, threshold: float) -> np.ndarray:
    """Sec. 5.2.1 weights calculation: agents whose validation Sharpe ratio is
    below `threshold` are discarded (when none reaches it, the best agent,
    lowest index on ties, is kept alone); the kept agents get
    softmax(Sharpe) -- exp(S_j - max S) / sum_k exp(S_k - max S), the max
    taken over the kept agents, the sum in agent order -- the others 0."""
    S = [float(x) for x in sharpe]
    keep = [j for j, x in enumerate(S) if x >= threshold]
    if not keep:
        best = 0
        for j in range(1, len(S)):
            if S[j] > S[best]:
                best = j
        keep = [best]
    m = max(S[j] for j in keep)
    w = [0.0] * len(S)
    total = 0.0
    for j in keep:
        w[j] = math.exp(S[j] - m)
        total += w[j]
    for j in keep:
        w[j] = w[j] / total
    return np.array(w, dtype=np.float64)


def validation_sharpe(market, Ke, start, W, bps, dims, params, *, init_cash: int, hmax: int,
                      fee_bps: int, T: int, nthreads: int = 0) -> np.ndarray:
    """Each agent trading the validation envs alone (fp64 actor): the mean over
    the envs of the episode Sharpe ratio after T steps."""
    out = []
    for j in range(params.shape[0]):
        r = stock_run(market, Ke, start, W, bps, init_cash=init_cash, hmax=hmax, fee_bps=fee_bps, T=T,
                      ensemble=(dims, params[j:j + 1], None), nthreads=nthreads, want=("metrics",))
        out.append(float(np.mean(r["metrics"][:, 1])))
    return np.array(out)


def stock_run(market, Ke, start, W, bps, *, init_cash: int, hmax: int,
              fee_bps: int, T: int, auto_reset: bool = False,
              act_i32=None, act_f32=None, ensemble=None, nthreads: int = 0,
              want=("obs", "q", "rew", "rew_f32", "done", "cash", "hold",
                    "metrics", "act"), buy_order: int = 0) -> dict:
    """Run T steps of N stock envs from reset.

    market: object with ``close`` int64[n_days][K] and either an indicator
    table ``ind`` f32[n_days][I][K] or ``high`` / ``low`` (the table is then
    the oracle's own ``indicators``).
    Exactly one action source: act_i32[T][N][K] (mode 0), act_f32[T][N][K]
    (mode 1) or ensemble = (dims, params[M][P] f32, weights or None) (mode 2).
    buy_order: 0 buys in ascending asset order, 1 largest requested count
    first (ties in ascending asset order).
    """
    close = _c(market.close, np.int64)
    ind = _c(market_table(market), np.float32)
    n_days, K = close.shape
    I = ind.shape[1]
    D = 1 + 2 * K + I * K
    Ke = _c(Ke, np.int32)
    N = Ke.size
    start = _c(start, np.int32)
    W = _c(W, np.int32)
    bps = _c(bps, np.int16)
    mode, M, L = 0, 0, 0
    dims = params = wts = None
    ai = af = None
    if act_i32 is not None:
        ai = _c(act_i32, np.int32)
    elif act_f32 is not None:
        mode, af = 1, _c(act_f32, np.float32)
    else:
        mode = 2
        dims_, params_, w_ = ensemble
        dims = _c(dims_, np.int32)
        params = _c(params_, np.float32)
        M, L = params.shape[0], dims.size - 1
        wts = _c(w_, np.float64)
    o = {}

    def mk(name, shape, dt):
        if name in want:
            o[name] = np.zeros(shape, dt)
        return o.get(name)

    obs = mk("obs", (T, N, D), np.float32)
    act = mk("act", (T, N, K), np.float64) if mode == 2 else None
    q = mk("q", (T, N, K), np.int32)
    rew = mk("rew", (T, N), np.int64)
    rf = mk("rew_f32", (T, N), np.float32)
    dn = mk("done", (T, N), np.uint8)
    cash = mk("cash", (T, N), np.int64)
    hold = mk("hold", (T, N, K), np.int32)
    met = mk("metrics", (N, 3), np.float64)
    rc = _load().orc_stock_run(
        n_days, K, I, _p(close), _p(ind), N, _p(Ke), _p(start), _p(W), _p(bps),
        int(init_cash), int(hmax), int(fee_bps), int(bool(auto_reset)), int(T),
        mode, _p(ai), _p(af), M, L, _p(dims), _p(params), _p(wts),
        _p(obs), _p(act), _p(q), _p(rew), _p(rf), _p(dn), _p(cash), _p(hold),
        _p(met), nthreads or max_threads(), int(buy_order))
    if rc != 0:
        raise ValueError(f"oracle stock_run rejected its inputs (code {rc})")
    return o


def crypto_run(market, start, W, *, init_cash: int, pmax: int, T: int,
               auto_reset: bool = False, act_u8=None, ensemble=None,
               nthreads: int = 0,
               want=("obs", "act", "agent_act", "rew", "rew_f32", "done",
                     "cash", "pos", "metrics")) -> dict:
    """Run T steps of N crypto envs from reset (mode 0: act_u8[T][N];
    mode 2: ensemble = (dims, params[M][P]))."""
    mid = _c(market.mid, np.int64)
    spread = _c(market.spread, np.uint8)
    fac = _c(market.fac, np.float32)
    S = mid.size
    start = _c(start, np.int32)
    W = _c(W, np.int32)
    N = start.size
    mode, M, L = 0, 0, 0
    dims = params = au = None
    if act_u8 is not None:
        au = _c(act_u8, np.uint8)
    else:
        mode = 2
        dims_, params_ = ensemble[:2]
        dims = _c(dims_, np.int32)
        params = _c(params_, np.float32)
        M, L = params.shape[0], dims.size - 1
    o = {}

    def mk(name, shape, dt):
        if name in want:
            o[name] = np.zeros(shape, dt)
        return o.get(name)

    obs = mk("obs", (T, N, 10), np.float32)
    act = mk("act", (T, N), np.uint8)
    agent = mk("agent_act", (T, N, max(M, 1)), np.uint8) if mode == 2 else None
    rew = mk("rew", (T, N), np.int64)
    rf = mk("rew_f32", (T, N), np.float32)
    dn = mk("done", (T, N), np.uint8)
    cash = mk("cash", (T, N), np.int64)
    pos = mk("pos", (T, N), np.int32)
    met = mk("metrics", (N, 3), np.float64)
    rc = _load().orc_crypto_run(
        S, _p(mid), _p(spread), _p(fac), N, _p(start), _p(W), int(init_cash),
        int(pmax), int(bool(auto_reset)), int(T), mode, _p(au), M, L, _p(dims),
        _p(params), _p(obs), _p(act), _p(agent), _p(rew), _p(rf), _p(dn),
        _p(cash), _p(pos), _p(met), nthreads or max_threads())
    if rc != 0:
        raise ValueError(f"oracle crypto_run rejected its inputs (code {rc})")
    return o
