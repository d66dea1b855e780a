"""Seeded synthetic inputs shaped like the paper's workloads.

The paper trains and samples on daily OHLCV of the 30 Dow Jones stocks with
MACD, Bollinger, RSI, CCI, DX and SMA indicators (Sec. 6.1, stock data) and on
second-level Bitcoin limit-order-book data reduced to 8 factors (Sec. 6.1,
cryptocurrency data).  Neither dataset exists here, so this module generates
stand-ins of the same shape: geometric-Brownian-motion daily OHLCV in
integer cents (the technical indicators are computed from them, by the
library on the device and by the oracle on the CPU, not here) and
backward-looking momentum factors in place of the 8 learned crypto factors.
It also draws actor weights, environment start days, per-asset basis-point
perturbations and prescribed action sequences.

This module holds none of the method's arithmetic (no indicator, trading,
valuation, observation or ensemble rule).  Both the CUDA library's tests and
the oracle's tests draw their inputs from it.

Random numbers: a counter-based SplitMix64 stream (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), so every draw
is a pure function of (seed, stream, index) and identical on every machine;
normals by the Box-Muller transform.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 250110709
SUB_MARKET, SUB_WEIGHTS, SUB_ENVS, SUB_ACTIONS, SUB_ARRIVALS = 1, 2, 3, 4, 5

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based SplitMix64 stream keyed by (seed, stream id)."""

    def __init__(self, seed: int, stream: int):
        with np.errstate(over="ignore"):
            k = np.array([(seed * 0x100000001B3 + stream) & 0xFFFFFFFFFFFFFFFF],
                         dtype=np.uint64)
            self.key = _mix(k + _GAMMA)[0]
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        i = np.arange(self.pos + 1, self.pos + 1 + n, dtype=np.uint64)
        self.pos += n
        with np.errstate(over="ignore"):
            return _mix(self.key + i * _GAMMA)

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        u1 = 1.0 - self.uniform(n)          # (0, 1]
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Integers uniform in [lo, hi] (inclusive)."""
        span = hi - lo + 1
        return lo + np.floor(self.uniform(n) * span).astype(np.int64)


# ------------------------------------------------------------------ markets

STOCK_INDICATORS = ("macd", "boll_ub", "boll_lb", "rsi_30", "cci_30", "dx_30",
                    "sma_30", "sma_60")
STOCK_WARMUP_DAYS = 60
CRYPTO_LAGS = (1, 5, 15, 30, 60, 300, 900, 3600)
CRYPTO_WARMUP_S = 3600


@dataclass
class StockMarket:
    close: np.ndarray      # int64 [n_days][K] cents
    open: np.ndarray       # int64 [n_days][K]
    high: np.ndarray       # int64 [n_days][K]
    low: np.ndarray        # int64 [n_days][K]
    volume: np.ndarray     # int64 [n_days][K]
    # the indicator table f_t is not generated here: the library computes it
    # on the device from close / high / low (market_indicators), the oracle
    # on the CPU; a caller may set an explicit float32 [n_days][I][K] table
    ind: np.ndarray | None = None

    @property
    def n_days(self):
        return self.close.shape[0]

    @property
    def K(self):
        return self.close.shape[1]

    @property
    def I(self):
        return 8 if self.ind is None else self.ind.shape[1]


@dataclass
class CryptoMarket:
    mid: np.ndarray        # int64 [S] cents per lot
    spread: np.ndarray     # uint8 [S] cents, 1..5
    fac: np.ndarray        # float32 [S][8]

    @property
    def S(self):
        return self.mid.size


def _round_cents(x: np.ndarray) -> np.ndarray:
    return np.maximum(1, np.rint(x)).astype(np.int64)      # half-even


def stock_market(n_days: int, K: int = 30, seed: int = MASTER_SEED,
                 drift: float = 0.0003, vol: float = 0.02) -> StockMarket:
    """GBM daily closes, ln(c_{t+1}/c_t) = (drift - vol^2/2) + vol Z, starting
    uniform in [$20, $400], in int64 cents (half-even, floor 1 cent)."""
    st = Stream(seed, SUB_MARKET)
    c0 = 2000.0 + st.uniform(K) * 38000.0
    z = st.normal(n_days * K).reshape(n_days, K)
    z[0] = 0.0
    logp = np.log(c0)[None, :] + np.cumsum((drift - vol * vol / 2.0) + vol * z, axis=0)
    close_f = np.exp(logp)
    close = _round_cents(close_f)
    zo = st.normal(n_days * K).reshape(n_days, K)
    zh = np.abs(st.normal(n_days * K).reshape(n_days, K))
    zl = np.abs(st.normal(n_days * K).reshape(n_days, K))
    zv = st.normal(n_days * K).reshape(n_days, K)
    prev = np.vstack([close_f[:1], close_f[:-1]])
    open_f = prev * np.exp(0.005 * zo)
    high = _round_cents(np.maximum(open_f, close_f) * (1.0 + 0.005 * zh))
    low = _round_cents(np.minimum(open_f, close_f) * (1.0 - 0.005 * zl))
    high = np.maximum(high, close)
    low = np.minimum(low, close)
    volume = np.rint(1e6 * np.exp(0.3 * zv)).astype(np.int64)
    return StockMarket(close=close, open=_round_cents(open_f), high=high, low=low, volume=volume)


def crypto_market(S: int, seed: int = MASTER_SEED, vol: float = 1e-4,
                  mid0_cents: int = 6_000_000) -> CryptoMarket:
    """Second-level GBM mid price (per lot, int64 cents), spread uniform in
    1..5 cents, 8 momentum factors ln(mid_s / mid_{s-L}) / (vol sqrt L)
    clipped to +-5 for L in CRYPTO_LAGS (backward-looking only)."""
    st = Stream(seed, SUB_MARKET + 100)
    z = st.normal(S)
    z[0] = 0.0
    logm = np.log(float(mid0_cents)) + np.cumsum(-vol * vol / 2.0 + vol * z)
    mid = _round_cents(np.exp(logm))
    spread = st.integers(1, 5, S).astype(np.uint8)
    lm = np.log(mid.astype(np.float64))
    fac = np.empty((S, 8), np.float64)
    for i, L in enumerate(CRYPTO_LAGS):
        lag = np.concatenate([np.full(min(L, S), lm[0]), lm[:max(S - L, 0)]])
        fac[:, i] = np.clip((lm - lag) / (vol * np.sqrt(L)), -5.0, 5.0)
    return CryptoMarket(mid=mid, spread=spread, fac=fac.astype(np.float32))


# ------------------------------------------------------------------- actors

def actor_params(dims, M: int, seed: int = MASTER_SEED, out_scale: float = 1.0,
                 stream: int = SUB_WEIGHTS) -> np.ndarray:
    """M actors with fp32 master weights uniform in +-1/sqrt(fan_in) (biases
    too), packed per layer as W_l[out][in] then b_l[out]: float32 [M][P].
    out_scale multiplies the output layer (used for Q-nets so that Q gaps are
    not all near zero)."""
    st = Stream(seed, stream)
    L = len(dims) - 1
    blocks = []
    for _ in range(M):
        parts = []
        for l in range(L):
            fi, fo = dims[l], dims[l + 1]
            s = 1.0 / np.sqrt(fi)
            W = (st.uniform(fo * fi) * 2.0 - 1.0) * s
            b = (st.uniform(fo) * 2.0 - 1.0) * s
            if l == L - 1:
                W, b = W * out_scale, b * out_scale
            parts += [W, b]
        blocks.append(np.concatenate(parts))
    return np.stack(blocks).astype(np.float32)


def unpack_params(dims, flat: np.ndarray):
    """Inverse of the packing: list of (W[out][in], b[out]) per layer."""
    out, o = [], 0
    for l in range(len(dims) - 1):
        fi, fo = dims[l], dims[l + 1]
        W = flat[o:o + fo * fi].reshape(fo, fi)
        o += fo * fi
        b = flat[o:o + fo]
        o += fo
        out.append((W, b))
    return out


# --------------------------------------------------------------- env batches

@dataclass
class StockEnvs:
    Ke: np.ndarray         # int32 [N] assets traded (first Ke of the market)
    start: np.ndarray      # int32 [N] first day of the window
    W: np.ndarray          # int32 [N] window length in days (W - 1 steps)
    bps: np.ndarray | None  # int16 [N][K] per-asset perturbation, or None
    init_cash: int = 100_000_000
    hmax: int = 100
    fee_bps: int = 10

    @property
    def N(self):
        return self.Ke.size


@dataclass
class CryptoEnvs:
    start: np.ndarray      # int32 [N] first second of the window
    W: np.ndarray          # int32 [N] window length in seconds
    init_cash: int = 100_000_000
    pmax: int = 10

    @property
    def N(self):
        return self.start.size


def stock_envs_cohorts(N: int, K: int, n_days: int, W: int, cohort: int = 128,
                       seed: int = MASTER_SEED, bps: bool = True) -> StockEnvs:
    """Cohorts of `cohort` envs share a start day uniform in
    [warm-up, n_days - W]; every env trades all K assets."""
    st = Stream(seed, SUB_ENVS)
    n_coh = (N + cohort - 1) // cohort
    cs = st.integers(STOCK_WARMUP_DAYS, n_days - W, n_coh)
    start = np.repeat(cs, cohort)[:N].astype(np.int32)
    b = st.integers(-100, 100, N * K).reshape(N, K).astype(np.int16) if bps else None
    return StockEnvs(Ke=np.full(N, K, np.int32), start=start,
                     W=np.full(N, W, np.int32), bps=b)


def stock_envs_uneven(N: int, K: int, n_days: int, k_lo: int = 10, w_lo: int = 5,
                      w_hi: int = 250, seed: int = MASTER_SEED) -> StockEnvs:
    """Asset counts uniform in k_lo..K, windows uniform in w_lo..w_hi days,
    starts uniform in [warm-up, n_days - W]."""
    st = Stream(seed, SUB_ENVS + 10)
    Ke = st.integers(k_lo, K, N).astype(np.int32)
    W = st.integers(w_lo, w_hi, N).astype(np.int32)
    u = st.uniform(N)
    start = (STOCK_WARMUP_DAYS + np.floor(u * (n_days - W - STOCK_WARMUP_DAYS + 1))).astype(np.int32)
    b = st.integers(-100, 100, N * K).reshape(N, K).astype(np.int16)
    return StockEnvs(Ke=Ke, start=start, W=W, bps=b)


def crypto_envs(N: int, S: int, W: int, seed: int = MASTER_SEED) -> CryptoEnvs:
    st = Stream(seed, SUB_ENVS + 20)
    start = st.integers(CRYPTO_WARMUP_S, S - W, N).astype(np.int32)
    return CryptoEnvs(start=start, W=np.full(N, W, np.int32))


def prescribed_shares(T: int, N: int, K: int, hmax: int = 100,
                      seed: int = MASTER_SEED, p_zero: float = 0.3) -> np.ndarray:
    """int32 [T][N][K] share orders in [-hmax, hmax], a fraction zero."""
    st = Stream(seed, SUB_ACTIONS)
    q = st.integers(-hmax, hmax, T * N * K)
    z = st.uniform(T * N * K) < p_zero
    q[z] = 0
    return q.reshape(T, N, K).astype(np.int32)


def prescribed_unit(T: int, N: int, K: int, seed: int = MASTER_SEED) -> np.ndarray:
    """float32 [T][N][K] unit actions, mostly in [-1, 1] with some beyond."""
    st = Stream(seed, SUB_ACTIONS + 1)
    return (st.uniform(T * N * K) * 2.4 - 1.2).reshape(T, N, K).astype(np.float32)


def prescribed_discrete(T: int, N: int, seed: int = MASTER_SEED) -> np.ndarray:
    st = Stream(seed, SUB_ACTIONS + 2)
    return st.integers(0, 2, T * N).reshape(T, N).astype(np.uint8)


def poisson_arrivals(rate: float, duration: float, seed: int = MASTER_SEED) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of the given rate."""
    st = Stream(seed, SUB_ARRIVALS)
    n = int(rate * duration * 2 + 100)
    gaps = -np.log(1.0 - st.uniform(n)) / rate
    t = np.cumsum(gaps)
    return t[t < duration]


def serving_trace_stock(rate: float, duration: float, n_days: int = 1000, max_envs: int = 512,
                        max_window: int = 500, seed: int = MASTER_SEED) -> list:
    """Stock backtest requests arriving as a Poisson process: per request
    N ~ U{1..max_envs} envs, window W ~ U{5..max_window} days, a start day
    uniform over the days with 60 warm-up days before, +-1% per-env price
    perturbations (bps range 100) from a per-request seed."""
    times = poisson_arrivals(rate, duration, seed)
    st = Stream(seed, SUB_ARRIVALS + 1)
    n = len(times)
    nenv = st.integers(1, max_envs, n)
    win = st.integers(5, max_window, n)
    u = st.uniform(n)
    seeds = st.u64(n)
    out = []
    for i in range(n):
        lo, hi = 60, n_days - int(win[i])
        out.append({"t": float(times[i]), "n_envs": int(nenv[i]), "window": int(win[i]),
                    "start": int(lo + int(u[i] * (hi - lo + 1))), "bps_range": 100, "seed": int(seeds[i])})
    return out


def serving_trace_mixed(rate: float, duration: float, crypto_frac: float = 0.5, traj_frac: float = 0.1,
                        n_days: int = 1000, n_seconds: int = 480_000, seed: int = MASTER_SEED) -> list:
    """Backtest requests of both tasks arriving as one Poisson process:
    each request is crypto with probability crypto_frac, else stock, and
    records its trajectory with probability traj_frac.  Stock as
    serving_trace_stock (N ~ U{1..512}, W ~ U{5..500} days, 30 assets,
    +-1% perturbations); crypto N ~ U{1..2048} envs, W ~ U{3,600..86,400}
    seconds, env i starting start + i * stride seconds (stride ~ U{0..60}),
    the first start uniform over the seconds that leave the window inside
    the market after 3,600 warm-up seconds."""
    times = poisson_arrivals(rate, duration, seed)
    st = Stream(seed, SUB_ARRIVALS + 2)
    n = len(times)
    kind = st.uniform(n)
    rec = st.uniform(n)
    s_env = st.integers(1, 512, n)
    s_win = st.integers(5, 500, n)
    c_env = st.integers(1, 2048, n)
    c_win = st.integers(3600, 86_400, n)
    c_stride = st.integers(0, 60, n)
    u = st.uniform(n)
    seeds = st.u64(n)
    out = []
    for i in range(n):
        r = {"t": float(times[i]), "want_traj": bool(rec[i] < traj_frac)}
        if kind[i] < crypto_frac:
            nv, w, sd = int(c_env[i]), int(c_win[i]), int(c_stride[i])
            lo, hi = 3600, n_seconds - (nv - 1) * sd - w
            r.update(task=1, n_envs=nv, window=w, start_stride=sd, start=int(lo + int(u[i] * (hi - lo + 1))))
        else:
            w = int(s_win[i])
            lo, hi = 60, n_days - w
            r.update(task=0, n_envs=int(s_env[i]), window=w, start_stride=0,
                     start=int(lo + int(u[i] * (hi - lo + 1))), bps_range=100, seed=int(seeds[i]))
        out.append(r)
    return out


# ----------------------------------------------------------------- workloads

STOCK_DIMS_SMALL = (301, 64, 64, 30)
STOCK_DIMS = (301, 256, 256, 30)
CRYPTO_DIMS = (10, 128, 128, 3)


@dataclass
class StockWorkload:
    name: str
    market: StockMarket
    envs: StockEnvs
    T: int
    dims: tuple
    params: np.ndarray      # float32 [M][P]
    weights: np.ndarray | None = None
    extra: dict = field(default_factory=dict)


@dataclass
class CryptoWorkload:
    name: str
    market: CryptoMarket
    envs: CryptoEnvs
    T: int
    dims: tuple
    params: np.ndarray
    extra: dict = field(default_factory=dict)


def workload_stock_small(seed: int = MASTER_SEED) -> StockWorkload:
    """8 envs x 30 assets, a 35-day window (34 steps) after a 60-day warm-up,
    bps perturbation on, 3 fp32 actors 301-64-64-30."""
    mk = stock_market(95, 30, seed)
    st = Stream(seed, SUB_ENVS)
    envs = StockEnvs(Ke=np.full(8, 30, np.int32), start=np.full(8, 60, np.int32),
                     W=np.full(8, 35, np.int32),
                     bps=st.integers(-100, 100, 8 * 30).reshape(8, 30).astype(np.int16))
    return StockWorkload("stock 8 envs x 30 assets x 34 steps, 3 x 301-64-64-30",
                         mk, envs, 34, STOCK_DIMS_SMALL,
                         actor_params(STOCK_DIMS_SMALL, 3, seed))


def workload_stock_2048(seed: int = MASTER_SEED, N: int = 2048, T: int = 256,
                        n_days: int = 1000) -> StockWorkload:
    """2,048 envs x 30 assets over 1,000 GBM days, 16 cohorts of 128 sharing a
    start day, 256-step rollouts, 3 actors 301-256-256-30."""
    mk = stock_market(n_days, 30, seed)
    envs = stock_envs_cohorts(N, 30, n_days, T + 1, 128, seed)
    return StockWorkload(f"stock {N} envs x 30 assets x {T} steps, 3 x 301-256-256-30",
                         mk, envs, T, STOCK_DIMS, actor_params(STOCK_DIMS, 3, seed))


def workload_crypto(seed: int = MASTER_SEED, N: int = 8192, T: int = 1024,
                    S: int = 480_000) -> CryptoWorkload:
    mk = crypto_market(S, seed)
    envs = crypto_envs(N, S, T + 1, seed)
    return CryptoWorkload(f"crypto {N} envs x {T} steps, 5 x 10-128-128-3 vote",
                          mk, envs, T, CRYPTO_DIMS,
                          actor_params(CRYPTO_DIMS, 5, seed, out_scale=4.0))


def workload_uneven(seed: int = MASTER_SEED, N: int = 4096,
                    n_days: int = 1000) -> StockWorkload:
    mk = stock_market(n_days, 30, seed)
    envs = stock_envs_uneven(N, 30, n_days, seed=seed)
    T = int(envs.W.max()) - 1
    return StockWorkload(f"uneven stock {N} envs, K 10-30, W 5-250",
                         mk, envs, T, STOCK_DIMS, actor_params(STOCK_DIMS, 3, seed))
