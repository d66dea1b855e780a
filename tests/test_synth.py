"""The seeded synthetic inputs (CPU): the shapes and statistics the input
recipe states, so that a mistake in a generator (a wrong drift, a wrong
volatility scale, a window that runs past the market) fails here rather than
silently changing every workload."""
import numpy as np

from paper_2501_10709_gb300 import synth


def test_stock_gbm_log_returns_have_the_stated_moments():
    drift, vol = 0.0003, 0.02
    mk = synth.stock_market(2000, 30, seed=101)
    c = mk.close.astype(np.float64)
    lr = np.log(c[1:] / c[:-1]).ravel()
    n = lr.size
    # the daily closes round to cents: at >= $20 that moves a log price by at
    # most 2.5e-4, well inside the bands below
    mean_want = drift - vol * vol / 2.0
    assert abs(lr.mean() - mean_want) < 4.0 * vol / np.sqrt(n) + 1e-5
    var_rel = lr.var(ddof=1) / (vol * vol)
    assert abs(var_rel - 1.0) < 4.0 * np.sqrt(2.0 / n) + 0.01


def test_stock_start_prices_and_ohlc_order():
    mk = synth.stock_market(300, 30, seed=102)
    assert mk.close.dtype == np.int64 and (mk.close >= 1).all()
    assert ((mk.close[0] >= 2000) & (mk.close[0] <= 40000)).all()     # $20 .. $400
    assert (mk.high >= mk.close).all() and (mk.low <= mk.close).all()
    assert (mk.high >= mk.open).all() and (mk.low <= mk.open).all()
    assert (mk.low >= 1).all() and (mk.volume > 0).all()


def test_crypto_mid_spread_and_factor_scale():
    vol = 1e-4
    mk = synth.crypto_market(200_000, seed=103, vol=vol)
    assert (mk.mid >= 1).all()
    assert mk.spread.min() >= 1 and mk.spread.max() <= 5
    assert set(np.unique(mk.spread).tolist()) == {1, 2, 3, 4, 5}
    assert np.abs(mk.fac).max() <= 5.0
    # the one-second factor is a normalised log return: mean 0, variance 1
    # (up to the cent rounding of a $60,000 mid, ~1.4e-5 of vol)
    f1 = mk.fac[synth.CRYPTO_WARMUP_S:, 0].astype(np.float64)
    assert abs(f1.mean()) < 4.0 / np.sqrt(f1.size) + 0.01
    assert abs(f1.var() - 1.0) < 0.05
    # longer lags see more of the same random walk: still unit variance
    f60 = mk.fac[synth.CRYPTO_WARMUP_S::60, 4].astype(np.float64)
    assert abs(f60.var() - 1.0) < 0.15


def test_actor_weights_are_uniform_in_the_fan_in_range():
    dims = synth.STOCK_DIMS
    p = synth.actor_params(dims, 3, seed=104)
    assert p.dtype == np.float32 and p.shape[0] == 3
    for j in range(3):
        for l, (W, b) in enumerate(synth.unpack_params(dims, p[j])):
            s = 1.0 / np.sqrt(dims[l])
            assert W.shape == (dims[l + 1], dims[l]) and b.shape == (dims[l + 1],)
            assert np.abs(W).max() <= s * (1 + 1e-6) and np.abs(b).max() <= s * (1 + 1e-6)
            # uniform on [-s, s]: variance s^2 / 3
            assert abs(W.astype(np.float64).var() / (s * s / 3.0) - 1.0) < 0.1


def test_env_windows_fit_the_market_after_the_warm_up():
    n_days = 1000
    e = synth.stock_envs_cohorts(2048, 30, n_days, 257, 128, seed=105)
    assert (e.start >= synth.STOCK_WARMUP_DAYS).all() and (e.start + e.W <= n_days).all()
    assert (e.start.reshape(16, 128) == e.start.reshape(16, 128)[:, :1]).all()   # cohorts share a day
    assert e.bps.min() >= -100 and e.bps.max() <= 100
    u = synth.stock_envs_uneven(4096, 30, n_days, seed=106)
    assert (u.Ke >= 10).all() and (u.Ke <= 30).all()
    assert (u.W >= 5).all() and (u.W <= 250).all()
    assert (u.start >= synth.STOCK_WARMUP_DAYS).all() and (u.start + u.W <= n_days).all()
    c = synth.crypto_envs(8192, 480_000, 1025, seed=107)
    assert (c.start >= synth.CRYPTO_WARMUP_S).all() and (c.start + c.W <= 480_000).all()


def test_generators_are_deterministic_per_seed():
    a, b, c = (synth.stock_market(50, 30, seed=s) for s in (7, 7, 8))
    assert np.array_equal(a.close, b.close) and np.array_equal(a.high, b.high)
    assert not np.array_equal(a.close, c.close)
    x, y = synth.actor_params((10, 16, 3), 2, seed=9), synth.actor_params((10, 16, 3), 2, seed=9)
    assert np.array_equal(x, y)
