"""On-device data preparation: the 8 technical indicators from OHLC
(market_indicators, and markets created with device_indicators) and the
per-env price perturbations (env_perturb, and the server's draws), each
bit-exact against the oracle."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(mk, dev):
    return [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (mk.close, mk.high, mk.low)]


# sizes: one asset / one day; several 128-day tiles with a ragged tail; more
# than 32 assets (two recurrence blocks); ten years of daily data at 30 assets
@pytest.mark.parametrize("T, K, seed", [(1, 1, 1), (2, 3, 2), (300, 30, 3), (129, 33, 4), (700, 45, 5),
                                        (2520, 30, 6)])
def test_market_indicators_match_oracle(dev, built_lib, T, K, seed):
    mk = synth.stock_market(T, K, seed=seed)
    c, h, lo = _dev(mk, dev)
    got = fr.market_indicators(c, h, lo)
    torch.cuda.synchronize()
    want = oracle.indicators(mk.close, mk.high, mk.low)
    assert np.array_equal(got.cpu().numpy(), want)


def test_market_indicators_degenerate_series(dev, built_lib):
    # constant prices, a flat-then-jump series and a one-sided ramp: the
    # zero-denominator branches (MAD, DI sum, losses) on the device
    T = 200
    flat = np.full((T, 1), 5000, np.int64)
    jump = flat.copy()
    jump[100:] = 7000
    ramp = (10_000 + 37 * np.arange(T, dtype=np.int64))[:, None]
    close = np.hstack([flat, jump, ramp, ramp[::-1].copy()])
    got = fr.market_indicators(*[torch.from_numpy(close).to(dev)] * 3)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), oracle.indicators(close, close, close))


def test_market_created_with_device_indicators(ctx, dev):
    mk = synth.stock_market(500, 30, seed=9)
    want = oracle.indicators(mk.close, mk.high, mk.low)
    assert np.array_equal(fr.fr_market_indicators(fr.fr_market_create(ctx, mk)), want)
    # an explicit host table is uploaded as given
    host = SimpleNamespace(close=mk.close, ind=want[:, ::-1].copy())
    assert np.array_equal(fr.fr_market_indicators(fr.fr_market_create(ctx, host)), want[:, ::-1])
    bad = SimpleNamespace(close=mk.close, high=mk.low, low=mk.high, ind=None)     # low > close somewhere
    with pytest.raises(fr.FrError):
        fr.fr_market_create(ctx, bad)


def test_market_indicators_rejects_bad_arguments(dev, built_lib):
    c = torch.ones(4, 2, dtype=torch.int64, device=dev)
    out = torch.empty(4, 8, 2, device=dev)
    p = c.data_ptr()
    assert fr.lib().market_indicators(p, p, None, 4, 2, out.data_ptr(), None) == fr._lib.FR_EINVAL
    assert fr.lib().market_indicators(p, p, p, 0, 2, out.data_ptr(), None) == fr._lib.FR_EINVAL
    assert fr.lib().market_indicators(p, p, p, 4, 0, out.data_ptr(), None) == fr._lib.FR_EINVAL


def _bps_table(N, K, seed, R):
    b = np.zeros((N, K), np.int16)
    for e in range(N):
        for k in range(K):
            b[e, k] = oracle.perturb_bps(seed, e, k, R)
    return b


@pytest.mark.parametrize("R", [100, 37, 0])
def test_env_perturb_matches_oracle_draws(ctx, dev, R):
    w = synth.workload_stock_2048(N=300, T=24, seed=31)
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_FP32)
    seed = 0xFEEDFACE12345678
    a = fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke)
    fr.env_perturb(a, seed, R)
    fr.env_reset(a)
    b = fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=_bps_table(e.N, 30, seed, R))
    ma = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    mb = torch.empty_like(ma)
    fr.rollout(a, ens, w.T, metrics=ma)
    fr.rollout(b, ens, w.T, metrics=mb)
    torch.cuda.synchronize()
    assert np.array_equal(ma.cpu().numpy(), mb.cpu().numpy())


def test_env_perturb_trajectory_against_oracle(ctx, dev):
    # prescribed trades on a perturbed batch: rewards, cash and metrics
    # bit-exact with the oracle's run on the oracle's draws
    w = synth.workload_stock_small()
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke)
    fr.env_perturb(env, 99, 100)
    fr.env_reset(env)
    T = w.T
    acts = synth.prescribed_shares(T, e.N, 30, seed=3)
    a = torch.from_numpy(acts).to(dev)
    rew, cash = [], []
    for t in range(T):
        r = torch.empty(e.N, dtype=torch.int64, device=dev)
        c = torch.empty(e.N, dtype=torch.int64, device=dev)
        fr.env_step(env, a[t], fr.ACT_I32_SHARES, rew=r)
        fr.env_get_state(env, cash=c)
        rew.append(r)
        cash.append(c)
    met = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    fr.env_metrics(env, met)
    torch.cuda.synchronize()
    ref = oracle.stock_run(w.market, e.Ke, e.start, e.W, _bps_table(e.N, 30, 99, 100), init_cash=e.init_cash,
                           hmax=100, fee_bps=10, T=T, act_i32=acts)
    assert np.array_equal(torch.stack(rew).cpu().numpy(), ref["rew"])
    assert np.array_equal(torch.stack(cash).cpu().numpy(), ref["cash"])
    assert np.array_equal(met.cpu().numpy(), ref["metrics"])


def test_env_perturb_errors(ctx, dev):
    w = synth.workload_crypto(N=8, T=8, S=5000)
    mk = fr.fr_market_create(ctx, w.market)
    env = fr.env_create(ctx, mk, start=w.envs.start, window=w.envs.W)
    with pytest.raises(fr.FrError):
        fr.env_perturb(env, 1, 100)                                # stock envs only
    s = synth.workload_stock_small()
    env = fr.env_create(ctx, fr.fr_market_create(ctx, s.market), start=s.envs.start, window=s.envs.W)
    with pytest.raises(fr.FrError):
        fr.env_perturb(env, 1, 101)
