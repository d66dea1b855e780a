"""GPU env kernels against the CPU oracle, bit for bit: prescribed action
sequences (integer shares, unit floats, discrete crypto actions) must give
identical rewards, cash, holdings, done flags, observations and FP64 metrics."""
import itertools
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import synth

pytestmark = pytest.mark.gpu


def _stock_env(ctx, mk_handle, envs, auto_reset=False):
    return fr.env_create(ctx, mk_handle, start=envs.start, window=envs.W, n_assets=envs.Ke,
                         bps=envs.bps, init_cash=envs.init_cash, hmax=envs.hmax,
                         fee_bps=envs.fee_bps, auto_reset=auto_reset)


def _run_stock_steps(env, acts, kind, dev):
    """Step T times; return per-step rew, rew_f32, done, obs-after, cash, hold and metrics."""
    T, N = acts.shape[:2]
    out = {k: [] for k in ("rew", "rew_f32", "done", "obs", "cash", "hold")}
    a = torch.from_numpy(acts).to(dev)
    for t in range(T):
        rew = torch.empty(N, dtype=torch.int64, device=dev)
        rf = torch.empty(N, dtype=torch.float32, device=dev)
        dn = torch.empty(N, dtype=torch.uint8, device=dev)
        obs = torch.empty(N, env.D, dtype=torch.float32, device=dev)
        cash = torch.empty(N, dtype=torch.int64, device=dev)
        hold = torch.empty(N, env.K, dtype=torch.int32, device=dev)
        fr.env_step(env, a[t], kind, rew=rew, rew_f32=rf, done=dn, obs=obs)
        fr.env_get_state(env, cash=cash, hold=hold)
        for k, v in zip(("rew", "rew_f32", "done", "obs", "cash", "hold"), (rew, rf, dn, obs, cash, hold)):
            out[k].append(v)
    met = torch.empty(N, 3, dtype=torch.float64, device=dev)
    fr.env_metrics(env, met)
    torch.cuda.synchronize()
    res = {k: torch.stack(v).cpu().numpy() for k, v in out.items()}
    res["metrics"] = met.cpu().numpy()
    return res


def _check_stock(res, ref, T):
    for k in ("rew", "rew_f32", "done", "cash", "hold"):
        assert np.array_equal(res[k], ref[k]), k
    # observation after step t == observation the oracle's step t+1 acted on
    assert np.array_equal(res["obs"][:T - 1], ref["obs"][1:T])
    assert np.array_equal(res["metrics"], ref["metrics"])


@pytest.mark.parametrize("kind", [fr.ACT_I32_SHARES, fr.ACT_F32_UNIT])
def test_stock_small_prescribed_bit_exact(ctx, dev, kind):
    w = synth.workload_stock_small()
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    env = _stock_env(ctx, mk, e)
    obs0 = torch.empty(e.N, env.D, device=dev)
    fr.env_observe(env, obs0)
    if kind == fr.ACT_I32_SHARES:
        acts = synth.prescribed_shares(w.T, e.N, 30)
        ref = oracle.stock_run(w.market, e.Ke, e.start, e.W, e.bps, init_cash=e.init_cash, hmax=100,
                               fee_bps=10, T=w.T, act_i32=acts)
    else:
        acts = synth.prescribed_unit(w.T, e.N, 30)
        acts[2, 3, 4] = np.nan
        acts[5, 1, 0] = -np.inf
        ref = oracle.stock_run(w.market, e.Ke, e.start, e.W, e.bps, init_cash=e.init_cash, hmax=100,
                               fee_bps=10, T=w.T, act_f32=acts)
    res = _run_stock_steps(env, acts, kind, dev)
    assert np.array_equal(obs0.cpu().numpy(), ref["obs"][0])
    _check_stock(res, ref, w.T)
    if kind == fr.ACT_F32_UNIT:
        assert fr.env_error_count(env) == 2


@pytest.mark.parametrize("auto_reset", [False, True])
def test_stock_uneven_prescribed_bit_exact(ctx, dev, auto_reset):
    # uneven asset counts (1..30), windows (2..45 days) and starts; more steps
    # than the longest window so frozen (or restarted) envs are covered
    mk_np = synth.stock_market(200, 30, seed=17)
    envs = synth.stock_envs_uneven(300, 30, 200, k_lo=1, w_lo=2, w_hi=45, seed=17)
    T = 50
    acts = synth.prescribed_shares(T, envs.N, 30, seed=18, p_zero=0.2)
    ref = oracle.stock_run(mk_np, envs.Ke, envs.start, envs.W, envs.bps, init_cash=envs.init_cash,
                           hmax=100, fee_bps=10, T=T, act_i32=acts, auto_reset=auto_reset)
    mk = fr.fr_market_create(ctx, mk_np)
    env = _stock_env(ctx, mk, envs, auto_reset)
    res = _run_stock_steps(env, acts, fr.ACT_I32_SHARES, dev)
    _check_stock(res, ref, T)


def test_stock_partial_fills_and_fees(ctx, dev):
    # low cash and large fees: almost every buy is partial or rejected
    mk_np = synth.stock_market(120, 30, seed=5)
    envs = synth.stock_envs_uneven(256, 30, 120, k_lo=20, w_lo=30, w_hi=60, seed=6)
    envs.init_cash = 2_500_000
    envs.fee_bps = 250
    T = 40
    acts = synth.prescribed_shares(T, envs.N, 30, seed=7, p_zero=0.0)
    acts = np.abs(acts) * np.where(np.arange(T)[:, None, None] % 5 == 4, -1, 1)
    acts = acts.astype(np.int32)
    ref = oracle.stock_run(mk_np, envs.Ke, envs.start, envs.W, envs.bps, init_cash=envs.init_cash,
                           hmax=100, fee_bps=250, T=T, act_i32=acts)
    mk = fr.fr_market_create(ctx, mk_np)
    env = _stock_env(ctx, mk, envs)
    res = _run_stock_steps(env, acts, fr.ACT_I32_SHARES, dev)
    _check_stock(res, ref, T)


def test_stock_all_tiny_action_sequences(ctx, dev):
    close = np.array([[310, 655], [290, 700], [333, 640], [301, 689]], np.int64)
    mk_np = SimpleNamespace(close=close, ind=np.zeros((4, 1, 2), np.float32))
    seqs = list(itertools.product(itertools.product(range(-2, 3), repeat=2), repeat=3))
    N, T = len(seqs), 3
    acts = np.array(seqs, np.int32).transpose(1, 0, 2).copy()
    bps = np.tile(np.array([37, -64], np.int16), (N, 1))
    ref = oracle.stock_run(mk_np, np.full(N, 2), np.zeros(N), np.full(N, 4), bps, init_cash=1500,
                           hmax=2, fee_bps=250, T=T, act_i32=acts)
    mk = fr.fr_market_create(ctx, mk_np)
    env = fr.env_create(ctx, mk, start=np.zeros(N), window=4, bps=bps, init_cash=1500, hmax=2,
                        fee_bps=250)
    res = _run_stock_steps(env, acts, fr.ACT_I32_SHARES, dev)
    _check_stock(res, ref, T)


def test_stock_tiny_action_sequences_in_a_30_asset_market(ctx, dev):
    """The same 15,625 sequences with two live assets of a 30-asset market:
    the two-envs-per-warp step kernel (30 assets, 8 indicators, 32-bit
    accounting) against the oracle, neighbouring envs in one warp taking
    different fills."""
    close = np.full((4, 30), 1000, np.int64)
    close[:, :2] = [[310, 655], [290, 700], [333, 640], [301, 689]]
    mk_np = SimpleNamespace(close=close, ind=np.zeros((4, 8, 30), np.float32))
    seqs = list(itertools.product(itertools.product(range(-2, 3), repeat=2), repeat=3))
    N, T = len(seqs), 3
    acts = np.zeros((T, N, 30), np.int32)
    acts[:, :, :2] = np.array(seqs, np.int32).transpose(1, 0, 2)
    bps = np.zeros((N, 30), np.int16)
    bps[:, :2] = [37, -64]
    ref = oracle.stock_run(mk_np, np.full(N, 2), np.zeros(N), np.full(N, 4), bps, init_cash=1500,
                           hmax=2, fee_bps=250, T=T, act_i32=acts)
    mk = fr.fr_market_create(ctx, mk_np)
    env = fr.env_create(ctx, mk, start=np.zeros(N), window=4, n_assets=np.full(N, 2), bps=bps,
                        init_cash=1500, hmax=2, fee_bps=250)
    res = _run_stock_steps(env, acts, fr.ACT_I32_SHARES, dev)
    _check_stock(res, ref, T)


@pytest.mark.parametrize("auto_reset", [False, True])
def test_crypto_prescribed_bit_exact(ctx, dev, auto_reset):
    mk_np = synth.crypto_market(30_000, seed=9)
    st = synth.Stream(9, 77)
    N, T = 1000, 300
    W = st.integers(2, 250, N).astype(np.int32)
    start = (3600 + np.floor(st.uniform(N) * (30_000 - 3600 - W))).astype(np.int32)
    acts = synth.prescribed_discrete(T, N, seed=10)
    acts[7, 3] = 9                                  # invalid -> hold, counted
    ref = oracle.crypto_run(mk_np, start, W, init_cash=20_000_000, pmax=3, T=T, act_u8=acts,
                            auto_reset=auto_reset)
    mk = fr.fr_market_create(ctx, mk_np)
    env = fr.env_create(ctx, mk, start=start, window=W, init_cash=20_000_000, pmax=3,
                        auto_reset=auto_reset)
    a = torch.from_numpy(acts).to(dev)
    rew = torch.empty(T, N, dtype=torch.int64, device=dev)
    rf = torch.empty(T, N, dtype=torch.float32, device=dev)
    dn = torch.empty(T, N, dtype=torch.uint8, device=dev)
    obs = torch.empty(T, N, 10, dtype=torch.float32, device=dev)
    cash = torch.empty(T, N, dtype=torch.int64, device=dev)
    pos = torch.empty(T, N, dtype=torch.int32, device=dev)
    for t in range(T):
        fr.env_step(env, a[t], fr.ACT_U8_DISCRETE, rew=rew[t], rew_f32=rf[t], done=dn[t], obs=obs[t])
        fr.env_get_state(env, cash=cash[t], hold=pos[t])
    met = torch.empty(N, 3, dtype=torch.float64, device=dev)
    fr.env_metrics(env, met)
    torch.cuda.synchronize()
    assert np.array_equal(rew.cpu().numpy(), ref["rew"])
    assert np.array_equal(rf.cpu().numpy(), ref["rew_f32"])
    assert np.array_equal(dn.cpu().numpy(), ref["done"])
    assert np.array_equal(cash.cpu().numpy(), ref["cash"])
    assert np.array_equal(pos.cpu().numpy(), ref["pos"])
    assert np.array_equal(obs.cpu().numpy()[:T - 1], ref["obs"][1:])
    assert np.array_equal(met.cpu().numpy(), ref["metrics"])
    assert fr.env_error_count(env) == 1


def test_snapshot_restore_continues_bit_exact(ctx, dev):
    w = synth.workload_stock_small()
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    acts = synth.prescribed_shares(w.T, e.N, 30, seed=3)
    a = torch.from_numpy(acts).to(dev)
    env = _stock_env(ctx, mk, e)
    for t in range(10):
        fr.env_step(env, a[t], fr.ACT_I32_SHARES)
    blob = fr.env_snapshot(env)
    rest = []
    for t in range(10, w.T):
        r = torch.empty(e.N, dtype=torch.int64, device=dev)
        fr.env_step(env, a[t], fr.ACT_I32_SHARES, rew=r)
        rest.append(r)
    m1 = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    fr.env_metrics(env, m1)
    env2 = _stock_env(ctx, mk, e)
    fr.env_restore(env2, blob)
    rest2 = []
    for t in range(10, w.T):
        r = torch.empty(e.N, dtype=torch.int64, device=dev)
        fr.env_step(env2, a[t], fr.ACT_I32_SHARES, rew=r)
        rest2.append(r)
    m2 = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    fr.env_metrics(env2, m2)
    torch.cuda.synchronize()
    assert torch.equal(torch.stack(rest), torch.stack(rest2))
    assert torch.equal(m1, m2)
    with pytest.raises(fr.FrError):
        fr.env_restore(env2, blob[:-8])
    # the same snapshot from page-locked memory restores the same state
    env3 = _stock_env(ctx, mk, e)
    fr.env_restore(env3, torch.frombuffer(bytearray(blob), dtype=torch.uint8).pin_memory())
    assert fr.env_snapshot(env3) == blob
    with pytest.raises(ValueError):
        fr.env_restore(env3, torch.zeros(len(blob), dtype=torch.int32))


def test_invalid_configurations_are_rejected(ctx):
    w = synth.workload_stock_small()
    mk = fr.fr_market_create(ctx, w.market)
    with pytest.raises(fr.FrError):
        fr.env_create(ctx, mk, start=[60], window=[36])        # runs past the market end
    with pytest.raises(fr.FrError):
        fr.env_create(ctx, mk, start=[60], window=[1])
    with pytest.raises(fr.FrError):
        fr.env_create(ctx, mk, start=[60], window=[10], n_assets=[31])
    with pytest.raises(fr.FrError):
        fr.env_create(ctx, mk, start=[60], window=[10], bps=np.full((1, 30), 101))
    big = SimpleNamespace(close=np.ones((5, 33), np.int64), ind=np.zeros((5, 1, 33), np.float32))
    with pytest.raises(fr.FrError):
        fr.fr_market_create(ctx, big)


def test_hbm_budget_is_enforced():
    c = fr.fr_ctx_create(0, hbm_budget_bytes=1 << 20)
    w = synth.workload_stock_2048()
    with pytest.raises(fr.FrError) as ei:
        mk = fr.fr_market_create(c, w.market)                  # 1.3 MB of tables > 1 MiB
        fr.env_create(c, mk, start=w.envs.start, window=w.envs.W, bps=w.envs.bps)
    assert ei.value.code == fr._lib.FR_ENOMEM
    assert c.bytes_in_use <= 1 << 20


@pytest.mark.parametrize("scale, hmax", [(1, 100), (3000, 100), (1, 60000)])
def test_stock_step_32_and_64_bit_accounting(ctx, dev, scale, hmax):
    # The step kernel runs its prices, orders and sums in 32-bit arithmetic
    # when env_create proves they fit (the bench's market); prices scaled
    # x3,000 (up to millions of dollars a share) or 60,000-share orders fail
    # that proof and take the 64-bit forms.  Both are bit-exact against the
    # oracle, partial fills included (cash for few of the orders).
    w = synth.workload_stock_small()
    mkt = SimpleNamespace(close=np.ascontiguousarray(w.market.close * scale), ind=w.market.ind,
                          high=w.market.high * scale, low=w.market.low * scale)
    e = w.envs
    mk = fr.fr_market_create(ctx, mkt)
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps, init_cash=e.init_cash,
                        hmax=hmax, fee_bps=10)
    acts = synth.prescribed_unit(w.T, e.N, 30)
    ref = oracle.stock_run(mkt, e.Ke, e.start, e.W, e.bps, init_cash=e.init_cash, hmax=hmax,
                           fee_bps=10, T=w.T, act_f32=acts)
    res = _run_stock_steps(env, acts, fr.ACT_F32_UNIT, dev)
    _check_stock(res, ref, w.T)
