"""Largest-first buy order (buy_order = 1: a step's buys fill largest requested
count first, equal counts in ascending asset order) against the oracle, bit
for bit: prescribed steps where cash runs short, every tiny action sequence
with ties, and a BF16 rollout teacher-forced (the fused kernels take only
ascending order, so the rollout runs the unfused path)."""
import itertools
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import synth

pytestmark = pytest.mark.gpu


def _steps(env, acts, kind, dev):
    T, N = acts.shape[:2]
    a = torch.from_numpy(acts).to(dev)
    keys = ("rew", "done", "obs", "cash", "hold")
    out = {k: [] for k in keys}
    for t in range(T):
        rew = torch.empty(N, dtype=torch.int64, device=dev)
        dn = torch.empty(N, dtype=torch.uint8, device=dev)
        obs = torch.empty(N, env.D, device=dev)
        cash = torch.empty(N, dtype=torch.int64, device=dev)
        hold = torch.empty(N, env.K, dtype=torch.int32, device=dev)
        fr.env_step(env, a[t], kind, rew=rew, done=dn, obs=obs)
        fr.env_get_state(env, cash=cash, hold=hold)
        for k, v in zip(keys, (rew, dn, obs, cash, hold)):
            out[k].append(v)
    met = torch.empty(N, 3, dtype=torch.float64, device=dev)
    fr.env_metrics(env, met)
    torch.cuda.synchronize()
    res = {k: torch.stack(v).cpu().numpy() for k, v in out.items()}
    res["metrics"] = met.cpu().numpy()
    return res


def _check(res, ref, T):
    for k in ("rew", "done", "cash", "hold"):
        assert np.array_equal(res[k], ref[k]), k
    assert np.array_equal(res["obs"][:T - 1], ref["obs"][1:T])
    assert np.array_equal(res["metrics"], ref["metrics"])


@pytest.mark.parametrize("kind", [fr.ACT_I32_SHARES, fr.ACT_F32_UNIT])
def test_largest_first_partial_fills_bit_exact(ctx, dev, kind):
    # low cash, large fees: most steps cannot fill every buy, so the order
    # decides which assets are bought
    mk_np = synth.stock_market(120, 30, seed=5)
    envs = synth.stock_envs_uneven(512, 30, 120, k_lo=2, w_lo=20, w_hi=60, seed=6)
    T = 40
    if kind == fr.ACT_I32_SHARES:
        acts = synth.prescribed_shares(T, envs.N, 30, seed=7, p_zero=0.1)
        acts = (np.abs(acts) * np.where(np.arange(T)[:, None, None] % 5 == 4, -1, 1)).astype(np.int32)
        src = dict(act_i32=acts)
    else:
        acts = synth.prescribed_unit(T, envs.N, 30, seed=7)
        acts = (np.abs(acts) * np.where(np.arange(T)[:, None, None] % 5 == 4, -1, 1)).astype(np.float32)
        src = dict(act_f32=acts)
    kw = dict(init_cash=2_500_000, hmax=100, fee_bps=250, T=T, **src)
    ref = oracle.stock_run(mk_np, envs.Ke, envs.start, envs.W, envs.bps, buy_order=1, **kw)
    asc = oracle.stock_run(mk_np, envs.Ke, envs.start, envs.W, envs.bps, buy_order=0, **kw)
    assert np.mean(ref["hold"] != asc["hold"]) > 0.05        # the order matters here
    mk = fr.fr_market_create(ctx, mk_np)
    env = fr.env_create(ctx, mk, start=envs.start, window=envs.W, n_assets=envs.Ke, bps=envs.bps,
                        init_cash=2_500_000, hmax=100, fee_bps=250, buy_order=fr.BUY_LARGEST_FIRST)
    _check(_steps(env, acts, kind, dev), ref, T)


def test_largest_first_every_tiny_sequence_with_ties(ctx, dev):
    close = np.array([[400, 390, 410], [405, 385, 420], [398, 400, 401]], np.int64)
    mk_np = SimpleNamespace(close=close, ind=np.zeros((3, 1, 3), np.float32))
    seqs = list(itertools.product(itertools.product(range(-1, 3), repeat=3), repeat=2))
    N, T = len(seqs), 2
    acts = np.array(seqs, np.int32).transpose(1, 0, 2).copy()
    bps = np.tile(np.array([0, 55, -100], np.int16), (N, 1))
    ref = oracle.stock_run(mk_np, np.full(N, 3), np.zeros(N), np.full(N, 3), bps, init_cash=1700,
                           hmax=2, fee_bps=30, T=T, act_i32=acts, buy_order=1)
    mk = fr.fr_market_create(ctx, mk_np)
    env = fr.env_create(ctx, mk, start=np.zeros(N), window=3, bps=bps, init_cash=1700, hmax=2,
                        fee_bps=30, buy_order=fr.BUY_LARGEST_FIRST)
    _check(_steps(env, acts, fr.ACT_I32_SHARES, dev), ref, T)


def test_largest_first_rollout_teacher_forced(ctx, dev):
    w = synth.workload_stock_2048(T=32)
    e = w.envs
    cash0 = 5_000_000                              # $50,000: the actors' buys rarely all fit
    mk = fr.fr_market_create(ctx, w.market)
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps, init_cash=cash0,
                        buy_order=fr.BUY_LARGEST_FIRST)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    T, N = 32, e.N
    tr = {"obs": torch.empty(T, N, env.D, device=dev), "act": torch.empty(T, N, 30, device=dev),
          "rew": torch.empty(T, N, dtype=torch.int64, device=dev),
          "rew_f32": torch.empty(T, N, device=dev), "done": torch.empty(T, N, dtype=torch.uint8, device=dev)}
    met = torch.empty(N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, traj=tr, metrics=met)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in tr.items()}
    kw = dict(init_cash=cash0, hmax=100, fee_bps=10, T=T, act_f32=g["act"])
    ref = oracle.stock_run(w.market, e.Ke, e.start, e.W, e.bps, buy_order=1, **kw)
    for k in ("obs", "rew", "rew_f32", "done"):
        assert np.array_equal(g[k], ref[k]), k
    assert np.array_equal(met.cpu().numpy(), ref["metrics"])
    asc = oracle.stock_run(w.market, e.Ke, e.start, e.W, e.bps, buy_order=0, **kw)
    assert not np.array_equal(asc["rew"], ref["rew"])        # an ascending-order path would fail above


def test_buy_order_validation(ctx):
    w = synth.workload_stock_small()
    mk = fr.fr_market_create(ctx, w.market)
    with pytest.raises(fr.FrError):
        fr.env_create(ctx, mk, start=[60], window=[10], buy_order=2)
    cm = fr.fr_market_create(ctx, synth.crypto_market(8_000, seed=1))
    with pytest.raises(fr.FrError):
        fr.env_create(ctx, cm, start=[3600], window=[10], buy_order=fr.BUY_LARGEST_FIRST)
