"""The rollout autotuner: it times the launch configurations of an env /
ensemble pair on the env's own state and keeps the fastest.  The env must be
left as it was, the choice must be the fastest reported, a second env of
the same shape must take it from the cache, and rollouts under it must be
the same as a rollout on the default path where the configurations agree
(packing, ring depth and actor kernel never change results)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import synth

pytestmark = pytest.mark.gpu


def _metrics(env, ens, T, dev):
    m = torch.empty(env.N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, metrics=m)
    torch.cuda.synchronize()
    return m.cpu().numpy()


def test_autotune_uneven_stock(ctx, dev):
    w = synth.workload_uneven(N=1024)
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    make = lambda: fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps)
    env = make()
    rep = fr.env_autotune(env, ens, 32, force=True)
    c = rep["candidates"]
    paths = {x["path"] for x in c}
    assert {2, 0} <= paths and any(x["path"] == 2 and x["packed"] == 0 for x in c)   # packing on and off
    assert all(x["ms"] > 0 for x in c) and not rep["cached"]
    assert c[rep["chosen"]]["ms"] == min(x["ms"] for x in c)
    print("autotune:", [(x["path"], x["packed"], x["stages"], x["tiled"], round(x["ms"], 3)) for x in c])
    # the env was left as it was: the tuned env and a fresh env give the same
    # metrics under the same configuration (the second env takes it from the cache)
    env2 = make()
    rep2 = fr.env_autotune(env2, ens, 32)
    assert rep2["cached"] and rep2["candidates"][0]["path"] == c[rep["chosen"]]["path"]
    T = w.T
    m1, m2 = _metrics(env, ens, T, dev), _metrics(env2, ens, T, dev)
    assert np.array_equal(m1, m2)
    # on the resident fused kernel, packing never changes results
    env3 = make()
    fr.env_tune_clear(env3)
    if c[rep["chosen"]]["path"] == 2:
        assert np.array_equal(_metrics(env3, ens, T, dev), m1)


def test_autotune_crypto_every_ring_depth_agrees(ctx, dev):
    w = synth.workload_crypto(N=2048, T=64, S=40_000)
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16, combine=fr.COMBINE_VOTE, out_act=0)
    make = lambda: fr.env_create(ctx, mk, start=e.start, window=e.W, init_cash=e.init_cash, pmax=e.pmax)
    env = make()
    rep = fr.env_autotune(env, ens, 16, force=True)
    c = rep["candidates"]
    ring = [x for x in c if x["path"] == 1]
    assert len(ring) >= 2 and len({x["stages"] for x in ring}) == len(ring)
    print("autotune:", [(x["path"], x["stages"], x["tiled"], round(x["ms"], 3)) for x in c])
    # resident and streamed weight rings give the same rollout, bit for bit
    ms = []
    for x in ring:
        env_x = make()
        fr.env_tune_set(env_x, 1, stages=x["stages"])
        ms.append(_metrics(env_x, ens, w.T, dev))
    assert all(np.array_equal(m, ms[0]) for m in ms[1:])
    if c[rep["chosen"]]["path"] == 1:
        assert np.array_equal(_metrics(env, ens, w.T, dev), ms[0])


def test_packing_and_actor_kernel_choices_agree(ctx, dev):
    w = synth.workload_uneven(N=1024)
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    make = lambda: fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps)
    a, b = make(), make()
    fr.env_tune_set(a, 2, packed=True)
    fr.env_tune_set(b, 2, packed=False)
    assert np.array_equal(_metrics(a, ens, w.T, dev), _metrics(b, ens, w.T, dev))
    # unfused, large-batch actor kernel vs single-agent kernel (20,480 envs > one tile per SM)
    big = synth.stock_envs_uneven(20480, 30, w.market.close.shape[0], k_lo=10, w_lo=5, w_hi=40, seed=3)
    envs = [fr.env_create(ctx, mk, start=big.start, window=big.W, n_assets=big.Ke, bps=big.bps) for _ in range(2)]
    fr.env_tune_set(envs[0], 0, tiled=True)
    fr.env_tune_set(envs[1], 0, tiled=False)
    assert np.array_equal(_metrics(envs[0], ens, 12, dev), _metrics(envs[1], ens, 12, dev))


def test_autotune_errors_and_fp32(ctx, dev):
    s = synth.workload_stock_small()
    mk = fr.fr_market_create(ctx, s.market)
    make = lambda: fr.env_create(ctx, mk, start=s.envs.start, window=s.envs.W, n_assets=s.envs.Ke, bps=s.envs.bps)
    env = make()
    ens = fr.ensemble_create(ctx, s.dims, s.params, precision=fr.PREC_FP32)
    with pytest.raises(fr.FrError):
        fr.env_autotune(env, ens, 0)
    with pytest.raises(fr.FrError):
        fr.env_tune_set(env, 3)
    rep = fr.env_autotune(env, ens, 8, force=True)
    assert [x["path"] for x in rep["candidates"]] == [0]       # FP32: only the unfused path
    # the env was restored: its rollout equals a fresh env's
    assert np.array_equal(_metrics(env, ens, s.T, dev), _metrics(make(), ens, s.T, dev))
