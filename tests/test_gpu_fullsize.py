"""Parity at the benchmark's full sizes, in the launch configuration it times.

Stock: 2,048 envs x 30 assets x 256 steps, 3 BF16 actors 301-256-256-30, the
fused rollout with metrics only (no trajectory; tiles packed).  Crypto:
8,192 envs x 1,024 steps, 5 Q-nets 10-128-128-3, majority vote, in FP16 and
BF16X3 (both meet the 99.9% vote bar; FP16 is the benchmark's crypto
headline) and in BF16 (reported; at least 99%, the differences at near-tied
Q values).

* The timed launch (metrics only) and a launch that also records the
  trajectory give bit-identical metrics: the recorded actions are the ones
  the timed launch took.
* The oracle replays every env's recorded actions and reproduces every
  reward, done flag and the FP64 metrics bit for bit.
* The oracle's fp64 actors on sampled observations (taken from the oracle's
  own replay) agree with the GPU's actions within the stated tolerance
  (stock: relative L2 2e-2 and shares within one; crypto FP16 and BF16X3:
  vote agreement >= 99.9%)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import synth

pytestmark = pytest.mark.gpu


def test_stock_2048_envs_256_steps_bench_launch(ctx, dev):
    w = synth.workload_stock_2048()
    e = w.envs
    T, N = w.T, e.N
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps)
    met_timed = torch.empty(N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, metrics=met_timed)                    # the benchmark's launch
    fr.env_reset(env)
    tr = {"act": torch.empty(T, N, 30, device=dev), "rew": torch.empty(T, N, dtype=torch.int64, device=dev),
          "done": torch.empty(T, N, dtype=torch.uint8, device=dev)}
    met = torch.empty(N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, traj=tr, metrics=met)
    torch.cuda.synchronize()
    assert fr.ensemble_device_errors(ens) == 0
    assert torch.equal(met_timed, met)
    g = {k: v.cpu().numpy() for k, v in tr.items()}
    ref = oracle.stock_run(w.market, e.Ke, e.start, e.W, e.bps, init_cash=e.init_cash, hmax=100, fee_bps=10,
                           T=T, act_f32=g["act"], want=("rew", "done", "metrics"))
    assert np.array_equal(g["rew"], ref["rew"])
    assert np.array_equal(g["done"], ref["done"])
    assert np.array_equal(met.cpu().numpy(), ref["metrics"])
    # actors on sampled observations: 64 envs spread over the 16 cohorts
    rng = np.random.default_rng(7)
    envs = np.sort(rng.choice(N, 64, replace=False))
    sub = oracle.stock_run(w.market, e.Ke[envs], e.start[envs], e.W[envs], e.bps[envs], init_cash=e.init_cash,
                           hmax=100, fee_bps=10, T=T, act_f32=g["act"][:, envs].copy(), want=("obs", "rew"))
    assert np.array_equal(sub["rew"], g["rew"][:, envs])
    rows = rng.choice(T * envs.size, 512, replace=False)
    obs = sub["obs"].reshape(-1, sub["obs"].shape[-1])[rows]
    act = g["act"][:, envs].reshape(-1, 30)[rows].astype(np.float64)
    ys = np.stack([oracle.net_forward(w.dims, w.params[j], obs, 1) for j in range(3)])
    want = np.stack([oracle.ensemble_mean(ys[:, i]) for i in range(rows.size)])
    err = np.linalg.norm(act - want, axis=-1) / np.maximum(np.linalg.norm(want, axis=-1), 1e-3)
    assert err.max() <= 2e-2, err.max()
    qg = oracle.discretise_many(act.astype(np.float32), 100)
    qw = np.array([oracle.discretise(x, 100) for x in want.ravel()])
    print(f"stock full size: max rel err {err.max():.2e}, exact shares {np.mean(qg == qw):.4f}")
    assert np.mean(np.abs(qg - qw) <= 1) >= 0.999


@pytest.mark.parametrize("precision", [fr.PREC_FP16, fr.PREC_BF16X3, fr.PREC_BF16])
def test_crypto_8192_envs_1024_steps_bench_launch(ctx, dev, precision):
    w = synth.workload_crypto()
    e = w.envs
    T, N = w.T, e.N
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=precision, combine=fr.COMBINE_VOTE, out_act=0)
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, init_cash=e.init_cash, pmax=e.pmax)
    met_timed = torch.empty(N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, metrics=met_timed)
    fr.env_reset(env)
    tr = {"act": torch.empty(T, N, dtype=torch.uint8, device=dev),
          "rew": torch.empty(T, N, dtype=torch.int64, device=dev),
          "done": torch.empty(T, N, dtype=torch.uint8, device=dev)}
    met = torch.empty(N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, traj=tr, metrics=met)
    torch.cuda.synchronize()
    assert fr.ensemble_device_errors(ens) == 0
    assert torch.equal(met_timed, met)
    g = {k: v.cpu().numpy() for k, v in tr.items()}
    ref = oracle.crypto_run(w.market, e.start, e.W, init_cash=e.init_cash, pmax=e.pmax, T=T, act_u8=g["act"],
                            want=("rew", "done", "metrics"))
    assert np.array_equal(g["rew"], ref["rew"])
    assert np.array_equal(g["done"], ref["done"])
    assert np.array_equal(met.cpu().numpy(), ref["metrics"])
    rng = np.random.default_rng(8)
    envs = np.sort(rng.choice(N, 64, replace=False))
    sub = oracle.crypto_run(w.market, e.start[envs], e.W[envs], init_cash=e.init_cash, pmax=e.pmax, T=T,
                            act_u8=g["act"][:, envs].copy(), want=("obs", "rew"))
    assert np.array_equal(sub["rew"], g["rew"][:, envs])
    rows = rng.choice(T * envs.size, 16384, replace=False)
    obs = sub["obs"].reshape(-1, 10)[rows]
    q = np.stack([oracle.net_forward(w.dims, w.params[j], obs, 0) for j in range(5)])
    votes = np.array([oracle.vote(b) for b in q.argmax(-1).T])
    miss = votes != g["act"][:, envs].reshape(-1)[rows]
    agree = 1.0 - miss.mean()
    srt = np.sort(q, axis=-1)
    gap = (srt[..., -1] - srt[..., -2]).min(axis=0)           # the closest agent decision of each row
    print(f"crypto full size, precision {precision}: vote agreement {agree:.5f}; smallest agent Q-gap "
          f"median {np.median(gap):.3e} overall, {np.median(gap[miss]) if miss.any() else 0:.3e} "
          f"where the vote differs")
    if precision == fr.PREC_BF16:
        # BF16 inputs move Q by more than the gap of near-tied rows: the bar
        # is met by FP16 and BF16X3; here the differences must sit at near-ties
        assert agree >= 0.99
        assert not miss.any() or np.median(gap[miss]) < 0.1 * np.median(gap)
    else:
        assert agree >= 0.999
