"""Exploring rollouts: Gaussian action noise (stock) and epsilon-greedy
votes (crypto) from Philox4x32-10 draws, checked against the oracle's own
Philox."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import synth

pytestmark = pytest.mark.gpu


def _traj(T, N, D, K, dev, stock=True):
    return {"obs": torch.full((T, N, D), np.nan, device=dev),
            "act": (torch.full((T, N, K), np.nan, device=dev) if stock
                    else torch.full((T, N), 255, dtype=torch.uint8, device=dev)),
            "rew": torch.zeros(T, N, dtype=torch.int64, device=dev),
            "done": torch.zeros(T, N, dtype=torch.uint8, device=dev)}


def _stock(ctx, N=256, T=20, seed=71):
    w = synth.workload_stock_2048(N=N, T=T, seed=seed)
    mk = fr.fr_market_create(ctx, w.market)
    return w, mk


def _env(ctx, mk, e):
    return fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps)


@pytest.mark.parametrize("precision, tol", [(fr.PREC_FP32, 1e-4), (fr.PREC_BF16, 2e-2)])
def test_gaussian_exploration(ctx, dev, precision, tol):
    w, mk = _stock(ctx)
    e = w.envs
    N, T, sigma, seed = e.N, w.T, 0.3, 0xC0FFEE
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=precision)
    env = _env(ctx, mk, e)
    fr.env_set_exploration(env, fr.EXPLORE_GAUSSIAN, sigma=sigma, seed=seed)
    tr = _traj(T, N, env.D, 30, dev)
    met = torch.empty(N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, traj=tr, metrics=met)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in tr.items()}
    # the env executes the recorded (explored) actions exactly
    ref = oracle.stock_run(w.market, e.Ke, e.start, e.W, e.bps, init_cash=e.init_cash, hmax=100, fee_bps=10,
                           T=T, act_f32=g["act"])
    for k in ("obs", "rew", "done"):
        assert np.array_equal(g[k], ref[k]), k
    assert np.array_equal(met.cpu().numpy(), ref["metrics"])
    # executed - sigma z recovers the clean ensemble action
    rows = [(t, i) for t in range(0, T, 3) for i in range(0, N, 7)]
    z = np.array([[oracle.explore_normal(seed, i, t, k) for k in range(30)] for t, i in rows])
    act = np.array([g["act"][t, i] for t, i in rows], dtype=np.float64)
    obs = np.array([g["obs"][t, i] for t, i in rows], dtype=np.float64)
    ys = np.stack([oracle.net_forward(w.dims, w.params[j], obs, 1) for j in range(3)])
    clean = np.stack([oracle.ensemble_mean(ys[:, r]) for r in range(len(rows))])
    resid = act - sigma * z
    err = np.linalg.norm(resid - clean, axis=-1) / np.maximum(np.linalg.norm(clean, axis=-1), 1e-3)
    assert err.max() <= tol + 1e-5, err.max()
    assert np.linalg.norm(act - clean) > 0.5 * sigma * np.sqrt(act.size)       # the noise is there


def test_exploration_is_reproducible_and_continues_across_pieces(ctx, dev):
    w, mk = _stock(ctx, N=200, T=16)
    e = w.envs
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    acts = []
    for seed, pieces in ((5, (16,)), (5, (7, 9)), (6, (16,))):
        env = _env(ctx, mk, e)
        fr.env_set_exploration(env, fr.EXPLORE_GAUSSIAN, sigma=0.2, seed=seed)
        tr = _traj(16, e.N, env.D, 30, dev)
        t0 = 0
        for p in pieces:
            fr.rollout(env, ens, p, traj={k: v[t0:t0 + p] for k, v in tr.items()})
            t0 += p
        torch.cuda.synchronize()
        acts.append(tr["act"].cpu().numpy())
    assert np.array_equal(acts[0], acts[1])          # same seed: the same draws, in one or two rollouts
    assert not np.array_equal(acts[0], acts[2])      # another seed: other draws


def test_epsilon_greedy_votes(ctx, dev):
    w = synth.workload_crypto(N=512, T=40, S=40_000)
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, init_cash=e.init_cash, pmax=e.pmax)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16X3, combine=fr.COMBINE_VOTE, out_act=0)
    eps, seed = 0.1, 777
    fr.env_set_exploration(env, fr.EXPLORE_EPS_GREEDY, eps=eps, seed=seed)
    T = w.T
    tr = _traj(T, e.N, 10, 1, dev, stock=False)
    fr.rollout(env, ens, T, traj=tr)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in tr.items()}
    ref = oracle.crypto_run(w.market, e.start, e.W, init_cash=e.init_cash, pmax=e.pmax, T=T, act_u8=g["act"])
    for k in ("obs", "rew", "done"):
        assert np.array_equal(g[k], ref[k]), k
    obs = g["obs"].reshape(-1, 10)
    q = np.stack([oracle.net_forward(w.dims, w.params[j], obs, 0) for j in range(5)])
    votes = np.array([oracle.vote(b) for b in q.argmax(-1).T]).reshape(T, e.N)
    replaced = 0
    agree = 0
    for t in range(T):
        for i in range(e.N):
            want = oracle.explore_greedy(seed, i, t, eps, 255)
            if want != 255:                      # the oracle's Philox says: replace, by this action
                replaced += 1
                assert g["act"][t, i] == want
            else:
                agree += int(g["act"][t, i] == votes[t, i])
    kept = T * e.N - replaced
    assert agree / kept >= 0.999
    assert abs(replaced / (T * e.N) - eps) < 4 * np.sqrt(eps * (1 - eps) / (T * e.N))
