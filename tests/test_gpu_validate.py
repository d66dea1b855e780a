"""Sec. 5.2.1 Sharpe-softmax ensemble weighting from a validation window."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS = (301, 64, 64, 30)


def _setup(ctx, N=96, W=6, seed=61):
    mk_np = synth.stock_market(200, 30, seed=seed)
    e = synth.stock_envs_cohorts(N, 30, 200, W, cohort=32, seed=seed)
    mk = fr.fr_market_create(ctx, mk_np)
    return mk_np, mk, e


def _env(ctx, mk, e):
    return fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps)


@pytest.mark.parametrize("threshold", [0.0, -1e9, 1e9])
def test_validation_weights(ctx, dev, threshold):
    mk_np, mk, e = _setup(ctx)
    params = synth.actor_params(DIMS, 4, seed=62)
    ens = fr.ensemble_create(ctx, DIMS, params, precision=fr.PREC_FP32)
    env = _env(ctx, mk, e)
    T = 5                                            # a 6-day window: 5 trading periods
    snap0 = fr.env_snapshot(env)
    S, w = fr.ensemble_validate(ens, env, T, threshold)
    assert fr.env_snapshot(env) == snap0             # the validation envs are left as they were
    # each agent's Sharpe: the mean (in env order) of a standalone single-agent rollout
    for j in range(4):
        one = fr.ensemble_create(ctx, DIMS, params[j:j + 1], precision=fr.PREC_FP32)
        envj = _env(ctx, mk, e)
        met = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
        fr.rollout(envj, one, T, metrics=met)
        torch.cuda.synchronize()
        acc = 0.0
        for x in met[:, 1].cpu().numpy():
            acc += float(x)
        assert S[j] == acc / e.N
    assert np.array_equal(w, oracle.sharpe_softmax_weights(S, threshold).astype(np.float32))
    if threshold == 1e9:
        assert (w == 1.0).sum() == 1 and (w == 0.0).sum() == 3
    # the ensemble now combines with those weights
    rng = np.random.default_rng(3)
    obs = torch.from_numpy(rng.uniform(-1, 1, (64, 301)).astype(np.float32)).to(dev)
    y = torch.empty(4, 64, 30, device=dev)
    act = torch.empty(64, 30, device=dev)
    fr.ensemble_forward(ens, obs, y)
    fr.ensemble_act(ens, obs, act)
    torch.cuda.synchronize()
    yn = y.cpu().numpy().astype(np.float64)
    want = np.stack([oracle.ensemble_mean(yn[:, i], w.astype(np.float64)) for i in range(64)])
    assert np.abs(act.cpu().numpy() - want).max() < 1e-5
    # and close to the oracle's own validation (fp64 actors)
    S_or = oracle.validation_sharpe(mk_np, e.Ke, e.start, e.W, e.bps, DIMS, params, init_cash=e.init_cash,
                                    hmax=100, fee_bps=10, T=T)
    assert np.abs(S - S_or).max() < 0.05, (S, S_or)


def test_validation_rejects_vote_ensembles_and_bad_weights(ctx):
    mk_np, mk, e = _setup(ctx, N=8)
    env = _env(ctx, mk, e)
    vote = fr.ensemble_create(ctx, (301, 64, 3), synth.actor_params((301, 64, 3), 3), combine=fr.COMBINE_VOTE,
                              out_act=0)
    with pytest.raises(fr.FrError):
        fr.ensemble_validate(vote, env, 5)
    ens = fr.ensemble_create(ctx, DIMS, synth.actor_params(DIMS, 3, seed=1), precision=fr.PREC_FP32)
    with pytest.raises(fr.FrError):
        fr.ensemble_set_weights(ens, [0.5, np.nan, 0.5])
