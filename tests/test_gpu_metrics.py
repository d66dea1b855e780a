"""Trajectory metrics on the device (Sec. 6.1 metric list, Sec. 4.3 discounted
return) against the oracle on the same stored rewards."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import synth

pytestmark = pytest.mark.gpu

EXACT = [0, 1, 2, 4, 5, 6, 8, 9, 10]       # every metric but the two through pow()


@pytest.mark.parametrize("N, T", [(256, 40), (1000, 61)])
def test_trajectory_metrics_match_oracle(ctx, dev, N, T):
    w = synth.workload_stock_2048(N=N, T=T)
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    env = fr.env_create(ctx, mk, start=e.start, window=np.minimum(e.W, 30 + np.arange(N) % 40),
                        n_assets=e.Ke, bps=e.bps)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    rew = torch.empty(T, N, dtype=torch.int64, device=dev)
    done = torch.empty(T, N, dtype=torch.uint8, device=dev)
    met = torch.empty(N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, traj={"rew": rew, "done": done}, metrics=met)
    got = fr.trajectory_metrics(rew, done, v0=e.init_cash, ann=252.0, gamma=0.99)
    torch.cuda.synchronize()
    g = got.cpu().numpy()
    want = oracle.trajectory_metrics(rew.cpu().numpy(), done.cpu().numpy(), e.init_cash, 252.0, 0.99)
    assert np.array_equal(g[:, EXACT], want[:, EXACT])
    assert np.allclose(g[:, [3, 7]], want[:, [3, 7]], rtol=1e-13, atol=0)
    assert np.array_equal(g[:, :3], met.cpu().numpy())          # = the env's own episode metrics


def test_trajectory_metrics_edges(ctx, dev):
    rew = torch.zeros(0, 5, dtype=torch.int64, device=dev)
    got = fr.trajectory_metrics(rew, None, v0=1000)              # no rows: nothing happened
    torch.cuda.synchronize()
    assert (got == 0).all()
    with pytest.raises(fr.FrError):
        fr.trajectory_metrics(torch.zeros(3, 2, dtype=torch.int64, device=dev), None, v0=0)
