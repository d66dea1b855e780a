"""The crypto ensemble of Sec. 5.2.2 with DQN, Double DQN and Dueling DQN
agents: per-agent heads in the vote, Q-values after the heads, and the
DQN / Double DQN learning targets, against the oracle's fp64 definitions.

Tolerances: Q-values per row within twice the actor tolerance (1e-4 FP32,
2e-3 BF16X3, 2e-2 BF16) of the batch's RMS output norm (the head is a
linear map of norm <= 2), argmax agreement >= 99.9% (BF16: 98%); targets
within the tolerance of
the largest |y|; votes agree on >= 99.9% of rows; env trajectories
teacher-forced bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS = (10, 128, 128, 4)            # 3 actions + the dueling head's V
HEADS = [fr.HEAD_Q, fr.HEAD_Q, fr.HEAD_DUELING, fr.HEAD_DUELING, fr.HEAD_Q]   # DQN, DDQN, Dueling, ...
TOL = {fr.PREC_FP32: 1e-4, fr.PREC_BF16X3: 2e-3, fr.PREC_BF16: 2e-2}


def _obs(n, seed=5):
    w = synth.workload_crypto(N=512, T=64, S=60_000)
    acts = synth.prescribed_discrete(64, 512, seed=seed)
    o = oracle.crypto_run(w.market, w.envs.start, w.envs.W, init_cash=w.envs.init_cash, pmax=10, T=64,
                          act_u8=acts, want=("obs",))
    obs = o["obs"].reshape(-1, 10)
    return np.ascontiguousarray(obs[np.linspace(0, obs.shape[0] - 1, n).astype(int)])


def _params(seed):
    return synth.actor_params(DIMS, len(HEADS), seed=seed, out_scale=4.0)


def _rel(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-3)


@pytest.mark.parametrize("precision", [fr.PREC_FP32, fr.PREC_BF16X3, fr.PREC_BF16])
def test_q_values_after_heads(ctx, dev, precision):
    params = _params(3)
    obs = _obs(2000)
    ens = fr.ensemble_create(ctx, DIMS, params, precision=precision, combine=fr.COMBINE_VOTE, out_act=0, heads=HEADS)
    assert ens.n_act == 3
    q = fr.ensemble_q(ens, torch.from_numpy(obs).to(dev))
    torch.cuda.synchronize()
    got = q.cpu().numpy()
    for j, h in enumerate(HEADS):
        y = oracle.net_forward(DIMS, params[j], obs, 0)
        want = oracle.head_q(y, h, 3)
        # the head is a fixed linear map of the outputs (norm <= 2), so the
        # error scales with the outputs, not with Q (a dueling Q can be far
        # smaller than the V and A it comes from); BF16 rows whose outputs
        # nearly cancel are measured against the batch's output scale
        scale = np.sqrt(np.mean(np.sum(y * y, axis=-1)))
        err = np.linalg.norm(got[j] - want, axis=-1) / scale
        assert err.max() <= 2 * TOL[precision], (j, err.max())
        assert np.mean(got[j].argmax(-1) == want.argmax(-1)) >= (0.999 if precision != fr.PREC_BF16 else 0.98)


@pytest.mark.parametrize("precision", [fr.PREC_FP32, fr.PREC_BF16X3])
def test_mixed_head_ensemble_rollout(ctx, dev, precision):
    # the unfused path (dueling ensembles do not take the fused kernel):
    # env bit-exact on the emitted votes, votes as the oracle's heads give them
    w = synth.workload_crypto(N=1024, T=48, S=40_000)
    e = w.envs
    params = _params(4)
    mk = fr.fr_market_create(ctx, w.market)
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, init_cash=e.init_cash, pmax=e.pmax)
    ens = fr.ensemble_create(ctx, DIMS, params, precision=precision, combine=fr.COMBINE_VOTE, out_act=0, heads=HEADS)
    T = 48
    tr = {"obs": torch.full((T, e.N, 10), np.nan, device=dev),
          "act": torch.full((T, e.N), 255, dtype=torch.uint8, device=dev),
          "rew": torch.zeros(T, e.N, dtype=torch.int64, device=dev),
          "done": torch.zeros(T, e.N, dtype=torch.uint8, device=dev)}
    met = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, traj=tr, metrics=met)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in tr.items()}
    ref = oracle.crypto_run(w.market, e.start, e.W, init_cash=e.init_cash, pmax=e.pmax, T=T, act_u8=g["act"])
    for k in ("obs", "rew", "done"):
        assert np.array_equal(g[k], ref[k]), k
    assert np.array_equal(met.cpu().numpy(), ref["metrics"])
    obs = g["obs"].reshape(-1, 10)
    qs = [oracle.head_q(oracle.net_forward(DIMS, params[j], obs, 0), h, 3) for j, h in enumerate(HEADS)]
    votes = np.array([oracle.vote(b) for b in np.stack([q.argmax(-1) for q in qs]).T])
    agree = np.mean(votes == g["act"].ravel())
    print(f"prec {precision}: vote agreement with dueling heads {agree:.5f}")
    assert agree >= 0.999
    # a dueling agent's action is not the argmax of its first three outputs
    y2 = oracle.net_forward(DIMS, params[2], obs, 0)
    assert np.mean(y2[:, :3].argmax(-1) != qs[2].argmax(-1)) > 0.1


@pytest.mark.parametrize("double_q", [True, False])
@pytest.mark.parametrize("precision", [fr.PREC_FP32, fr.PREC_BF16X3])
def test_dqn_targets_from_replay_samples(ctx, dev, precision, double_q):
    p_on, p_tg = _params(6), _params(7)
    n = 3000
    obs = _obs(n, seed=8)
    rng = np.random.default_rng(9)
    rew = rng.normal(0, 0.01, n).astype(np.float32)
    done = (rng.random(n) < 0.1).astype(np.uint8)
    on = fr.ensemble_create(ctx, DIMS, p_on, precision=precision, combine=fr.COMBINE_VOTE, out_act=0, heads=HEADS)
    tg = fr.ensemble_create(ctx, DIMS, p_tg, precision=precision, combine=fr.COMBINE_VOTE, out_act=0, heads=HEADS)
    y = fr.ensemble_q_targets(on, tg, torch.from_numpy(obs).to(dev), torch.from_numpy(rew).to(dev),
                              torch.from_numpy(done).to(dev), gamma=0.97, double_q=double_q)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.float64)
    want = oracle.q_targets(DIMS, p_on, p_tg, HEADS, obs, rew, done, 0.97, double_q)
    scale = np.abs(want).max()
    err = np.abs(got - want).max() / scale
    print(f"prec {precision} double {double_q}: max err {err:.2e} of max |y| {scale:.3f}")
    assert err <= TOL[precision]
    assert np.array_equal(got[:, done == 1], np.broadcast_to(rew[done == 1], got[:, done == 1].shape))
    other = oracle.q_targets(DIMS, p_on, p_tg, HEADS, obs, rew, done, 0.97, not double_q)
    assert np.abs(other - want).max() > 10 * TOL[precision] * scale     # the two targets really differ


def test_heads_errors_and_validation(ctx, dev):
    p = _params(10)
    with pytest.raises(fr.FrError):                  # dueling needs a vote
        fr.ensemble_create(ctx, DIMS, p, combine=fr.COMBINE_MEAN, out_act=0, heads=HEADS)
    with pytest.raises(fr.FrError):                  # and an identity output
        fr.ensemble_create(ctx, DIMS, p, combine=fr.COMBINE_VOTE, out_act=1, heads=HEADS)
    with pytest.raises(fr.FrError):
        fr.ensemble_create(ctx, DIMS, p, combine=fr.COMBINE_VOTE, out_act=0, heads=[0, 0, 2, 0, 0])
    a = fr.ensemble_create(ctx, DIMS, p, combine=fr.COMBINE_VOTE, out_act=0, heads=HEADS)
    with pytest.raises(fr.FrError):                  # all plain heads: 4 outputs are 4 actions, too many
        fr.ensemble_create(ctx, DIMS, p, combine=fr.COMBINE_VOTE, out_act=0)
    d3 = (10, 128, 128, 3)
    b = fr.ensemble_create(ctx, d3, synth.actor_params(d3, 5, seed=11), combine=fr.COMBINE_VOTE, out_act=0)
    with pytest.raises(fr.FrError):                  # online and target of different shapes
        fr.ensemble_q_targets(a, b, torch.zeros(4, 10, device=dev), torch.zeros(4, device=dev))
    # one agent: the vote path and the Q path agree (vote = argmax of the head's Q)
    obs = torch.from_numpy(_obs(4000, seed=12)).to(dev)
    for j in (1, 2):
        one = fr.ensemble_create(ctx, DIMS if HEADS[j] else d3, p[j:j + 1] if HEADS[j] else
                                 synth.actor_params(d3, 1, seed=13), combine=fr.COMBINE_VOTE, out_act=0,
                                 heads=[HEADS[j]])
        votes = torch.empty(obs.shape[0], dtype=torch.uint8, device=dev)
        fr.ensemble_act(one, obs, votes)
        q = fr.ensemble_q(one, obs)
        torch.cuda.synchronize()
        assert np.array_equal(votes.cpu().numpy(), q[0].argmax(-1).cpu().numpy().astype(np.uint8))


def test_rollout_replay_targets_pipeline(ctx, dev):
    # producer -> reservoir -> consumer (Sec. 3.2) on the device: an
    # epsilon-greedy crypto rollout of a mixed DQN / Dueling ensemble fills
    # the replay buffer; a sampled batch gives Double DQN targets.  The
    # oracle replays the same trajectory into its replay model and evaluates
    # the targets of the same sampled transitions.
    w = synth.workload_crypto(N=512, T=40, S=30_000)
    e = w.envs
    params = _params(14)
    mk = fr.fr_market_create(ctx, w.market)
    env = fr.env_create(ctx, mk, start=e.start, window=np.full(e.N, 30, np.int32), init_cash=e.init_cash,
                        pmax=e.pmax)
    ens = fr.ensemble_create(ctx, DIMS, params, precision=fr.PREC_FP32, combine=fr.COMBINE_VOTE, out_act=0,
                             heads=HEADS)
    tgt = fr.ensemble_create(ctx, DIMS, _params(15), precision=fr.PREC_FP32, combine=fr.COMBINE_VOTE, out_act=0,
                             heads=HEADS)
    fr.env_set_exploration(env, fr.EXPLORE_EPS_GREEDY, eps=0.05, seed=77)
    T = 36
    tr = {"obs": torch.empty(T, e.N, 10, device=dev), "act": torch.empty(T, e.N, dtype=torch.uint8, device=dev),
          "rew_f32": torch.empty(T, e.N, device=dev), "done": torch.empty(T, e.N, dtype=torch.uint8, device=dev)}
    fr.rollout(env, ens, T, traj=tr)
    last = torch.empty(e.N, 10, device=dev)
    fr.env_observe(env, last)
    rb = fr.replay_create(ctx, env, 100_000)
    fr.replay_push(rb, env, tr, T, last)
    B = 2048
    smp = fr.replay_sample(rb, B, seed=3, counter=1)
    y = fr.ensemble_q_targets(ens, tgt, smp["next_obs"], smp["rew"], smp["done"], gamma=0.99, double_q=True)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in tr.items()}
    ref = oracle.ReplayRef(100_000)
    ref.push(g["obs"], g["act"], g["rew_f32"], g["done"], last.cpu().numpy())
    assert fr.replay_size(rb)[0] == len(ref.contents()) < T * e.N       # frozen rows after the 29 steps
    pos = ref.sample_positions(B, 3, 1)
    assert np.array_equal(smp["index"].cpu().numpy(), np.array(pos))
    items = ref.contents()
    nxt = np.stack([items[p][3] for p in pos])
    rew = np.array([items[p][2] for p in pos], np.float32)
    dn = np.array([items[p][4] for p in pos], np.uint8)
    assert dn.sum() > 0 and np.array_equal(smp["next_obs"].cpu().numpy(), nxt)
    want = oracle.q_targets(DIMS, params, _params(15), HEADS, nxt, rew, dn, 0.99, True)
    got = y.cpu().numpy().astype(np.float64)
    assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max()
