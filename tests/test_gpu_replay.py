"""Device replay buffer against the oracle's plain replay model.

The transitions come from real rollouts (envs with uneven windows, so many
finish and freeze inside the trajectory); the oracle pushes the same
trajectory arrays and must predict the buffer size, every sampled position
(its own Philox4x32-10) and every sampled transition bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import synth

pytestmark = pytest.mark.gpu


def _stock_rollout(ctx, dev, mk, envs, ens, T, auto_reset=False):
    env = fr.env_create(ctx, mk, start=envs.start, window=envs.W, n_assets=envs.Ke, bps=envs.bps,
                        auto_reset=auto_reset)
    tr = {"obs": torch.empty(T, envs.N, env.D, device=dev), "act": torch.empty(T, envs.N, 30, device=dev),
          "rew_f32": torch.empty(T, envs.N, device=dev), "done": torch.empty(T, envs.N, dtype=torch.uint8, device=dev)}
    return env, tr


def _run(env, ens, tr, T, dev):
    fr.rollout(env, ens, T, traj=tr)
    last = torch.empty(env.N, env.D, device=dev)
    fr.env_observe(env, last)
    return last


def _np(tr, last):
    torch.cuda.synchronize()
    return ({k: v.cpu().numpy() for k, v in tr.items()}, last.cpu().numpy())


def _check_samples(rb, ref, B, seed, counter, stock=True):
    s = fr.replay_sample(rb, B, seed, counter)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in s.items()}
    pos = ref.sample_positions(B, seed, counter)
    assert np.array_equal(g["index"], np.array(pos))
    items = ref.contents()
    for b in range(B):
        o, a, r, n, d = items[pos[b]]
        assert np.array_equal(g["obs"][b], o) and np.array_equal(g["next_obs"][b], n), b
        assert (np.array_equal(g["act"][b], a) if stock else g["act"][b] == a), b
        assert g["rew"][b] == r and g["done"][b] == d, b


@pytest.mark.parametrize("precision", [fr.PREC_FP32, fr.PREC_BF16])
def test_replay_push_and_sample_stock(ctx, dev, precision):
    mk_np = synth.stock_market(300, 30, seed=61)
    envs = synth.stock_envs_uneven(700, 30, 300, k_lo=5, w_lo=2, w_hi=40, seed=62)
    mk = fr.fr_market_create(ctx, mk_np)
    w = synth.workload_stock_2048(N=8, T=8)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=precision)
    T = 30
    env, tr = _stock_rollout(ctx, dev, mk, envs, ens, T)
    rb = fr.replay_create(ctx, env, 50_000)
    assert fr.replay_size(rb) == (0, 0, 0)
    last = _run(env, ens, tr, T, dev)
    fr.replay_push(rb, env, tr, T, last)
    g, l = _np(tr, last)
    ref = oracle.ReplayRef(50_000)
    ref.push(g["obs"], g["act"], g["rew_f32"], g["done"], l)
    assert 0 < len(ref.items) < T * envs.N                            # frozen rows were skipped
    size, pushed, err = fr.replay_size(rb)
    assert size == pushed == len(ref.items) and err == 0
    _check_samples(rb, ref, 3000, seed=77, counter=0)
    _check_samples(rb, ref, 513, seed=77, counter=1)


def test_replay_fifo_wraps_across_pushes(ctx, dev):
    mk_np = synth.stock_market(300, 30, seed=63)
    envs = synth.stock_envs_uneven(300, 30, 300, k_lo=5, w_lo=10, w_hi=60, seed=64)
    mk = fr.fr_market_create(ctx, mk_np)
    w = synth.workload_stock_2048(N=8, T=8)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    C = 4099
    T = 12
    env, tr = _stock_rollout(ctx, dev, mk, envs, ens, T)
    rb = fr.replay_create(ctx, env, C)
    ref = oracle.ReplayRef(C)
    live = torch.ones(envs.N, dtype=torch.uint8, device=dev)
    for piece in range(4):                                          # one 48-step rollout in 4 pieces
        done_before = torch.empty(envs.N, dtype=torch.uint8, device=dev)
        fr.env_get_state(env, done=done_before)
        live0 = (1 - done_before).contiguous()
        last = _run(env, ens, tr, T, dev)
        fr.replay_push(rb, env, tr, T, last, live0=live0)
        g, l = _np(tr, last)
        ref.push(g["obs"], g["act"], g["rew_f32"], g["done"], l, live0=live0.cpu().numpy())
        size, pushed, _ = fr.replay_size(rb)
        assert pushed == len(ref.items) and size == min(pushed, C)
    assert len(ref.items) > C
    _check_samples(rb, ref, 2000, seed=5, counter=9)


def test_replay_auto_reset_and_crypto(ctx, dev):
    w = synth.workload_crypto(N=256, T=40, S=30_000)
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    W = np.where(np.arange(e.N) % 3 == 0, 7, 25).astype(np.int32)
    env = fr.env_create(ctx, mk, start=e.start, window=W, init_cash=e.init_cash, pmax=e.pmax, auto_reset=True)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16X3, combine=fr.COMBINE_VOTE, out_act=0)
    T = 30
    tr = {"obs": torch.empty(T, e.N, 10, device=dev), "act": torch.empty(T, e.N, dtype=torch.uint8, device=dev),
          "rew_f32": torch.empty(T, e.N, device=dev), "done": torch.empty(T, e.N, dtype=torch.uint8, device=dev)}
    rb = fr.replay_create(ctx, env, 100_000)
    last = _run(env, ens, tr, T, dev)
    fr.replay_push(rb, env, tr, T, last)
    g, l = _np(tr, last)
    assert g["done"].sum() > 0
    ref = oracle.ReplayRef(100_000)
    ref.push(g["obs"], g["act"], g["rew_f32"], g["done"], l, auto_reset=True)
    assert fr.replay_size(rb)[1] == len(ref.items) == T * e.N
    _check_samples(rb, ref, 1500, seed=2**40 + 3, counter=2**33 + 1, stock=False)


def test_replay_empty_errors_and_graph_capture(ctx, dev):
    s = synth.workload_stock_small()
    mk = fr.fr_market_create(ctx, s.market)
    env = fr.env_create(ctx, mk, start=s.envs.start, window=s.envs.W, n_assets=s.envs.Ke, bps=s.envs.bps)
    rb = fr.replay_create(ctx, env, 1000)
    out = fr.replay_sample(rb, 8, 1)
    torch.cuda.synchronize()
    assert (out["index"].cpu().numpy() == -1).all() and fr.replay_size(rb)[2] == 1
    with pytest.raises(fr.FrError):
        fr.replay_create(ctx, env, 0)
    crypto = synth.workload_crypto(N=8, T=8, S=5000)
    cenv = fr.env_create(ctx, fr.fr_market_create(ctx, crypto.market), start=crypto.envs.start, window=crypto.envs.W)
    T = 5
    tr = {"obs": torch.zeros(T, cenv.N, 10, device=dev), "act": torch.zeros(T, cenv.N, dtype=torch.uint8, device=dev),
          "rew_f32": torch.zeros(T, cenv.N, device=dev), "done": torch.zeros(T, cenv.N, dtype=torch.uint8, device=dev)}
    with pytest.raises(fr.FrError):                                 # env of another shape
        fr.replay_push(rb, cenv, tr, T, tr["obs"][0])
    # push + sample captured into a CUDA graph, replayed: the device counter advances
    ens = fr.ensemble_create(ctx, s.dims, s.params, precision=fr.PREC_FP32)
    T = 4
    st = {"obs": torch.empty(T, env.N, env.D, device=dev), "act": torch.empty(T, env.N, 30, device=dev),
          "rew_f32": torch.empty(T, env.N, device=dev), "done": torch.empty(T, env.N, dtype=torch.uint8, device=dev)}
    last = _run(env, ens, st, T, dev)
    rb2 = fr.replay_create(ctx, env, 10_000)
    smp = {"index": torch.empty(16, dtype=torch.int64, device=dev)}
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fr.replay_push(rb2, env, st, T, last)                      # warm-up outside the capture
        fr.replay_sample(rb2, 16, 3, 0, out=smp)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fr.replay_push(rb2, env, st, T, last)
        fr.replay_sample(rb2, 16, 3, 0, out=smp)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert fr.replay_size(rb2)[1] == 4 * T * env.N
