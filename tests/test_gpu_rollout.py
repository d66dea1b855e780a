"""Rollouts (observe -> ensemble -> step for T steps) checked teacher-forced:
the oracle replays the GPU's emitted actions and must reproduce rewards, done
flags and observations bit for bit; the oracle's fp64 actors evaluated on the
GPU's recorded observations must agree with the GPU's actions within the
stated tolerance."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import synth

pytestmark = pytest.mark.gpu

REL_TOL = {fr.PREC_FP32: 1e-4, fr.PREC_BF16: 2e-2, fr.PREC_BF16X3: 2e-3, fr.PREC_FP16: 2.5e-3}


def _traj(T, N, D, K, dev, stock=True):
    return {
        "obs": torch.full((T, N, D), np.nan, device=dev),
        "act": (torch.full((T, N, K), np.nan, device=dev) if stock
                else torch.full((T, N), 255, dtype=torch.uint8, device=dev)),
        "rew": torch.zeros(T, N, dtype=torch.int64, device=dev),
        "rew_f32": torch.zeros(T, N, device=dev),
        "done": torch.zeros(T, N, dtype=torch.uint8, device=dev),
    }


def _stock_rollout_check(ctx, dev, w, precision, T, sample_rows=256):
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=precision)
    tr = _traj(T, e.N, env.D, 30, dev)
    met = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, traj=tr, metrics=met)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in tr.items()}
    ref = oracle.stock_run(w.market, e.Ke, e.start, e.W, e.bps, init_cash=e.init_cash, hmax=100,
                           fee_bps=10, T=T, act_f32=g["act"])
    for k in ("obs", "rew", "rew_f32", "done"):
        assert np.array_equal(g[k], ref[k]), k
    assert np.array_equal(met.cpu().numpy(), ref["metrics"])
    # actors on the GPU's own observations
    rng = np.random.default_rng(0)
    rows = rng.choice(T * e.N, size=min(sample_rows, T * e.N), replace=False)
    obs = g["obs"].reshape(-1, env.D)[rows]
    act = g["act"].reshape(-1, 30)[rows].astype(np.float64)
    ys = np.stack([oracle.net_forward(w.dims, w.params[j], obs, 1) for j in range(3)])
    want = np.stack([oracle.ensemble_mean(ys[:, i]) for i in range(len(rows))])
    err = np.linalg.norm(act - want, axis=-1) / np.maximum(np.linalg.norm(want, axis=-1), 1e-3)
    assert err.max() <= REL_TOL[precision], err.max()
    qg = oracle.discretise_many(act.astype(np.float32), 100)
    qw = np.array([oracle.discretise(x, 100) for x in want.ravel()])
    assert np.mean(np.abs(qg - qw) <= 1) >= 0.999
    return g


@pytest.mark.parametrize("dims", [(301, 192, 128, 30), (301, 128, 64, 30)])
def test_fused_stock_rollout_8_warp_shapes_teacher_forced(ctx, dev, dims):
    # hidden widths that are not both multiples of 128 run the resident
    # kernel's 8-warp form (the metric shape runs 16 warps); 1,024 envs span
    # several clusters and a ragged last tile
    from dataclasses import replace
    w = synth.workload_stock_2048(N=1000, T=20)
    w = replace(w, dims=dims, params=synth.actor_params(dims, 3, seed=71))
    _stock_rollout_check(ctx, dev, w, fr.PREC_BF16, 20)


@pytest.mark.parametrize("precision", [fr.PREC_FP32, fr.PREC_BF16, fr.PREC_FP16])
def test_stock_rollout_small_teacher_forced(ctx, dev, precision):
    w = synth.workload_stock_small()
    _stock_rollout_check(ctx, dev, w, precision, w.T)


@pytest.mark.parametrize("precision", [fr.PREC_FP32, fr.PREC_BF16])
def test_stock_rollout_2048_envs_teacher_forced(ctx, dev, precision):
    # the 2,048-env, 301-256-256-30 workload at a shortened horizon
    w = synth.workload_stock_2048(T=24)
    _stock_rollout_check(ctx, dev, w, precision, 24)


@pytest.mark.parametrize("precision", [fr.PREC_FP32, fr.PREC_BF16X3, fr.PREC_FP16])
def test_crypto_rollout_teacher_forced(ctx, dev, precision):
    w = synth.workload_crypto(N=1024, T=64, S=40_000)
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, init_cash=e.init_cash, pmax=e.pmax)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=precision, combine=fr.COMBINE_VOTE,
                             out_act=0)
    T = w.T
    tr = _traj(T, e.N, 10, 1, dev, stock=False)
    met = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, traj=tr, metrics=met)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in tr.items()}
    ref = oracle.crypto_run(w.market, e.start, e.W, init_cash=e.init_cash, pmax=e.pmax, T=T,
                            act_u8=g["act"])
    for k in ("obs", "rew", "rew_f32", "done"):
        assert np.array_equal(g[k], ref[k]), k
    assert np.array_equal(met.cpu().numpy(), ref["metrics"])
    obs = g["obs"].reshape(-1, 10)
    q = np.stack([oracle.net_forward(w.dims, w.params[j], obs, 0) for j in range(5)])
    votes = np.array([oracle.vote(b) for b in q.argmax(-1).T])
    agree = np.mean(votes == g["act"].ravel())
    print(f"prec {precision}: vote agreement {agree:.5f}")
    assert agree >= 0.999


def test_rollout_zero_steps_and_bad_pairs(ctx, dev):
    w = synth.workload_stock_small()
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, bps=e.bps)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_FP32)
    met = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, 0, metrics=met)
    torch.cuda.synchronize()
    assert (met == 0).all()
    bad = fr.ensemble_create(ctx, (301, 64, 3), synth.actor_params((301, 64, 3), 3),
                             combine=fr.COMBINE_VOTE, out_act=0)
    with pytest.raises(fr.FrError):
        fr.rollout(env, bad, 4)


def _stock_env(ctx, mk, e, auto_reset=False):
    return fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps,
                         init_cash=e.init_cash, hmax=e.hmax, fee_bps=e.fee_bps, auto_reset=auto_reset)


@pytest.mark.parametrize("auto_reset", [False, True])
def test_fused_uneven_windows_and_assets(ctx, dev, auto_reset):
    # uneven asset counts and windows in one launch, frozen (or restarted)
    # envs, a ragged last tile: teacher-forced against the oracle
    mk_np = synth.stock_market(300, 30, seed=41)
    e = synth.stock_envs_uneven(300, 30, 300, k_lo=10, w_lo=5, w_hi=60, seed=41)
    params = synth.actor_params(synth.STOCK_DIMS, 3, seed=42)
    mk = fr.fr_market_create(ctx, mk_np)
    env = _stock_env(ctx, mk, e, auto_reset)
    ens = fr.ensemble_create(ctx, synth.STOCK_DIMS, params, precision=fr.PREC_BF16)
    T = 70
    tr = _traj(T, e.N, env.D, 30, dev)
    met = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, traj=tr, metrics=met)
    torch.cuda.synchronize()
    assert fr.ensemble_device_errors(ens) == 0
    g = {k: v.cpu().numpy() for k, v in tr.items()}
    ref = oracle.stock_run(mk_np, e.Ke, e.start, e.W, e.bps, init_cash=e.init_cash, hmax=100,
                           fee_bps=10, T=T, act_f32=g["act"], auto_reset=auto_reset)
    for k in ("obs", "rew", "rew_f32", "done"):
        assert np.array_equal(g[k], ref[k]), k
    assert np.array_equal(met.cpu().numpy(), ref["metrics"])
    cash = torch.empty(e.N, dtype=torch.int64, device=dev)
    hold = torch.empty(e.N, 30, dtype=torch.int32, device=dev)
    steps = torch.empty(e.N, dtype=torch.int32, device=dev)
    fr.env_get_state(env, cash=cash, hold=hold, steps=steps)
    torch.cuda.synchronize()
    assert np.array_equal(cash.cpu().numpy(), ref["cash"][-1])
    assert np.array_equal(hold.cpu().numpy(), ref["hold"][-1])


def test_fused_rollout_in_pieces_equals_one_rollout(ctx, dev):
    w = synth.workload_stock_2048(N=512, T=60)        # 61-day windows: 40 steps leave 20
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    env1 = _stock_env(ctx, mk, e)
    env2 = _stock_env(ctx, mk, e)
    r1 = torch.zeros(40, e.N, dtype=torch.int64, device=dev)
    r2 = torch.zeros(40, e.N, dtype=torch.int64, device=dev)
    m1 = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    m2 = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env1, ens, 40, traj={"rew": r1}, metrics=m1)
    fr.rollout(env2, ens, 15, traj={"rew": r2[:15]})
    fr.rollout(env2, ens, 25, traj={"rew": r2[15:]}, metrics=m2)
    torch.cuda.synchronize()
    assert torch.equal(r1, r2) and torch.equal(m1, m2)
    # and the unfused env step continues from the fused rollout's state
    q = torch.zeros(e.N, 30, dtype=torch.int32, device=dev)
    rw = torch.empty(e.N, dtype=torch.int64, device=dev)
    fr.env_step(env2, q, fr.ACT_I32_SHARES, rew=rw)
    steps = torch.empty(e.N, dtype=torch.int32, device=dev)
    fr.env_get_state(env2, steps=steps)
    torch.cuda.synchronize()
    assert (steps == 41).all()


def test_fused_and_unfused_paths_agree_on_prices_and_accounting(ctx, dev):
    # both paths replayed by the oracle stay bit-exact; their actions differ
    # only by the exchange precision of the agents' outputs
    w = synth.workload_stock_small()
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    acts = []
    for path in (fr.PATH_AUTO, fr.PATH_UNFUSED):
        env = _stock_env(ctx, mk, e)
        fr.env_set_rollout_path(env, path)
        tr = _traj(w.T, e.N, env.D, 30, dev)
        fr.rollout(env, ens, w.T, traj=tr)
        torch.cuda.synchronize()
        acts.append(tr["act"].cpu().numpy())
    # the first step acts on identical observations
    assert np.abs(acts[0][0] - acts[1][0]).max() < 1e-2


def test_kernel_timing_hook(ctx, dev):
    w = synth.workload_stock_2048(N=256, T=8)
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    env = _stock_env(ctx, mk, e)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    with pytest.raises(fr.FrError):
        fr.env_last_kernel_ms(env)                 # nothing recorded yet
    fr.env_set_kernel_timing(env, True)
    with pytest.raises(fr.FrError):
        fr.env_last_kernel_ms(env)
    with pytest.raises(fr.FrError):
        fr.env_last_launch_shape(env)              # no fused launch yet
    fr.rollout(env, ens, 8)
    ms = fr.env_last_kernel_ms(env)
    assert 0.0 < ms < 1e3
    # 256 envs do not fill the co-resident clusters: tiles of the 64-env minimum
    ctas, tile = fr.env_last_launch_shape(env)
    assert tile == 64 and ctas == 6 * 4
    fr.env_set_kernel_timing(env, False)
    with pytest.raises(fr.FrError):
        fr.env_last_kernel_ms(env)


@pytest.mark.parametrize("N", [700, 1000])
def test_packed_tiles_equal_unpacked(ctx, dev, N):
    # Without trajectory outputs the fused kernel packs envs by window into
    # tiles (longest first) and stops each tile after its longest window; with
    # a trajectory it runs the envs in their own order for all T steps.  Every
    # env's arithmetic is the same either way: equal metrics and final state.
    mk_np = synth.stock_market(400, 30, seed=51)
    e = synth.stock_envs_uneven(N, 30, 400, k_lo=10, w_lo=5, w_hi=120, seed=51)
    params = synth.actor_params(synth.STOCK_DIMS, 3, seed=52)
    mk = fr.fr_market_create(ctx, mk_np)
    ens = fr.ensemble_create(ctx, synth.STOCK_DIMS, params, precision=fr.PREC_BF16)
    T = 130
    out = []
    for with_traj in (False, True):
        env = _stock_env(ctx, mk, e)
        met = torch.empty(N, 3, dtype=torch.float64, device=dev)
        tr = _traj(T, N, env.D, 30, dev) if with_traj else None
        # two pieces: the packed path keeps each env's steps and state across calls
        fr.rollout(env, ens, 50, traj=None if tr is None else {k: v[:50] for k, v in tr.items()}, metrics=met)
        fr.rollout(env, ens, T - 50, traj=None if tr is None else {k: v[50:] for k, v in tr.items()}, metrics=met)
        cash = torch.empty(N, dtype=torch.int64, device=dev)
        hold = torch.empty(N, 30, dtype=torch.int32, device=dev)
        steps = torch.empty(N, dtype=torch.int32, device=dev)
        done = torch.empty(N, dtype=torch.uint8, device=dev)
        fr.env_get_state(env, cash=cash, hold=hold, steps=steps, done=done)
        torch.cuda.synchronize()
        out.append([x.cpu().numpy() for x in (met, cash, hold, steps, done)])
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
    assert out[0][4].all()                                  # every window finished within T
    # and with packing switched off, no trajectory
    env = _stock_env(ctx, mk, e)
    fr.env_set_tile_packing(env, False)
    met = torch.empty(N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, metrics=met)
    torch.cuda.synchronize()
    assert np.array_equal(met.cpu().numpy(), out[0][0])
    assert fr.env_tile_packing_efficiency(env) == 1.0


@pytest.mark.parametrize("case", ["stock_bf16_fused", "stock_fp32_plain", "crypto_bf16x3_fused"])
def test_rollout_graph_capture(ctx, dev, case):
    # after one warm-up call (cached tables, scratch, kernel attributes) a
    # reset + rollout can be captured into a CUDA graph; replays equal direct calls
    if case.startswith("stock"):
        w = synth.workload_stock_2048(N=384, T=24)
        e = w.envs
        mk = fr.fr_market_create(ctx, w.market)
        env = _stock_env(ctx, mk, e)
        ens = fr.ensemble_create(ctx, w.dims, w.params,
                                 precision=fr.PREC_BF16 if "bf16" in case else fr.PREC_FP32)
    else:
        w = synth.workload_crypto(N=384, T=24, S=40_000)
        e = w.envs
        mk = fr.fr_market_create(ctx, w.market)
        env = fr.env_create(ctx, mk, start=e.start, window=e.W, init_cash=e.init_cash, pmax=e.pmax)
        ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16X3, combine=fr.COMBINE_VOTE,
                                 out_act=0)
    T = w.T
    met = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            fr.env_reset(env)
            fr.rollout(env, ens, T, metrics=met)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    ref = met.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fr.env_reset(env)
        fr.rollout(env, ens, T, metrics=met)
    for _ in range(3):
        met.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(met, ref)


def test_split_rollout_equals_one_launch_and_replays_in_a_graph(ctx, dev):
    # 200 steps without trajectory outputs run as three launches (66, 67, 67
    # steps), each piece's FP64 replay beside the next piece's launch; state
    # and metrics equal the single launch bit for bit, directly and as a
    # graph replay
    w = synth.workload_stock_2048(N=700, T=200)
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    out = []
    for split in (False, True):
        env = _stock_env(ctx, mk, e)
        fr.env_set_rollout_split(env, split)
        met = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
        fr.rollout(env, ens, 200, metrics=met)
        cash = torch.empty(e.N, dtype=torch.int64, device=dev)
        hold = torch.empty(e.N, 30, dtype=torch.int32, device=dev)
        steps = torch.empty(e.N, dtype=torch.int32, device=dev)
        done = torch.empty(e.N, dtype=torch.uint8, device=dev)
        fr.env_get_state(env, cash=cash, hold=hold, steps=steps, done=done)
        torch.cuda.synchronize()
        out.append([x.cpu().numpy() for x in (met, cash, hold, steps, done)])
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)
    # a second split rollout (two pieces) continues from the first
    met2 = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, 130, metrics=met2)
    env1 = _stock_env(ctx, mk, e)
    fr.env_set_rollout_split(env1, False)
    met1 = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env1, ens, 200, metrics=met1)
    fr.rollout(env1, ens, 130, metrics=met1)
    torch.cuda.synchronize()
    assert torch.equal(met2, met1)
    # captured: reset + split rollout, replayed
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    met3 = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    with torch.cuda.stream(side):
        fr.env_reset(env)
        fr.rollout(env, ens, 200, metrics=met3)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fr.env_reset(env)
        fr.rollout(env, ens, 200, metrics=met3)
    for _ in range(2):
        met3.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(met3.cpu().numpy(), out[0][0])


def test_indicator_table_rebuilt_each_rollout_equals_kept(ctx, dev):
    # the fused stock kernel's indicator table rebuilt by every rollout (as
    # the benchmark's headline times it, inside a captured graph) gives the
    # same rollout bit for bit as the kept table
    w = synth.workload_stock_2048(N=256, T=24)
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps)
    out = []
    for keep in (True, False, False):
        fr.env_set_table_cache(env, keep)
        fr.env_reset(env)
        met = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
        fr.rollout(env, ens, w.T, metrics=met)
        out.append(met)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    met_g = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    with torch.cuda.graph(g, stream=side):
        fr.env_reset(env)
        fr.rollout(env, ens, w.T, metrics=met_g)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out[0], out[1]) and torch.equal(out[1], out[2]) and torch.equal(out[0], met_g)


def test_fused_stock_rollout_64_bit_accounting(ctx, dev):
    # prices scaled x3,000 fail env_create's 32-bit range proof, so the
    # resident-weight fused kernel runs its owners' 64-bit accounting (the
    # bench's market takes the 32-bit one); teacher-forced bit-exact either way
    from types import SimpleNamespace
    w = synth.workload_stock_2048(N=256, T=24)
    e = w.envs
    mkt = SimpleNamespace(close=np.ascontiguousarray(w.market.close * 3000), ind=w.market.ind,
                          high=w.market.high * 3000, low=w.market.low * 3000)
    mk = fr.fr_market_create(ctx, mkt)
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps,
                        init_cash=100_000_000_000)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    T = w.T
    tr = _traj(T, e.N, env.D, 30, dev)
    met = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, traj=tr, metrics=met)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in tr.items()}
    ref = oracle.stock_run(mkt, e.Ke, e.start, e.W, e.bps, init_cash=100_000_000_000, hmax=100,
                           fee_bps=10, T=T, act_f32=g["act"])
    for k in ("obs", "rew", "rew_f32", "done"):
        assert np.array_equal(g[k], ref[k]), k
    assert np.array_equal(met.cpu().numpy(), ref["metrics"])
