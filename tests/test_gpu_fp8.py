"""FP8 E4M3 actors (tcgen05 kind::f8f6f4) against the oracle's FP8 model.

Exact checks: single-layer networks whose outputs are one E4M3 product times
a float32 factor (one-hot inputs expose every weight code and its channel
scale; an identity layer exposes the activation codes), bit for bit.
Whole networks: per row ||a_gpu - a_fp8||_2 / max(||a_fp8||_2, 1e-3) <= 2e-2
against the oracle's FP8 forward with the GPU's calibrated scales (the two
differ only in fp32 vs exact accumulation, and in the rare activation codes
that this flips); crypto argmax agreement >= 99%.  Calibrated scales within
1e-5 of the oracle's fp64 calibration."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import synth

pytestmark = pytest.mark.gpu

FP8_TOL = 2e-2


def _fwd(ens, obs, dev, out):
    n = obs.shape[0]
    y = torch.full((ens.M, n, out), np.nan, device=dev)
    fr.ensemble_forward(ens, torch.from_numpy(np.ascontiguousarray(obs, np.float32)).to(dev), y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def _zero_bias(dims, params):
    params = params.copy()
    off = 0
    for fin, fout in zip(dims[:-1], dims[1:]):
        off += fin * fout
        params[:, off:off + fout] = 0
        off += fout
    return params


@pytest.mark.parametrize("fin, fout", [(301, 30), (64, 256), (10, 48), (37, 3), (512, 16)])
def test_fp8_weight_codes_and_channel_scales_exact(ctx, dev, fin, fout):
    # one-hot rows of 1.0 with activation scale 1: output (k, n) is
    # RN32(code(W[n][k] / sw[n]) * sw[n]) -- every code, its place in the
    # tcgen05 layout and every channel scale
    dims = (fin, fout)
    params = _zero_bias(dims, synth.actor_params(dims, 2, seed=fin + fout))
    params[1, :fout] = 0.0                       # agent 1: first column zero (rows keep other entries)
    ens = fr.ensemble_create(ctx, dims, params, precision=fr.PREC_FP8, out_act=0)
    fr.ensemble_set_act_scales(ens, np.ones((2, 1), np.float32))
    obs = np.eye(fin, dtype=np.float32)
    got = _fwd(ens, obs, dev, fout)
    for j in range(2):
        want = oracle.fp8_forward(dims, params[j], [1.0], obs, 0).astype(np.float32)
        assert np.array_equal(got[j], want), j
    assert fr.ensemble_device_errors(ens) == 0


@pytest.mark.parametrize("F, scale", [(256, 0.0371), (48, 1.7), (160, 0.0003)])
def test_fp8_activation_codes_exact(ctx, dev, F, scale):
    # an identity layer: output n is RN32(448 code(x_n / sx) * sx / 448)
    dims = (F, F)
    W = np.eye(F, dtype=np.float32)
    params = np.concatenate([W.ravel(), np.zeros(F, np.float32)])[None]
    ens = fr.ensemble_create(ctx, dims, params, precision=fr.PREC_FP8, out_act=0)
    fr.ensemble_set_act_scales(ens, np.full((1, 1), scale, np.float32))
    rng = np.random.default_rng(F)
    obs = (rng.normal(0, 1, (300, F)) * np.logspace(-3, 3, F)).astype(np.float32)   # spans saturation
    got = _fwd(ens, obs, dev, F)[0]
    want = oracle.fp8_forward(dims, params[0], [scale], obs, 0).astype(np.float32)
    assert np.array_equal(got, want)


def _stock_obs(n, seed=41):
    w = synth.workload_stock_2048(N=256, T=64)
    q = synth.prescribed_shares(64, 256, 30, seed=seed)
    o = oracle.stock_run(w.market, w.envs.Ke, w.envs.start, w.envs.W, w.envs.bps, init_cash=w.envs.init_cash,
                         hmax=100, fee_bps=10, T=64, act_i32=q, want=("obs",))
    obs = o["obs"].reshape(-1, o["obs"].shape[-1])
    return np.ascontiguousarray(obs[np.linspace(0, obs.shape[0] - 1, n).astype(int)])


def _crypto_obs(n, seed=42):
    w = synth.workload_crypto(N=512, T=64, S=60_000)
    acts = synth.prescribed_discrete(64, 512, seed=seed)
    o = oracle.crypto_run(w.market, w.envs.start, w.envs.W, init_cash=w.envs.init_cash, pmax=10, T=64,
                          act_u8=acts, want=("obs",))
    obs = o["obs"].reshape(-1, 10)
    return np.ascontiguousarray(obs[np.linspace(0, obs.shape[0] - 1, n).astype(int)])


def _rel(got, want):
    return np.linalg.norm(got - want, axis=-1) / np.maximum(np.linalg.norm(want, axis=-1), 1e-3)


@pytest.mark.parametrize("dims, n", [((301, 256, 256, 30), 2048), ((301, 256, 256, 30), 129),
                                     ((301, 64, 48, 30), 500)])
def test_fp8_stock_actors_match_oracle_fp8(ctx, dev, dims, n):
    params = synth.actor_params(dims, 3, seed=7)
    calib = _stock_obs(4096, seed=43)
    obs = _stock_obs(n)
    ens = fr.ensemble_create(ctx, dims, params, precision=fr.PREC_FP8)
    sx = fr.ensemble_calibrate_sync(ens, torch.from_numpy(calib).to(dev))
    for j in range(3):
        want = oracle.fp8_calibrate(dims, params[j], calib)
        assert np.allclose(sx[j], want, rtol=1e-5, atol=0), (j, sx[j], want)
    got = _fwd(ens, obs, dev, 30)
    err, err64 = [], []
    for j in range(3):
        want = oracle.fp8_forward(dims, params[j], sx[j], obs, 1)
        err.append(_rel(got[j], want))
        err64.append(_rel(got[j], oracle.net_forward(dims, params[j], obs, 1)))
    err, err64 = np.concatenate(err), np.concatenate(err64)
    print(f"FP8 {dims} n={n}: vs oracle FP8 max {err.max():.2e}; vs fp64 model max {err64.max():.2e} "
          f"mean {err64.mean():.2e}")
    assert np.isfinite(got).all()
    assert err.max() <= FP8_TOL
    assert fr.ensemble_device_errors(ens) == 0


def test_fp8_crypto_argmax_agreement(ctx, dev):
    w = synth.workload_crypto(N=64, T=8, S=20_000)
    n = 4096
    obs = _crypto_obs(n)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_FP8, combine=fr.COMBINE_VOTE, out_act=0)
    sx = fr.ensemble_calibrate_sync(ens, torch.from_numpy(obs).to(dev))
    got = _fwd(ens, obs, dev, 3)
    M = w.params.shape[0]
    q8 = np.stack([oracle.fp8_forward(w.dims, w.params[j], sx[j], obs, 0) for j in range(M)])
    agree = np.mean(got.argmax(-1) == q8.argmax(-1))
    print(f"FP8 crypto argmax agreement with the oracle FP8 model {agree:.5f}")
    assert agree >= 0.99
    votes_gpu = torch.empty(n, dtype=torch.uint8, device=dev)
    fr.ensemble_act(ens, torch.from_numpy(obs).to(dev), votes_gpu)
    torch.cuda.synchronize()
    votes = np.array([oracle.vote(b) for b in got.argmax(-1).T])
    assert np.array_equal(votes_gpu.cpu().numpy(), votes)     # the vote of the GPU's own Q-values


def _fp8_stock_rollout(ctx, dev, w, path, scales=None, T=24):
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps)
    if path == "unfused":
        fr.env_set_rollout_path(env, fr.PATH_UNFUSED)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_FP8)
    if scales is None:
        sx = fr.ensemble_calibrate_sync(ens, torch.from_numpy(_stock_obs(4096, seed=44)).to(dev))
    else:
        fr.ensemble_set_act_scales(ens, scales)
        sx = scales
    tr = {"obs": torch.full((T, e.N, env.D), np.nan, device=dev),
          "act": torch.full((T, e.N, 30), np.nan, device=dev),
          "rew": torch.zeros(T, e.N, dtype=torch.int64, device=dev),
          "done": torch.zeros(T, e.N, dtype=torch.uint8, device=dev)}
    met = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, traj=tr, metrics=met)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in tr.items()}
    ref = oracle.stock_run(w.market, e.Ke, e.start, e.W, e.bps, init_cash=e.init_cash, hmax=100, fee_bps=10, T=T,
                           act_f32=g["act"])
    for k in ("obs", "rew", "done"):
        assert np.array_equal(g[k], ref[k]), k
    assert np.array_equal(met.cpu().numpy(), ref["metrics"])
    return env, ens, sx, g


@pytest.mark.parametrize("path", ["fused", "unfused"])
def test_fp8_stock_rollout_teacher_forced(ctx, dev, path):
    # env bit-exact on the emitted actions either way.  Unfused: every input
    # of the first layer quantised (the actor kernel).  Fused (the agents
    # share the first layer's scale, as calibration on observations gives):
    # the 61 state entries quantised, the indicator block through the exact
    # fp32 table.  Actions within the FP8 tolerance of the matching oracle
    # model, discretised shares within one of it
    w = synth.workload_stock_2048(N=512, T=24)
    env, ens, sx, g = _fp8_stock_rollout(ctx, dev, w, path)
    assert np.all(sx[:, 0] == sx[0, 0])
    T, N = 24, w.envs.N
    rows = np.random.default_rng(1).choice(T * N, 512, replace=False)
    obs = g["obs"].reshape(-1, env.D)[rows]
    act = g["act"].reshape(-1, 30)[rows].astype(np.float64)
    if path == "fused":
        ys = np.stack([oracle.fp8_forward_exact_tail(w.dims, w.params[j], sx[j], obs, 1, 61) for j in range(3)])
    else:
        ys = np.stack([oracle.fp8_forward(w.dims, w.params[j], sx[j], obs, 1) for j in range(3)])
    want = np.stack([oracle.ensemble_mean(ys[:, i]) for i in range(len(rows))])
    err = _rel(act, want)
    print(f"{path}: rel err max {err.max():.3e} median {np.median(err):.3e}")
    assert err.max() <= FP8_TOL
    qg = oracle.discretise_many(act.astype(np.float32), 100)
    qw = np.array([oracle.discretise(x, 100) for x in want.ravel()])
    assert np.mean(np.abs(qg - qw) <= 1) >= 0.999


def test_fp8_fused_rollout_follows_new_scales_and_unshared_scales_fall_back(ctx, dev):
    # the fused kernel's image is repacked when the activation scales change;
    # agents with different first-layer scales run the unfused path (one set
    # of observation codes cannot serve them), whose model is fp8_forward
    w = synth.workload_stock_2048(N=256, T=16)
    env, ens, sx, g0 = _fp8_stock_rollout(ctx, dev, w, "fused", T=16)
    sx2 = (sx * np.float32(1.5)).astype(np.float32)
    fr.ensemble_set_act_scales(ens, sx2)
    fr.env_reset(env)
    act = torch.full((16, w.envs.N, 30), np.nan, device=dev)
    obs = torch.full((16, w.envs.N, env.D), np.nan, device=dev)
    fr.rollout(env, ens, 16, traj={"act": act, "obs": obs})
    torch.cuda.synchronize()
    a, o = act.cpu().numpy().reshape(-1, 30), obs.cpu().numpy().reshape(-1, env.D)
    rows = np.random.default_rng(2).choice(a.shape[0], 256, replace=False)
    ys = np.stack([oracle.fp8_forward_exact_tail(w.dims, w.params[j], sx2[j], o[rows], 1, 61) for j in range(3)])
    want = np.stack([oracle.ensemble_mean(ys[:, i]) for i in range(len(rows))])
    assert _rel(a[rows].astype(np.float64), want).max() <= FP8_TOL
    assert not np.array_equal(a, g0["act"].reshape(-1, 30))
    # unshared layer-0 scales
    sx3 = sx.copy()
    sx3[1, 0] *= np.float32(1.25)
    _, _, _, g3 = _fp8_stock_rollout(ctx, dev, w, "fused", scales=sx3, T=16)
    o3, a3 = g3["obs"].reshape(-1, env.D)[rows], g3["act"].reshape(-1, 30)[rows].astype(np.float64)
    ys = np.stack([oracle.fp8_forward(w.dims, w.params[j], sx3[j], o3, 1) for j in range(3)])
    want = np.stack([oracle.ensemble_mean(ys[:, i]) for i in range(len(rows))])
    assert _rel(a3, want).max() <= FP8_TOL


def test_fp8_fused_packed_tiles_and_graph_replay(ctx, dev):
    # uneven windows: packed tiles (no trajectory) equal the unpacked run;
    # a captured reset + rollout replays to the same metrics
    N, T = 700, 130
    mk_np = synth.stock_market(400, 30, seed=51)
    e = synth.stock_envs_uneven(N, 30, 400, k_lo=10, w_lo=5, w_hi=120, seed=51)
    params = synth.actor_params(synth.STOCK_DIMS, 3, seed=52)
    mk = fr.fr_market_create(ctx, mk_np)
    ens = fr.ensemble_create(ctx, synth.STOCK_DIMS, params, precision=fr.PREC_FP8)
    fr.ensemble_calibrate_sync(ens, torch.from_numpy(_stock_obs(2048, seed=46)).to(dev))
    mets = []
    for packing in (True, False):
        env = fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps)
        fr.env_set_tile_packing(env, packing)
        met = torch.empty(N, 3, dtype=torch.float64, device=dev)
        fr.rollout(env, ens, T, metrics=met)
        torch.cuda.synchronize()
        mets.append(met.cpu().numpy())
    assert np.array_equal(mets[0], mets[1])
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    met = torch.empty(N, 3, dtype=torch.float64, device=dev)
    with torch.cuda.stream(side):
        fr.env_reset(env)
        fr.rollout(env, ens, T, metrics=met)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fr.env_reset(env)
        fr.rollout(env, ens, T, metrics=met)
    for _ in range(2):
        met.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(met.cpu().numpy(), mets[1])


def test_fp8_scales_required_and_checked(ctx, dev):
    dims = (301, 64, 64, 30)
    params = synth.actor_params(dims, 2, seed=9)
    ens = fr.ensemble_create(ctx, dims, params, precision=fr.PREC_FP8)
    obs = torch.zeros(4, 301, device=dev)
    y = torch.empty(2, 4, 30, device=dev)
    with pytest.raises(fr.FrError) as ei:
        fr.ensemble_forward(ens, obs, y)
    assert ei.value.code == fr._lib.FR_ENOTREADY
    with pytest.raises(fr.FrError):
        fr.ensemble_get_act_scales(ens)
    for bad in (0.0, -1.0, np.inf, np.nan):
        with pytest.raises(fr.FrError):
            fr.ensemble_set_act_scales(ens, np.full((2, 3), bad, np.float32))
    fr.ensemble_set_act_scales(ens, np.full((2, 3), 0.5, np.float32))
    assert np.array_equal(fr.ensemble_get_act_scales(ens), np.full((2, 3), 0.5, np.float32))
    fr.ensemble_forward(ens, obs, y)
    torch.cuda.synchronize()
    bf = fr.ensemble_create(ctx, dims, params, precision=fr.PREC_BF16)
    with pytest.raises(fr.FrError):
        fr.ensemble_set_act_scales(bf, np.ones((2, 3), np.float32))
    with pytest.raises(fr.FrError):
        fr.ensemble_calibrate_sync(bf, obs)


def test_fp8_validation_keeps_each_agents_scales(ctx, dev):
    w = synth.workload_stock_2048(N=256, T=8)
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    env = fr.env_create(ctx, mk, start=e.start, window=np.full(e.N, 6, np.int32), n_assets=e.Ke, bps=e.bps)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_FP8)
    sx = fr.ensemble_calibrate_sync(ens, torch.from_numpy(_stock_obs(1024, seed=45)).to(dev))
    S, wts = fr.ensemble_validate(ens, env, 5)
    assert np.isfinite(S).all() and abs(float(wts.sum()) - 1.0) < 1e-5
    assert np.array_equal(fr.ensemble_get_act_scales(ens), sx)
    # each agent's Sharpe is that of the agent alone with its own scales
    for j in range(3):
        one = fr.ensemble_create(ctx, w.dims, w.params[j:j + 1], precision=fr.PREC_FP8)
        fr.ensemble_set_act_scales(one, sx[j:j + 1])
        env1 = fr.env_create(ctx, mk, start=e.start, window=np.full(e.N, 6, np.int32), n_assets=e.Ke, bps=e.bps)
        met = torch.empty(e.N, 3, dtype=torch.float64, device=dev)
        fr.rollout(env1, one, 5, metrics=met)
        torch.cuda.synchronize()
        acc = 0.0
        for v in met.cpu().numpy()[:, 1]:          # summed in env order, as the library does
            acc += float(v)
        assert S[j] == acc / e.N
