"""ensemble_act_noalloc -- the entry point for callers that cannot allocate
device memory while they run -- must give the same actions as ensemble_act,
call after call, from its fixed scratch array.

This file is collected last on purpose; it must pass alone in a fresh
process as well as after the rest of the suite."""
import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import build, synth

pytestmark = pytest.mark.gpu

REL_TOL = {fr.PREC_FP32: 1e-4, fr.PREC_BF16: 2e-2}


def _obs(n, dims):
    st = synth.Stream(77, 1)
    return (st.normal(n * dims[0]) * 0.5).reshape(n, dims[0]).astype(np.float32)


@pytest.mark.parametrize("precision", [fr.PREC_FP32, fr.PREC_BF16])
def test_noalloc_matches_ensemble_act_twice(precision):
    build.build()
    ctx = fr.fr_ctx_create(0)
    dev = torch.device("cuda:0")
    dims = synth.STOCK_DIMS
    params = synth.actor_params(dims, 3, seed=12)
    ens = fr.ensemble_create(ctx, dims, params, precision=precision)
    n = 1500
    obs = torch.from_numpy(_obs(n, dims)).to(dev)
    ref = torch.empty(n, 30, device=dev)
    fr.ensemble_act(ens, obs, ref)
    for _ in range(2):
        got = torch.full((n, 30), float("nan"), device=dev)
        fr.ensemble_act_noalloc(ens, obs, got)
        torch.cuda.synchronize()
        g, r = got.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(g - r, axis=-1) / np.maximum(np.linalg.norm(r, axis=-1), 1e-3)
        assert np.isfinite(g).all() and err.max() <= REL_TOL[precision], err.max()
        if precision == fr.PREC_BF16:
            # below one 128-row tile per SM ensemble_act runs the same
            # single-agent tensor-core kernel: identical results
            assert torch.equal(got, ref)
    # and against the fp64 oracle on a sample of rows
    o = obs.cpu().numpy()[:64]
    want = np.stack([oracle.ensemble_mean(np.stack([oracle.net_forward(dims, params[j], o[i:i + 1], 1)[0]
                                                    for j in range(3)])) for i in range(64)])
    err = np.linalg.norm(g[:64] - want, axis=-1) / np.maximum(np.linalg.norm(want, axis=-1), 1e-3)
    assert err.max() <= REL_TOL[precision]


def test_noalloc_bf16_equals_the_large_batch_kernel():
    """40,000 rows (313 tiles of 128, above one per SM): ensemble_act runs the
    tiling pass and the large-batch kernel, the allocation-free call the
    single-agent kernel; same products, order and roundings, so the actions
    are identical."""
    build.build()
    ctx = fr.fr_ctx_create(0)
    dev = torch.device("cuda:0")
    dims = synth.STOCK_DIMS
    params = synth.actor_params(dims, 3, seed=14)
    ens = fr.ensemble_create(ctx, dims, params, precision=fr.PREC_BF16)
    n = 40_000                     # 3 x 30 outputs per row: within the fixed scratch
    assert n > ctx.sm_count * 128
    obs = torch.from_numpy(_obs(n, dims)).to(dev)
    ref = torch.empty(n, 30, device=dev)
    fr.ensemble_act(ens, obs, ref)
    got = torch.full((n, 30), float("nan"), device=dev)
    fr.ensemble_act_noalloc(ens, obs, got)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


def test_noalloc_vote_and_size_limit():
    build.build()
    ctx = fr.fr_ctx_create(0)
    dev = torch.device("cuda:0")
    dims = synth.CRYPTO_DIMS
    params = synth.actor_params(dims, 5, seed=13, out_scale=4.0)
    ens = fr.ensemble_create(ctx, dims, params, precision=fr.PREC_FP32, combine=fr.COMBINE_VOTE,
                             out_act=0)
    n = 3000                       # within the fixed scratch for 5 fp32 agents
    obs = torch.from_numpy(_obs(n, dims)).to(dev)
    ref = torch.empty(n, dtype=torch.uint8, device=dev)
    fr.ensemble_act(ens, obs, ref)
    for _ in range(2):
        got = torch.full((n,), 255, dtype=torch.uint8, device=dev)
        fr.ensemble_act_noalloc(ens, obs, got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
    # a batch beyond the fixed scratch is refused on the host before any
    # launch (the size check comes first, so the short buffers are untouched)
    too_many = 1 << 20
    rc = fr.lib().ensemble_act_noalloc(ens, obs.data_ptr(), too_many, got.data_ptr(), None)
    assert rc == fr._lib.FR_EINVAL
    assert "scratch" in fr.lib().fr_last_error().decode()
