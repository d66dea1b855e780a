"""Backtest server (backtest_submit / backtest_poll, continuous batching).

Every request's metrics must equal, bit for bit, a standalone rollout of the
same envs through the same path: rows are independent in every kernel and
finished envs stay frozen, so chunked execution inside a shared pool of
slots, next to other requests' envs, may not change any result.  The
standalone rollout's own parity with the oracle is covered by the rollout
tests."""
import ctypes as C
import time

import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

def _request_bps(n, K, seed, rng):
    """The per-env, per-asset perturbation the server draws, from the oracle."""
    b = np.zeros((n, K), np.int16)
    if rng > 0:
        for i in range(n):
            for k in range(K):
                b[i, k] = oracle.perturb_bps(seed, i, k, rng)
    return b


def _wait_all(srv, tickets, timeout_s=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = fr.backtest_poll(srv, t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout_s, "server did not finish in time"
        time.sleep(0.002)
    return out


def _standalone(ctx, mk, ens, dev, req, K, stock=True):
    n = req["n_envs"]
    start = req["start"] + np.arange(n) * req.get("start_stride", 0)
    if stock:
        ke = req.get("n_assets", 0) or K
        env = fr.env_create(ctx, mk, start=start, window=req["window"], n_assets=ke,
                            bps=_request_bps(n, K, req.get("seed", 0), req.get("bps_range", 0)))
    else:
        env = fr.env_create(ctx, mk, start=start, window=req["window"])
    met = torch.empty(n, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, req["window"] - 1, metrics=met)
    torch.cuda.synchronize()
    return met.cpu().numpy()


STOCK_REQS = [
    dict(n_envs=10, window=20, start=100, start_stride=3, bps_range=100, seed=1),
    dict(n_envs=100, window=50, start=200, start_stride=1, bps_range=100, seed=2),
    dict(n_envs=40, window=5, start=300, start_stride=0, bps_range=0, seed=3),
    dict(n_envs=128, window=33, start=400, start_stride=2, bps_range=50, seed=4, n_assets=20),
    dict(n_envs=7, window=17, start=500, start_stride=5, bps_range=100, seed=5),
    dict(n_envs=60, window=64, start=600, start_stride=1, bps_range=100, seed=6),
]


@pytest.mark.parametrize("precision", [fr.PREC_BF16, fr.PREC_FP32])
def test_stock_server_matches_standalone_rollouts(ctx, dev, precision):
    w = synth.workload_stock_2048(N=128, T=16)
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=precision)
    srv = fr.fr_server_create(ctx, mk, ens, capacity=256, chunk_steps=16)
    tickets = [fr.backtest_submit(srv, **r) for r in STOCK_REQS]    # 345 envs > 256 slots: some queue
    res = _wait_all(srv, tickets)
    st = fr.fr_server_stats(srv)
    srv.close()
    assert st["completed"] == len(STOCK_REQS) and st["queued"] == 0 and st["running"] == 0
    for t, r in zip(tickets, STOCK_REQS):
        got = res[t]
        assert got["status"] == 0 and got["n_envs"] == r["n_envs"]
        assert 0.0 <= got["queue_s"] <= got["latency_s"]
        want = _standalone(ctx, mk, ens, dev, r, 30)
        assert np.array_equal(got["metrics"], want), r


def test_crypto_server_matches_standalone_rollouts(ctx, dev):
    w = synth.workload_crypto(N=64, T=64, S=40_000)
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16X3, combine=fr.COMBINE_VOTE,
                             out_act=0)
    srv = fr.fr_server_create(ctx, mk, ens, capacity=192, chunk_steps=32)
    reqs = [dict(n_envs=64, window=100, start=4000, start_stride=37),
            dict(n_envs=100, window=300, start=9000, start_stride=11),
            dict(n_envs=50, window=41, start=20000, start_stride=101)]
    tickets = [fr.backtest_submit(srv, **r) for r in reqs]
    res = _wait_all(srv, tickets)
    srv.close()
    for t, r in zip(tickets, reqs):
        assert res[t]["status"] == 0
        assert np.array_equal(res[t]["metrics"], _standalone(ctx, mk, ens, dev, r, 1, stock=False)), r


def test_server_queues_in_arrival_order(ctx, dev):
    w = synth.workload_stock_2048(N=128, T=16)
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    srv = fr.fr_server_create(ctx, mk, ens, capacity=64, chunk_steps=8)
    reqs = [dict(n_envs=40, window=40, start=100 + 10 * i, bps_range=100, seed=10 + i) for i in range(3)]
    tickets = [fr.backtest_submit(srv, **r) for r in reqs]          # 40 + 40 > 64: one at a time
    res = _wait_all(srv, tickets)
    srv.close()
    lat = [res[t]["latency_s"] for t in tickets]
    q = [res[t]["queue_s"] for t in tickets]
    assert lat[0] < lat[1] < lat[2]                                  # arrival order
    assert q[1] >= lat[0] - q[0] - 0.05 and q[2] > q[1]               # each waited for the one ahead
    for t, r in zip(tickets, reqs):
        assert np.array_equal(res[t]["metrics"], _standalone(ctx, mk, ens, dev, r, 30)), r


def test_server_errors(ctx, dev):
    w = synth.workload_stock_2048(N=128, T=16)
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    srv = fr.fr_server_create(ctx, mk, ens, capacity=32, chunk_steps=8)
    with pytest.raises(fr.FrError):                                    # can never fit
        fr.backtest_submit(srv, n_envs=33, window=10, start=100)
    with pytest.raises(fr.FrError):                                    # past the market end
        fr.backtest_submit(srv, n_envs=2, window=10, start=995)
    with pytest.raises(fr.FrError):
        fr.backtest_submit(srv, n_envs=2, window=1, start=100)
    with pytest.raises(fr.FrError):
        fr.backtest_submit(srv, n_envs=2, window=10, start=100, n_assets=31)
    met = np.zeros((2, 3))
    r = _lib.Request(2, 10, 100, 0, 0, 0, 0, 1, met.ctypes.data_as(C.c_void_p))   # want_traj
    t = C.c_uint64()
    assert fr.lib().backtest_submit(srv, C.byref(r), C.byref(t)) == _lib.FR_EINVAL
    res, done = _lib.Result(), C.c_int32()
    assert fr.lib().backtest_poll(srv, C.c_uint64(12345), C.byref(res), C.byref(done)) == _lib.FR_ENOTFOUND
    tk = fr.backtest_submit(srv, n_envs=4, window=12, start=100)
    out = _wait_all(srv, [tk])[tk]
    assert out["status"] == 0
    assert fr.lib().backtest_poll(srv, C.c_uint64(tk), C.byref(res), C.byref(done)) == _lib.FR_ENOTFOUND
    srv.close()
    with pytest.raises(fr.FrError):                                    # mismatched ensemble
        bad = fr.ensemble_create(ctx, (301, 64, 3), synth.actor_params((301, 64, 3), 3),
                                 combine=fr.COMBINE_VOTE, out_act=0)
        fr.fr_server_create(ctx, mk, bad, capacity=8)


def _crypto_server(ctx, capacity=64, chunk=8):
    w = synth.workload_crypto(N=64, T=64, S=200_000)
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16, combine=fr.COMBINE_VOTE, out_act=0)
    return mk, ens, fr.fr_server_create(ctx, mk, ens, capacity=capacity, chunk_steps=chunk)


def _until(pred, timeout_s=60.0):
    t0 = time.time()
    while not pred():
        assert time.time() - t0 < timeout_s
        time.sleep(0.001)


def test_cancel_queued_and_running_requests(ctx, dev):
    # a 100,000-step request runs for thousands of chunks, so it is surely
    # still running when it is cancelled; the request queued behind it then
    # runs and is exact
    mk, ens, srv = _crypto_server(ctx)
    long_req = dict(n_envs=64, window=100_000, start=4000, start_stride=7)
    short = dict(n_envs=64, window=300, start=9000, start_stride=11)
    ta = fr.backtest_submit(srv, **long_req)
    _until(lambda: fr.fr_server_stats(srv)["running"] == 1)
    tb = fr.backtest_submit(srv, **short)                        # queued behind the long one
    tc = fr.backtest_submit(srv, **short)
    fr.backtest_cancel(srv, tc)                                  # queued: finishes at once
    rc = fr.backtest_poll(srv, tc)
    assert rc is not None and rc["status"] == _lib.FR_ECANCELED
    fr.backtest_cancel(srv, ta)                                  # running: next chunk boundary
    res = _wait_all(srv, [ta, tb])
    with pytest.raises(fr.FrError) as ei:
        fr.backtest_cancel(srv, 10 ** 9)
    assert ei.value.code == _lib.FR_ENOTFOUND
    st = fr.fr_server_stats(srv)
    srv.close()
    assert res[ta]["status"] == _lib.FR_ECANCELED
    assert res[tb]["status"] == _lib.FR_OK
    assert st["failed"] == 2 and st["completed"] == 1
    assert np.array_equal(res[tb]["metrics"], _standalone(ctx, mk, ens, dev, short, 1, stock=False))


def test_request_timeouts_running_and_queued(ctx, dev):
    mk, ens, srv = _crypto_server(ctx)
    long_req = dict(n_envs=64, window=100_000, start=4000, start_stride=7)
    short = dict(n_envs=64, window=300, start=9000, start_stride=11)
    ta = fr.backtest_submit(srv, **long_req, timeout_s=0.05)     # times out while running
    _until(lambda: fr.fr_server_stats(srv)["running"] == 1)
    tb = fr.backtest_submit(srv, **short, timeout_s=0.01)        # times out while queued
    tc = fr.backtest_submit(srv, **short)                        # no deadline: runs after
    res = _wait_all(srv, [ta, tb, tc])
    with pytest.raises(fr.FrError):
        fr.backtest_submit(srv, **short, timeout_s=-1.0)
    srv.close()
    assert res[ta]["status"] == _lib.FR_ETIMEDOUT
    assert res[tb]["status"] == _lib.FR_ETIMEDOUT
    assert res[tc]["status"] == _lib.FR_OK
    assert np.array_equal(res[tc]["metrics"], _standalone(ctx, mk, ens, dev, short, 1, stock=False))
