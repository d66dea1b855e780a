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
    r = _lib.Request(2, 10, 100, 0, 0, 0, 0, 2, met.ctypes.data_as(C.c_void_p))   # want_traj not 0 / 1
    t = C.c_uint64()
    assert fr.lib().backtest_submit(srv, C.byref(r), C.byref(t)) == _lib.FR_EINVAL
    with pytest.raises(fr.FrError):                                    # no crypto pool
        fr.backtest_submit(srv, n_envs=2, window=10, start=100, task=fr.TASK_CRYPTO)
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
    assert st["canceled"] == 2 and st["failed"] == 0 and st["completed"] == 1
    assert np.array_equal(res[tb]["metrics"], _standalone(ctx, mk, ens, dev, short, 1, stock=False))


def test_request_timeouts_running_and_queued(ctx, dev):
    mk, ens, srv = _crypto_server(ctx)
    long_req = dict(n_envs=64, window=100_000, start=4000, start_stride=7)
    short = dict(n_envs=64, window=300, start=9000, start_stride=11)
    # the long request holds every slot for 0.5 s (its 100,000 steps take far
    # longer), so the request behind it is still queued when its own 10 ms
    # deadline passes, whatever the delay of this thread in between
    ta = fr.backtest_submit(srv, **long_req, timeout_s=0.5)      # times out while running
    _until(lambda: fr.fr_server_stats(srv)["running"] == 1)
    tb = fr.backtest_submit(srv, **short, timeout_s=0.01)        # times out while queued
    tc = fr.backtest_submit(srv, **short)                        # no deadline: runs after
    res = _wait_all(srv, [ta, tb, tc])
    with pytest.raises(fr.FrError):
        fr.backtest_submit(srv, **short, timeout_s=-1.0)
    st = fr.fr_server_stats(srv)
    srv.close()
    assert res[ta]["status"] == _lib.FR_ETIMEDOUT
    assert res[tb]["status"] == _lib.FR_ETIMEDOUT
    assert res[tb]["latency_s"] < res[ta]["latency_s"]          # tb left the queue first
    assert res[tc]["status"] == _lib.FR_OK
    assert st["timed_out"] == 2 and st["failed"] == 0
    assert np.array_equal(res[tc]["metrics"], _standalone(ctx, mk, ens, dev, short, 1, stock=False))


# ------------------------------------------------ pools, trajectories, budget
def _standalone_traj(ctx, mk, ens, dev, req, K, stock=True):
    """A standalone rollout of the request's envs with its trajectory."""
    n, T = req["n_envs"], req["window"] - 1
    start = req["start"] + np.arange(n) * req.get("start_stride", 0)
    if stock:
        ke = req.get("n_assets", 0) or K
        env = fr.env_create(ctx, mk, start=start, window=req["window"], n_assets=ke,
                            bps=_request_bps(n, K, req.get("seed", 0), req.get("bps_range", 0)))
    else:
        env = fr.env_create(ctx, mk, start=start, window=req["window"])
    tr = {"obs": torch.empty(T, n, env.D, device=dev),
          "act": torch.empty(T, n, K, device=dev) if stock else torch.empty(T, n, dtype=torch.uint8, device=dev),
          "rew": torch.empty(T, n, dtype=torch.int64, device=dev),
          "done": torch.empty(T, n, dtype=torch.uint8, device=dev)}
    met = torch.empty(n, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, T, traj=tr, metrics=met)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in tr.items()}, met.cpu().numpy(), env.D


def _stock_pair(ctx, precision=fr.PREC_BF16):
    w = synth.workload_stock_2048(N=128, T=16)
    return w, fr.fr_market_create(ctx, w.market), fr.ensemble_create(ctx, w.dims, w.params, precision=precision)


def _crypto_pair(ctx, precision=fr.PREC_FP16):
    w = synth.workload_crypto(N=64, T=64, S=60_000)
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=precision, combine=fr.COMBINE_VOTE, out_act=0)
    return w, mk, ens


CRYPTO_REQS = [dict(n_envs=64, window=100, start=4000, start_stride=37),
               dict(n_envs=100, window=300, start=9000, start_stride=11),
               dict(n_envs=50, window=41, start=20000, start_stride=101)]


def test_stock_and_crypto_pools_in_one_server(ctx, dev):
    # one server, a stock pool (BF16 fused) and a crypto pool (FP16 fused),
    # each on its own stream; requests of both tasks interleaved, more than
    # the pools hold at once: every result equals its standalone rollout
    ws, mks, enss = _stock_pair(ctx)
    wc, mkc, ensc = _crypto_pair(ctx)
    srv = fr.fr_server_create(ctx, mks, enss, capacity=256, chunk_steps=16)
    fr.fr_server_add_pool(srv, mkc, ensc, capacity=128, chunk_steps=32)
    with pytest.raises(fr.FrError):                                  # one pool per ensemble
        fr.fr_server_add_pool(srv, mkc, ensc, capacity=8)
    tickets = []
    for i in range(max(len(STOCK_REQS), len(CRYPTO_REQS))):
        if i < len(STOCK_REQS):
            tickets.append(("s", STOCK_REQS[i], fr.backtest_submit(srv, **STOCK_REQS[i], task=fr.TASK_STOCK)))
        if i < len(CRYPTO_REQS):
            tickets.append(("c", CRYPTO_REQS[i], fr.backtest_submit(srv, **CRYPTO_REQS[i], ens=ensc,
                                                                     task=fr.TASK_CRYPTO)))
    res = _wait_all(srv, [t for _, _, t in tickets])
    st = fr.fr_server_stats(srv)
    srv.close()
    assert st["pools"] == 2 and st["completed"] == len(tickets) and st["bytes_reserved"] == 0
    for kind, r, t in tickets:
        assert res[t]["status"] == 0 and res[t]["task"] == (fr.TASK_STOCK if kind == "s" else fr.TASK_CRYPTO)
        want = (_standalone(ctx, mks, enss, dev, r, 30) if kind == "s"
                else _standalone(ctx, mkc, ensc, dev, r, 1, stock=False))
        assert np.array_equal(res[t]["metrics"], want), (kind, r)


def test_trajectory_requests_equal_standalone_and_oracle(ctx, dev):
    # recording and metrics-only requests of both tasks share the pools; a
    # recorded trajectory equals a standalone rollout's bit for bit, and the
    # oracle replaying its actions reproduces its rewards, done flags and the
    # request's FP64 metrics (oracle parity of served results, directly)
    ws, mks, enss = _stock_pair(ctx)
    wc, mkc, ensc = _crypto_pair(ctx)
    srv = fr.fr_server_create(ctx, mks, enss, capacity=192, chunk_steps=16)
    fr.fr_server_add_pool(srv, mkc, ensc, capacity=128, chunk_steps=32)
    sreqs = [dict(STOCK_REQS[0], want_traj=True), STOCK_REQS[1], dict(STOCK_REQS[3], want_traj=True)]
    creqs = [dict(CRYPTO_REQS[0], want_traj=True), CRYPTO_REQS[2]]
    ts = [fr.backtest_submit(srv, **r) for r in sreqs]
    tc = [fr.backtest_submit(srv, **r, task=fr.TASK_CRYPTO) for r in creqs]
    res = _wait_all(srv, ts + tc)
    got = {}
    for t, r, D, K in [(t, r, 301, 30) for t, r in zip(ts, sreqs)] + \
                      [(t, r, 10, 1) for t, r in zip(tc, creqs)]:
        if r.get("want_traj"):
            assert res[t]["traj_steps"] == r["window"] - 1 and res[t]["traj_bytes"] > 0
            got[t] = {k: v.cpu().numpy() for k, v in fr.backtest_fetch_traj(srv, t, D=D, K=K).items()}
        else:
            assert res[t]["traj_steps"] == 0
    st = fr.fr_server_stats(srv)
    srv.close()
    assert st["bytes_reserved"] == 0 and st["bytes_peak"] > 0
    for t, r in zip(ts, sreqs):
        want_tr, want_met, _ = _standalone_traj(ctx, mks, enss, dev, r, 30)
        assert np.array_equal(res[t]["metrics"], want_met), r
        if not r.get("want_traj"):
            continue
        g = got[t]
        for k in ("obs", "act", "rew", "done"):
            assert np.array_equal(g[k], want_tr[k]), (k, r)
        n = r["n_envs"]
        start = r["start"] + np.arange(n) * r.get("start_stride", 0)
        ke = np.full(n, r.get("n_assets", 0) or 30, np.int32)
        ref = oracle.stock_run(ws.market, ke, start, np.full(n, r["window"], np.int32),
                               _request_bps(n, 30, r.get("seed", 0), r.get("bps_range", 0)),
                               init_cash=100_000_000, hmax=100, fee_bps=10, T=r["window"] - 1,
                               act_f32=g["act"], want=("obs", "rew", "done", "metrics"))
        assert np.array_equal(g["obs"], ref["obs"]) and np.array_equal(g["rew"], ref["rew"])
        assert np.array_equal(g["done"], ref["done"]) and np.array_equal(res[t]["metrics"], ref["metrics"])
    for t, r in zip(tc, creqs):
        want_tr, want_met, _ = _standalone_traj(ctx, mkc, ensc, dev, r, 1, stock=False)
        assert np.array_equal(res[t]["metrics"], want_met), r
        if not r.get("want_traj"):
            continue
        g = got[t]
        for k in ("obs", "act", "rew", "done"):
            assert np.array_equal(g[k], want_tr[k]), (k, r)
        n = r["n_envs"]
        start = r["start"] + np.arange(n) * r.get("start_stride", 0)
        ref = oracle.crypto_run(wc.market, start, np.full(n, r["window"], np.int32), init_cash=100_000_000, pmax=10,
                                T=r["window"] - 1, act_u8=g["act"], want=("obs", "rew", "done", "metrics"))
        assert np.array_equal(g["obs"], ref["obs"]) and np.array_equal(g["rew"], ref["rew"])
        assert np.array_equal(g["done"], ref["done"]) and np.array_equal(res[t]["metrics"], ref["metrics"])


def test_admission_by_hbm_budget(ctx, dev):
    # Two recording requests, each within the budget alone but not together:
    # the second waits in the queue, beyond the first's completion, until the
    # first's trajectory is released; one above the budget is refused at
    # submit.  Metrics-only requests of the other pool are not held up.
    ws, mks, enss = _stock_pair(ctx)
    wc, mkc, ensc = _crypto_pair(ctx, fr.PREC_BF16)
    row = 4 * 301 + 4 * 30 + 9                                      # trajectory bytes per stock env-step
    a = dict(n_envs=64, window=40, start=100, bps_range=100, seed=21, want_traj=True)
    need = 64 * 39 * row                                            # + the slots' state bytes
    srv = fr.fr_server_create(ctx, mks, enss, capacity=256, chunk_steps=8, hbm_budget=int(need * 1.5))
    fr.fr_server_add_pool(srv, mkc, ensc, capacity=64, chunk_steps=32)
    with pytest.raises(fr.FrError) as ei:                           # can never fit the budget
        fr.backtest_submit(srv, **dict(a, window=80))
    assert ei.value.code == _lib.FR_ENOMEM
    ta = fr.backtest_submit(srv, **a)
    tb = fr.backtest_submit(srv, **dict(a, start=200, seed=22))
    tc = fr.backtest_submit(srv, **CRYPTO_REQS[2], task=fr.TASK_CRYPTO)   # other pool, metrics only
    ra = _wait_all(srv, [ta, tc])
    assert ra[ta]["status"] == 0 and ra[tc]["status"] == 0
    time.sleep(0.05)                                                # several chunk boundaries
    st = fr.fr_server_stats(srv)
    assert fr.backtest_poll(srv, tb) is None and st["queued"] == 1   # held by the budget, not by slots
    assert st["bytes_reserved"] > need and st["bytes_reserved"] <= st["budget"]
    ga = {k: v.cpu().numpy() for k, v in fr.backtest_fetch_traj(srv, ta, D=301, K=30).items()}
    rb = _wait_all(srv, [tb])[tb]
    assert rb["status"] == 0 and rb["queue_s"] >= ra[ta]["latency_s"] - 0.01
    fr.backtest_release(srv, tb)
    st = fr.fr_server_stats(srv)
    srv.close()
    assert st["bytes_reserved"] == 0 and st["bytes_peak"] <= st["budget"]
    want_tr, want_met, _ = _standalone_traj(ctx, mks, enss, dev, a, 30)
    assert np.array_equal(ra[ta]["metrics"], want_met)
    for k in ("obs", "act", "rew", "done"):
        assert np.array_equal(ga[k], want_tr[k]), k
