"""Error paths under host-side fault injection (fr_fault_inject): a failed
device allocation, a rejected submit and dropped polls each surface as their
error code and leave the other requests intact.  Nothing here faults or traps
the GPU: those failures are made on the host.  The one device-side case is
the bounded-wait check, whose waits give up by design after 50 ms."""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_2501_10709_gb300 as fr
from paper_2501_10709_gb300 import _lib, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _disarm():
    yield
    for k in (fr.FAULT_ALLOC, fr.FAULT_SUBMIT, fr.FAULT_POLL):
        fr.fr_fault_inject(k, 0, 0)


def _standalone(ctx, mk, ens, dev, req, K=30):
    n = req["n_envs"]
    start = req["start"] + np.arange(n) * req.get("start_stride", 0)
    bps = np.zeros((n, K), np.int16)
    for i in range(n):
        for k in range(K):
            bps[i, k] = oracle.perturb_bps(req.get("seed", 0), i, k, req.get("bps_range", 0)) \
                if req.get("bps_range", 0) else 0
    env = fr.env_create(ctx, mk, start=start, window=req["window"], bps=bps)
    met = torch.empty(n, 3, dtype=torch.float64, device=dev)
    fr.rollout(env, ens, req["window"] - 1, metrics=met)
    torch.cuda.synchronize()
    return met.cpu().numpy()


def _wait(srv, tickets, timeout_s=120.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = fr.backtest_poll(srv, t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout_s
        time.sleep(0.002)
    return out


def test_allocation_failure_returns_enomem_without_leaks(ctx, dev):
    w = synth.workload_stock_small()
    e = w.envs
    used0 = ctx.bytes_in_use
    fr.fr_fault_inject(fr.FAULT_ALLOC, skip=1, count=1)        # the market's second table fails
    with pytest.raises(fr.FrError) as ei:
        fr.fr_market_create(ctx, w.market)
    assert ei.value.code == _lib.FR_ENOMEM and ctx.bytes_in_use == used0
    mk = fr.fr_market_create(ctx, w.market)
    fr.fr_fault_inject(fr.FAULT_ALLOC, skip=0, count=1)
    with pytest.raises(fr.FrError) as ei:
        fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps)
    assert ei.value.code == _lib.FR_ENOMEM
    # the next call succeeds and the env is exact
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps)
    acts = synth.prescribed_shares(6, e.N, 30, seed=4)
    rew = torch.empty(6, e.N, dtype=torch.int64, device=dev)
    a = torch.from_numpy(acts).to(dev)
    for t in range(6):
        fr.env_step(env, a[t], fr.ACT_I32_SHARES, rew=rew[t])
    torch.cuda.synchronize()
    ref = oracle.stock_run(w.market, e.Ke, e.start, e.W, e.bps, init_cash=e.init_cash, hmax=100,
                           fee_bps=10, T=6, act_i32=acts, want=("rew",))
    assert np.array_equal(rew.cpu().numpy(), ref["rew"])


def test_server_chunk_failure_fails_only_the_running_requests(ctx, dev):
    w = synth.workload_stock_2048(N=128, T=16)
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    srv = fr.fr_server_create(ctx, mk, ens, capacity=64, chunk_steps=8)
    a = dict(n_envs=64, window=20, start=100, start_stride=1, bps_range=100, seed=1)
    b = dict(n_envs=64, window=30, start=300, start_stride=2, bps_range=100, seed=2)
    # the pool's first rollout needs device memory (kernel images, scratch):
    # that allocation fails once
    fr.fr_fault_inject(fr.FAULT_ALLOC, skip=0, count=1)
    ta = fr.backtest_submit(srv, **a)
    tb = fr.backtest_submit(srv, **b)                          # 64 + 64 > 64: queued behind a
    res = _wait(srv, [ta, tb])
    st = fr.fr_server_stats(srv)
    srv.close()
    assert res[ta]["status"] == _lib.FR_ENOMEM
    assert res[tb]["status"] == _lib.FR_OK
    assert st["failed"] == 1 and st["completed"] == 1
    assert np.array_equal(res[tb]["metrics"], _standalone(ctx, mk, ens, dev, b))


def test_rejected_and_malformed_submits_leave_the_others_intact(ctx, dev):
    w = synth.workload_stock_2048(N=128, T=16)
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    srv = fr.fr_server_create(ctx, mk, ens, capacity=96, chunk_steps=8)
    reqs = [dict(n_envs=30, window=12, start=100, start_stride=3, bps_range=100, seed=7),
            dict(n_envs=50, window=25, start=400, start_stride=1, bps_range=100, seed=8),
            dict(n_envs=20, window=9, start=700, start_stride=0, bps_range=40, seed=9)]
    fr.fr_fault_inject(fr.FAULT_SUBMIT, skip=1, count=1)
    t0 = fr.backtest_submit(srv, **reqs[0])
    with pytest.raises(fr.FrError) as ei:                      # rejected
        fr.backtest_submit(srv, **reqs[1])
    assert ei.value.code == _lib.FR_EBUSY
    with pytest.raises(fr.FrError) as ei:                      # malformed windows
        fr.backtest_submit(srv, n_envs=4, window=1, start=100)
    assert ei.value.code == _lib.FR_EINVAL
    with pytest.raises(fr.FrError) as ei:
        fr.backtest_submit(srv, n_envs=4, window=50, start=980)
    assert ei.value.code == _lib.FR_EINVAL
    t1 = fr.backtest_submit(srv, **reqs[1])                    # resubmitted
    t2 = fr.backtest_submit(srv, **reqs[2])
    res = _wait(srv, [t0, t1, t2])
    st = fr.fr_server_stats(srv)
    srv.close()
    assert st["submitted"] == 3 and st["completed"] == 3 and st["failed"] == 0
    for t, r in zip((t0, t1, t2), reqs):
        assert res[t]["status"] == _lib.FR_OK
        assert np.array_equal(res[t]["metrics"], _standalone(ctx, mk, ens, dev, r)), r


def test_dropped_polls_keep_the_result(ctx, dev):
    w = synth.workload_stock_2048(N=128, T=16)
    mk = fr.fr_market_create(ctx, w.market)
    ens = fr.ensemble_create(ctx, w.dims, w.params, precision=fr.PREC_BF16)
    srv = fr.fr_server_create(ctx, mk, ens, capacity=32, chunk_steps=8)
    r = dict(n_envs=32, window=17, start=250, start_stride=4, bps_range=100, seed=3)
    t = fr.backtest_submit(srv, **r)
    t0 = time.time()
    while fr.fr_server_stats(srv)["completed"] < 1:
        assert time.time() - t0 < 120
        time.sleep(0.002)
    fr.fr_fault_inject(fr.FAULT_POLL, skip=0, count=2)
    assert fr.backtest_poll(srv, t) is None                    # dropped
    assert fr.backtest_poll(srv, t) is None                    # dropped
    got = fr.backtest_poll(srv, t)
    srv.close()
    assert got is not None and got["status"] == _lib.FR_OK
    assert np.array_equal(got["metrics"], _standalone(ctx, mk, ens, dev, r))


def test_bounded_waits_give_up_and_the_context_stays_usable(ctx, dev):
    # both wait forms of the fused kernels, on barriers nothing completes,
    # limited to 50 ms: each gives up, sets its error bit and returns
    r = fr.fr_wait_selftest(ctx, limit_us=50_000)
    assert r["status"] == _lib.FR_ETIMEDOUT
    assert r["flags"] == 3                                     # bit 2: the completed control wait
    for ns in r["waited_ns"]:
        assert 50e6 <= ns < 1e9
    with pytest.raises(fr.FrError):
        fr.fr_wait_selftest(ctx, limit_us=0)
    # the context still runs work exactly
    w = synth.workload_stock_small()
    e = w.envs
    mk = fr.fr_market_create(ctx, w.market)
    env = fr.env_create(ctx, mk, start=e.start, window=e.W, n_assets=e.Ke, bps=e.bps)
    acts = synth.prescribed_shares(4, e.N, 30, seed=9)
    rew = torch.empty(4, e.N, dtype=torch.int64, device=dev)
    a = torch.from_numpy(acts).to(dev)
    for t in range(4):
        fr.env_step(env, a[t], fr.ACT_I32_SHARES, rew=rew[t])
    torch.cuda.synchronize()
    ref = oracle.stock_run(w.market, e.Ke, e.start, e.W, e.bps, init_cash=e.init_cash, hmax=100,
                           fee_bps=10, T=4, act_i32=acts, want=("rew",))
    assert np.array_equal(rew.cpu().numpy(), ref["rew"])
