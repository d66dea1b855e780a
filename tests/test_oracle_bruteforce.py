"""The oracle's environments against an independently written exact reference
(Python integers and fractions, affordability by linear search) on every
action sequence of tiny cases, plus the MDP invariants (Sec. 3.1) on larger
random runs."""
import itertools
import math
from fractions import Fraction
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
from paper_2501_10709_gb300 import synth


# ------------------------------------------------ independent exact reference

def _price(close, bps):
    return max(1, math.floor(Fraction(close) * Fraction(10000 + bps, 10000) + Fraction(1, 2)))


def _fee(g, fee_bps):
    return math.ceil(Fraction(g * fee_bps, 10000))


def ref_stock_env(close, bps, start, W, init_cash, fee_bps, orders, largest_first=False):
    """One stock env, exact.  close[day][k]; orders: list of per-step share
    orders; buys in ascending asset order, or by decreasing requested count
    (ties ascending) when largest_first.  Returns per step (reward, cash,
    holdings, done)."""
    K = len(close[0])
    cash, h, t, done = init_cash, [0] * K, 0, False
    out = []
    for q in orders:
        if done:
            out.append((0, cash, list(h), 1))
            continue
        d = start + t
        p = [_price(close[d][k], bps[k]) for k in range(K)]
        v0 = cash + sum(a * b for a, b in zip(p, h))
        for k in range(K):
            if q[k] < 0:
                n = min(-q[k], h[k])
                h[k] -= n
                cash += n * p[k] - _fee(n * p[k], fee_bps)
        buy_seq = sorted(range(K), key=lambda k: (-q[k], k)) if largest_first else range(K)
        for k in buy_seq:
            if q[k] > 0:
                n = 0
                while n < q[k] and (n + 1) * p[k] + _fee((n + 1) * p[k], fee_bps) <= cash:
                    n += 1
                h[k] += n
                cash -= n * p[k] + _fee(n * p[k], fee_bps)
        t += 1
        p1 = [_price(close[d + 1][k], bps[k]) for k in range(K)]
        v1 = cash + sum(a * b for a, b in zip(p1, h))
        done = t == W - 1
        out.append((v1 - v0, cash, list(h), int(done)))
    return out


def ref_crypto_env(mid, spread, start, W, init_cash, pmax, acts):
    cash, pos, t, done = init_cash, 0, 0, False
    out = []
    for u in acts:
        if done:
            out.append((0, cash, pos, 1))
            continue
        d = start + t
        v0 = cash + pos * mid[d]
        bid = mid[d] - spread[d] // 2
        ask = bid + spread[d]
        if u == 2 and pos < pmax and cash >= ask:
            pos, cash = pos + 1, cash - ask
        elif u == 0 and pos > 0:
            pos, cash = pos - 1, cash + bid
        t += 1
        v1 = cash + pos * mid[d + 1]
        done = t == W - 1
        out.append((v1 - v0, cash, pos, int(done)))
    return out


# --------------------------------------------------------------- brute force

@pytest.mark.parametrize("buy_order", [0, 1])
@pytest.mark.parametrize("W,fee_bps,init_cash", [(4, 250, 1500), (3, 10, 2100), (4, 0, 999)])
def test_stock_all_action_sequences_tiny(W, fee_bps, init_cash, buy_order):
    close = np.array([[310, 655], [290, 700], [333, 640], [301, 689]], np.int64)
    ind = np.zeros((4, 1, 2), np.float32)
    mk = SimpleNamespace(close=close, ind=ind)
    vals = range(-2, 3)
    per_step = list(itertools.product(vals, repeat=2))
    seqs = list(itertools.product(per_step, repeat=3))
    N, T = len(seqs), 3
    acts = np.array(seqs, np.int32).transpose(1, 0, 2).copy()   # [T][N][K]
    bps_row = [37, -64]
    o = oracle.stock_run(mk, np.full(N, 2), np.zeros(N), np.full(N, W),
                         np.tile(np.array(bps_row, np.int16), (N, 1)),
                         init_cash=init_cash, hmax=2, fee_bps=fee_bps, T=T,
                         act_i32=acts, buy_order=buy_order)
    for e, seq in enumerate(seqs):
        ref = ref_stock_env(close.tolist(), bps_row, 0, W, init_cash, fee_bps, seq,
                            largest_first=buy_order == 1)
        for t, (r, c, h, dn) in enumerate(ref):
            assert o["rew"][t, e] == r, (seq, t)
            assert o["cash"][t, e] == c, (seq, t)
            assert o["hold"][t, e].tolist() == h, (seq, t)
            assert o["done"][t, e] == dn, (seq, t)


def test_stock_largest_first_three_assets_all_sequences():
    """Largest-first buys with ties: three assets, orders -1..2 each, two
    steps, cash for only part of the orders."""
    close = np.array([[400, 390, 410], [405, 385, 420], [398, 400, 401]], np.int64)
    ind = np.zeros((3, 1, 3), np.float32)
    mk = SimpleNamespace(close=close, ind=ind)
    per_step = list(itertools.product(range(-1, 3), repeat=3))
    seqs = list(itertools.product(per_step, repeat=2))
    N, T, W, cash0, fee = len(seqs), 2, 3, 1700, 30
    acts = np.array(seqs, np.int32).transpose(1, 0, 2).copy()
    bps_row = [0, 55, -100]
    o = oracle.stock_run(mk, np.full(N, 3), np.zeros(N), np.full(N, W),
                         np.tile(np.array(bps_row, np.int16), (N, 1)),
                         init_cash=cash0, hmax=2, fee_bps=fee, T=T, act_i32=acts,
                         buy_order=1, want=("rew", "cash", "hold", "done"))
    differs = 0
    for e, seq in enumerate(seqs):
        ref = ref_stock_env(close.tolist(), bps_row, 0, W, cash0, fee, seq, largest_first=True)
        asc = ref_stock_env(close.tolist(), bps_row, 0, W, cash0, fee, seq)
        differs += ref != asc
        for t, (r, c, h, dn) in enumerate(ref):
            assert (o["rew"][t, e], o["cash"][t, e], o["hold"][t, e].tolist(), o["done"][t, e]) == (r, c, h, dn), (seq, t)
    assert differs > 100            # the case exercises the order


def test_stock_buy_order_rejects_unknown():
    close = np.array([[400], [405]], np.int64)
    mk = SimpleNamespace(close=close, ind=np.zeros((2, 1, 1), np.float32))
    with pytest.raises(ValueError):
        oracle.stock_run(mk, [1], [0], [2], np.zeros((1, 1), np.int16), init_cash=1000, hmax=1,
                         fee_bps=0, T=1, act_i32=np.ones((1, 1, 1), np.int32), buy_order=2)


def test_crypto_all_action_sequences_tiny():
    mid = np.array([6_000_000, 6_000_300, 5_999_100, 6_001_000, 6_000_050,
                    6_002_000, 6_001_500, 6_000_000], np.int64)
    spread = np.array([1, 5, 2, 3, 4, 1, 2, 5], np.uint8)
    fac = np.zeros((8, 8), np.float32)
    mk = SimpleNamespace(mid=mid, spread=spread, fac=fac)
    seqs = list(itertools.product(range(3), repeat=6))
    N, T, W, cash0, pmax = len(seqs), 6, 6, 12_000_010, 2
    acts = np.array(seqs, np.uint8).T.copy()
    o = oracle.crypto_run(mk, np.zeros(N), np.full(N, W), init_cash=cash0,
                          pmax=pmax, T=T, act_u8=acts)
    for e, seq in enumerate(seqs):
        ref = ref_crypto_env(mid.tolist(), spread.tolist(), 0, W, cash0, pmax, seq)
        for t, (r, c, pos, dn) in enumerate(ref):
            assert (o["rew"][t, e], o["cash"][t, e], o["pos"][t, e], o["done"][t, e]) == (r, c, pos, dn)


# -------------------------------------------------------------- invariants

def _stock_setup(N=24, T=40, seed=3):
    mk = synth.stock_market(120, 30, seed)
    envs = synth.stock_envs_uneven(N, 30, 120, k_lo=1, w_lo=2, w_hi=45, seed=seed)
    q = synth.prescribed_shares(T, N, 30, 100, seed)
    if T > 5:
        q[5] = 0                                # one all-zero step for everyone
    return mk, envs, q, T


def test_stock_mdp_invariants():
    mk, envs, q, T = _stock_setup()
    o = oracle.stock_run(mk, envs.Ke, envs.start, envs.W, envs.bps,
                         init_cash=envs.init_cash, hmax=100, fee_bps=10, T=T,
                         act_i32=q)
    K = 30
    for e in range(envs.N):
        ke, s, W = int(envs.Ke[e]), int(envs.start[e]), int(envs.W[e])
        b = envs.bps[e]

        def prices(d):
            return oracle.perturb_many(mk.close[d, :ke], b[:ke].astype(np.int32))

        cash, h = envs.init_cash, np.zeros(ke, np.int64)
        v = cash
        for t in range(T):
            nc, nh = int(o["cash"][t, e]), o["hold"][t, e, :ke].astype(np.int64)
            assert nc >= 0 and (nh >= 0).all()                # no debt, no shorts
            assert (o["hold"][t, e, ke:] == 0).all()
            if t >= W - 1:                                   # frozen after window
                assert o["done"][t, e] == 1 and o["rew"][t, e] == 0
                assert nc == cash and (nh == h).all()
                continue
            d = s + t
            p0, p1 = prices(d), prices(d + 1)
            qq = q[t, e, :ke].astype(np.int64)
            dh = nh - h
            assert (dh <= np.maximum(qq, 0)).all()            # never buy beyond the order
            assert (-dh <= np.minimum(np.maximum(-qq, 0), h)).all()   # sells capped at holdings
            assert ((dh == 0) | (np.sign(dh) == np.sign(qq))).all()
            v_after = nc + int((p0 * nh).sum())               # same prices, after trading
            assert v - v_after >= 0                           # fees are never negative
            fees = v - v_after
            gross = int((np.abs(dh) * p0).sum())
            assert fees <= math.ceil(gross * 10 / 10000) + ke
            v1 = nc + int((p1 * nh).sum())
            assert v == cash + int((p0 * h).sum())            # v_t = b_t + p_t^T h_t
            assert o["rew"][t, e] == v1 - v                  # reward = v_{t+1} - v_t
            if not qq.any():
                assert o["rew"][t, e] == int((h * (p1 - p0)).sum())  # price moves only
            cash, h, v = nc, nh, v1
            assert o["done"][t, e] == int(t == W - 2)


def test_stock_observation_layout():
    mk, envs, q, T = _stock_setup(N=4, T=3)
    o = oracle.stock_run(mk, envs.Ke, envs.start, envs.W, envs.bps,
                         init_cash=envs.init_cash, hmax=100, fee_bps=10, T=T,
                         act_i32=q)
    K, I = 30, 8
    for e in range(4):
        ke, d = int(envs.Ke[e]), int(envs.start[e])
        ob = o["obs"][0, e]
        assert ob.shape == (1 + 2 * K + I * K,)
        assert ob[0] == np.float32(1.0)                      # 1e8 cents * 1e-8
        p = oracle.perturb_many(mk.close[d, :ke], envs.bps[e, :ke].astype(np.int32))
        assert np.array_equal(ob[1:1 + ke], p.astype(np.float32) * np.float32(1e-4))
        assert (ob[1 + ke:1 + K] == 0).all() and (ob[1 + K:1 + 2 * K] == 0).all()
        f = ob[1 + 2 * K:].reshape(I, K)                     # indicator-major
        assert np.array_equal(f[:, :ke], oracle.market_table(mk)[d, :, :ke]) and (f[:, ke:] == 0).all()


def test_stock_metrics_follow_value_series():
    mk, envs, q, T = _stock_setup(N=6, T=40)
    o = oracle.stock_run(mk, envs.Ke, envs.start, envs.W, envs.bps,
                         init_cash=envs.init_cash, hmax=100, fee_bps=10, T=T,
                         act_i32=q)
    for e in range(6):
        steps = min(T, int(envs.W[e]) - 1)
        v = np.concatenate([[envs.init_cash], envs.init_cash + np.cumsum(o["rew"][:steps, e])])
        want = oracle.metrics_series(v, 252.0)
        assert np.array_equal(o["metrics"][e], want)


def test_unit_actions_equal_their_discretised_shares():
    mk, envs, _, T = _stock_setup(N=10, T=20)
    a = synth.prescribed_unit(T, 10, 30, 4)
    a[3, 2, 5] = np.nan
    a[4, 1, 0] = np.inf
    o1 = oracle.stock_run(mk, envs.Ke, envs.start, envs.W, envs.bps,
                          init_cash=envs.init_cash, hmax=100, fee_bps=10, T=T, act_f32=a)
    q = oracle.discretise_many(a, 100).reshape(a.shape)
    o0 = oracle.stock_run(mk, envs.Ke, envs.start, envs.W, envs.bps,
                          init_cash=envs.init_cash, hmax=100, fee_bps=10, T=T, act_i32=q)
    for k in ("rew", "cash", "hold", "done", "obs"):
        assert np.array_equal(o0[k], o1[k]), k


def test_auto_reset_restarts_the_episode():
    mk, envs, q, _ = _stock_setup(N=3, T=12)
    W = np.full(3, 5, np.int32)
    o = oracle.stock_run(mk, envs.Ke, envs.start, W, envs.bps, init_cash=envs.init_cash,
                         hmax=100, fee_bps=10, T=12, act_i32=q[:12], auto_reset=True)
    for t in range(12):
        assert o["done"][t].tolist() == [int(t % 4 == 3)] * 3
        if t % 4 == 3:
            assert (o["cash"][t] == envs.init_cash).all() and (o["hold"][t] == 0).all()
    assert np.array_equal(o["obs"][4], o["obs"][0])


def test_identical_agents_ensemble_rollout_equals_single_agent():
    w = synth.workload_stock_small()
    one = w.params[:1]
    three = np.repeat(one, 3, axis=0)
    args = (w.market, w.envs.Ke, w.envs.start, w.envs.W, w.envs.bps)
    kw = dict(init_cash=w.envs.init_cash, hmax=100, fee_bps=10, T=w.T)
    o1 = oracle.stock_run(*args, ensemble=(w.dims, one, None), **kw)
    o3 = oracle.stock_run(*args, ensemble=(w.dims, three, None), **kw)
    for k in ("rew", "cash", "hold", "act", "metrics"):
        assert np.array_equal(o1[k], o3[k]), k


def test_crypto_invariants_and_vote_rollout():
    w = synth.workload_crypto(N=64, T=200, S=20_000)
    o = oracle.crypto_run(w.market, w.envs.start, w.envs.W, init_cash=w.envs.init_cash,
                          pmax=w.envs.pmax, T=w.T, ensemble=(w.dims, w.params))
    assert ((o["pos"] >= 0) & (o["pos"] <= w.envs.pmax)).all()
    assert (o["cash"] >= 0).all()
    for t in range(0, w.T, 37):
        for e in range(0, 64, 7):
            assert o["act"][t, e] == oracle.vote(o["agent_act"][t, e])
    # the actions are not degenerate for this weight recipe
    assert len(np.unique(o["act"])) >= 2
