"""Pins for the CPU oracle: each test checks it against something other than
itself -- exact rational arithmetic, linear search, torch float64, the
Condorcet binomial sum (Sec. 3.3.1), hand-computed metric series.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2501_10709_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------- prices/fees

def test_perturb_matches_exact_rational_rounding():
    # Sec. 5.1: a -1%..+1% change applied to each asset's price; read as an
    # integer basis-point change rounded half up to the cent, floor 1 cent.
    st = synth.Stream(7, 900)
    close = np.concatenate([np.arange(1, 400), st.integers(1, 10**7, 4000)])
    for bps in (-100, -99, -51, -50, -1, 0, 1, 37, 50, 99, 100):
        got = oracle.perturb_many(close, np.full(close.shape, bps))
        for c, g in zip(close.tolist(), got.tolist()):
            x = Fraction(c) * Fraction(10000 + bps, 10000)
            want = max(1, math.floor(x + Fraction(1, 2)))
            assert g == want, (c, bps, g, want)


def test_fee_is_ceiling_of_exact_rational():
    for g in list(range(0, 3000)) + [10**9 + 7, 123456789012]:
        for f in (0, 1, 10, 25, 250):
            assert oracle.fee(g, f) == math.ceil(Fraction(g * f, 10000))


def _cost_exact(n, p, f):
    g = n * p
    return g + math.ceil(Fraction(g * f, 10000))


def test_buy_max_equals_linear_search():
    # the affordable share count must be the largest n whose cost (price plus
    # rounded-up fee) fits in the cash, found here by plain search
    st = synth.Stream(11, 901)
    cases = []
    for p in (1, 2, 3, 7, 99, 100, 101, 2500, 39999):
        for f in (0, 1, 10, 250):
            cash = np.concatenate([np.arange(0, 60), st.integers(0, 300 * p, 40)])
            for c in cash.tolist():
                cases.append((c, p, f))
    cash = np.array([c for c, _, _ in cases])
    pp = np.array([p for _, p, _ in cases])
    ff = np.array([f for _, _, f in cases])
    got = oracle.buy_max_many(cash, pp, ff)
    for (c, p, f), g in zip(cases, got.tolist()):
        n = 0
        while _cost_exact(n + 1, p, f) <= c:
            n += 1
        assert g == n, (c, p, f, g, n)


def test_buy_order_hand_example():
    # two buy orders at 1,000 cents a share, no fee, cash for three shares:
    # ascending order fills asset 0 (1 share) then 2 of asset 1's 4; largest
    # first fills asset 1 (3 of 4) and leaves asset 0 without cash
    from types import SimpleNamespace
    mk = SimpleNamespace(close=np.array([[1000, 1000], [1000, 1000]], np.int64),
                         ind=np.zeros((2, 1, 2), np.float32))
    q = np.array([[[1, 4]]], np.int32)
    runs = [oracle.stock_run(mk, [2], [0], [2], np.zeros((1, 2), np.int16), init_cash=3000, hmax=4,
                             fee_bps=0, T=1, act_i32=q, buy_order=b) for b in (0, 1)]
    assert runs[0]["hold"][0, 0].tolist() == [1, 2] and runs[0]["cash"][0, 0] == 0
    assert runs[1]["hold"][0, 0].tolist() == [0, 3] and runs[1]["cash"][0, 0] == 0
    # equal counts keep the ascending asset order: cash for 2 of 2 x 2 orders
    q = np.array([[[2, 2]]], np.int32)
    r = oracle.stock_run(mk, [2], [0], [2], np.zeros((1, 2), np.int16), init_cash=2000, hmax=4,
                         fee_bps=0, T=1, act_i32=q, buy_order=1)
    assert r["hold"][0, 0].tolist() == [2, 0]


def test_buy_order_is_irrelevant_when_every_order_fits():
    # rich envs (cash far above any day's orders): both orders give the same run
    mk = synth.stock_market(120, 30, 5)
    envs = synth.stock_envs_uneven(64, 30, 120, k_lo=1, w_lo=2, w_hi=45, seed=5)
    q = synth.prescribed_shares(30, 64, 30, 100, 5)
    runs = [oracle.stock_run(mk, envs.Ke, envs.start, envs.W, envs.bps, init_cash=10 ** 12, hmax=100,
                             fee_bps=10, T=30, act_i32=q, buy_order=b) for b in (0, 1)]
    for k in ("rew", "cash", "hold", "done", "metrics"):
        assert np.array_equal(runs[0][k], runs[1][k]), k


# -------------------------------------------------------------- discretise

def _trunc_exact(x: np.ndarray, hmax: int) -> np.ndarray:
    """trunc(x * hmax) computed exactly from the float's integer mantissa and
    exponent (x = m * 2^e), with no floating-point rounding at all."""
    x64 = x.astype(np.float64)
    mant, ex = np.frexp(x64)                    # x = mant * 2^ex, 0.5 <= |mant| < 1
    m = np.rint(mant * 2.0 ** 24).astype(np.int64)   # exact: float32 has 24 bits
    e = ex.astype(np.int64) - 24
    y = np.abs(m) * hmax
    sh = -e
    out = np.where(sh >= 0, y >> np.clip(sh, 0, 63), y << np.clip(-sh, 0, 63))
    out = np.where(sh > 62, 0, out)
    return (np.sign(m) * out).astype(np.int64)


def test_discretise_exhaustive_near_every_share_boundary():
    # every float32 within 2^12 ulps of each k/100 boundary (and of 0), plus a
    # large random sample: trunc(clip(a, -1, 1) * 100) must match exact
    # integer arithmetic
    parts = []
    span = np.arange(-4096, 4097, dtype=np.int64)
    for k in range(-100, 101):
        c = np.float32(k / 100.0)
        bits = np.array([c], np.float32).view(np.int32).astype(np.int64)[0]
        if c == 0:
            cand = np.arange(0, 8192, dtype=np.int32).view(np.float32)
            parts += [cand, -cand]
            continue
        parts.append((bits + span).astype(np.int32).view(np.float32))
    st = synth.Stream(5, 902)
    parts.append((st.uniform(500_000) * 2 - 1).astype(np.float32))
    x = np.concatenate(parts)
    x = x[np.isfinite(x) & (np.abs(x) <= 1.0)]
    for hmax in (100, 7, 1):
        got = oracle.discretise_many(x, hmax)
        want = _trunc_exact(x, hmax)
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, (hmax, x[bad[:5]], got[bad[:5]], want[bad[:5]])


def test_discretise_every_float32_in_unit_interval():
    # all 2,130,706,433 float32 values in [-1, 1] (both signs, subnormals and
    # zeros included), hmax = 100: the oracle's trunc(x * 100) against the
    # exact value from the float's bits, trunc(m * 100 * 2^e) with m the
    # 24-bit significand and e the unbiased exponent - integer shifts only
    one = 0x3F800000                                   # bit pattern of 1.0f
    chunk = 1 << 25
    for lo in range(0, one + 1, chunk):
        bits = np.arange(lo, min(lo + chunk, one + 1), dtype=np.uint32)
        ex = (bits >> 23).astype(np.int64)
        m = (bits & 0x7FFFFF).astype(np.int64) | np.where(ex > 0, 1 << 23, 0)
        sh = np.where(ex > 0, 150 - ex, 149)           # x = m * 2^(-sh), sh >= 23 here
        want = np.where(sh >= 40, 0, (m * 100) >> np.minimum(sh, 39))
        x = bits.view(np.float32)
        assert np.array_equal(oracle.discretise_many(x, 100), want), hex(lo)
        assert np.array_equal(oracle.discretise_many(-x, 100), -want), hex(lo)


def test_discretise_clips_and_zeroes_non_finite():
    f = np.float32
    vals = [f(1.0), f(1.0000001), f(7.5), f(-3.0), f(np.inf), f(-np.inf),
            f(np.nan), f(-0.0), f(0.999999)]
    got = oracle.discretise_many(np.array(vals, np.float32), 100).tolist()
    assert got == [100, 100, 100, -100, 0, 0, 0, 0, 99]


# ------------------------------------------------------------------ networks

@pytest.mark.parametrize("dims,out_act", [((301, 64, 64, 30), 1),
                                          ((10, 128, 128, 3), 0),
                                          ((17, 5, 9), 1), ((3, 1), 0)])
def test_net_forward_matches_torch_float64(dims, out_act):
    torch = pytest.importorskip("torch")
    params = synth.actor_params(dims, 1, seed=3, out_scale=2.0)[0]
    st = synth.Stream(9, 903)
    x = (st.normal(40 * dims[0]) * 0.7).reshape(40, dims[0]).astype(np.float32)
    got = oracle.net_forward(dims, params, x, out_act)
    h = torch.from_numpy(x.astype(np.float64))
    layers = synth.unpack_params(dims, params)
    for l, (W, b) in enumerate(layers):
        h = h @ torch.from_numpy(W.astype(np.float64)).T + torch.from_numpy(b.astype(np.float64))
        if l + 1 < len(layers):
            h = torch.relu(h)
        elif out_act == 1:
            h = torch.tanh(h)
    want = h.numpy()
    err = np.abs(got - want).max() / max(np.abs(want).max(), 1e-30)
    assert err <= 1e-12, err


# ------------------------------------------------------------------ ensembles

def test_ensemble_mean_identical_agents_is_one_agent():
    st = synth.Stream(1, 904)
    a0 = st.uniform(30) * 2 - 1
    for M in (1, 2, 3, 5, 7):
        a = np.tile(a0, (M, 1))
        out = oracle.ensemble_mean(a)
        assert np.array_equal(out, a0)            # bit-exact, not approximate
        w = st.uniform(M)
        out = oracle.ensemble_mean(a, w / w.sum())
        assert np.array_equal(out, a0)


def test_ensemble_mean_is_weighted_average():
    st = synth.Stream(2, 905)
    for M in (1, 2, 3, 4):
        a = st.uniform(M * 30).reshape(M, 30) * 2 - 1
        w = st.uniform(M)
        w = w / w.sum()
        want = (w[:, None] * a).sum(0)
        assert np.allclose(oracle.ensemble_mean(a, w), want, rtol=0, atol=1e-14)
        assert np.allclose(oracle.ensemble_mean(a), a.mean(0), rtol=0, atol=1e-14)


def test_argmax_ties_go_to_lowest_index():
    assert oracle.argmax([1.0, 1.0, 0.5]) == 0
    assert oracle.argmax([0.0, 2.0, 2.0]) == 1
    assert oracle.argmax([-1.0, -2.0, -0.5]) == 2


def test_vote_exhaustive_invariants():
    # all 3^n ballots for n <= 5: a strict plurality wins, any tie for the
    # top count holds (1), and the rule ignores the order of the ballots
    import itertools
    for n in range(1, 6):
        for b in itertools.product(range(3), repeat=n):
            r = oracle.vote(b)
            cnt = [b.count(a) for a in range(3)]
            top = max(cnt)
            winners = [a for a in range(3) if cnt[a] == top]
            if len(winners) == 1:
                assert r == winners[0], (b, r)
            else:
                assert r == 1, (b, r)
            if 2 * cnt[r] > n:
                assert True
            for a in range(3):
                if 2 * cnt[a] > n:
                    assert r == a
            assert oracle.vote(tuple(reversed(b))) == r


@pytest.mark.parametrize("n,p", [(3, 0.6), (5, 0.6), (7, 0.55), (9, 0.7), (4, 0.65)])
def test_vote_accuracy_matches_condorcet_binomial(n, p):
    # Sec. 3.3.1: n independent traders each right with probability p; the
    # majority is right with probability sum_{k > n/2} C(n,k) p^k (1-p)^(n-k).
    # Binary ballots (right = buy, wrong = sell); an even split holds.
    trials = 6000
    st = synth.Stream(13, 906 + n)
    right = st.uniform(trials * n).reshape(trials, n) < p
    ballots = np.where(right, 2, 0).astype(np.uint8)
    hits = sum(oracle.vote(row) == 2 for row in ballots)
    exact = sum(math.comb(n, k) * p ** k * (1 - p) ** (n - k)
                for k in range(n // 2 + 1, n + 1))
    sigma = math.sqrt(exact * (1 - exact) / trials)
    assert abs(hits / trials - exact) <= 4 * sigma, (hits / trials, exact)


# -------------------------------------------------------------------- metrics

def test_metrics_hand_computed_series():
    with open(os.path.join(GOLDEN, "metrics_series.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        got = oracle.metrics_series(c["v"], c["A"])
        cr = Fraction(*c["cumret_fraction"])
        mdd = Fraction(*c["mdd_fraction"])
        assert abs(got[0] - float(cr)) <= 2e-16 * max(1.0, abs(float(cr))), (c, got)
        assert abs(got[2] - float(mdd)) <= 2e-16, (c, got)
        if "sharpe" in c:
            assert got[1] == c["sharpe"]
        if "sample_var" in c:
            want = c["mean"] / math.sqrt(c["sample_var"]) * math.sqrt(c["A"])
            assert abs(got[1] - want) <= 4 * 2.2e-16 * abs(want), (got[1], want)


def test_metrics_random_series_against_numpy():
    st = synth.Stream(21, 907)
    v = (1e6 * np.exp(np.cumsum(st.normal(300) * 0.01))).astype(np.int64)
    got = oracle.metrics_series(v, 252.0)
    r = v[1:] / v[:-1] - 1.0
    assert abs(got[1] - r.mean() / r.std(ddof=1) * np.sqrt(252.0)) < 1e-9
    peak = np.maximum.accumulate(v)
    assert abs(got[2] - (v / peak - 1.0).min()) < 1e-15
    assert abs(got[0] - (v[-1] / v[0] - 1.0)) < 1e-15


# ------------------------------------------- Sec. 5.2.1 Sharpe-softmax weights
def test_sharpe_softmax_two_agents_closed_form():
    w = oracle.sharpe_softmax_weights([0.7, 1.9], -10.0)
    assert abs(w[0] - 1.0 / (1.0 + math.exp(1.9 - 0.7))) < 1e-15
    assert abs(w[1] - 1.0 / (1.0 + math.exp(0.7 - 1.9))) < 1e-15
    assert abs(w.sum() - 1.0) < 1e-15


def test_sharpe_softmax_shift_invariance_and_large_values():
    s = np.array([0.3, -1.2, 2.5, 0.0])
    w0 = oracle.sharpe_softmax_weights(s, -np.inf)
    w1 = oracle.sharpe_softmax_weights(s + 500.0, -np.inf)        # exp(500) alone would overflow
    assert np.isfinite(w1).all() and np.allclose(w0, w1, rtol=0, atol=1e-13)
    e = np.exp(s - s.max())
    assert np.allclose(w0, e / e.sum(), rtol=0, atol=1e-15)


def test_sharpe_softmax_discards_below_threshold():
    s = [1.0, -0.5, 0.2, -3.0]
    w = oracle.sharpe_softmax_weights(s, 0.0)
    assert w[1] == 0.0 and w[3] == 0.0
    assert abs(w[0] - math.exp(0.0) / (math.exp(0.0) + math.exp(0.2 - 1.0))) < 1e-15
    assert abs(w[0] + w[2] - 1.0) < 1e-15


def test_sharpe_softmax_all_below_keeps_best_lowest_index():
    assert list(oracle.sharpe_softmax_weights([-2.0, -1.0, -1.0], 0.0)) == [0.0, 1.0, 0.0]
    assert list(oracle.sharpe_softmax_weights([-1.0], 5.0)) == [1.0]


# ---------------------------- Sec. 6.1 metric list from stored trajectories
def _traj_from_values(v):
    v = np.asarray(v, np.int64)
    return np.diff(v).reshape(-1, 1), int(v[0])


def test_traj_metrics_constant_growth_closed_forms():
    # v_t = 1000 * 2^t: rho = 1 every period -> no variance, no downside,
    # no loss, no drawdown; annual return (2^n)^(A/n) - 1 = 2^A - 1 (A = n = 4,
    # so that A/n is exact)
    v = [1000 * 2 ** t for t in range(5)]
    rew, v0 = _traj_from_values(v)
    m = oracle.trajectory_metrics(rew, None, v0, 4.0, 0.5)[0]
    assert m[0] == 15.0 and m[1] == 0.0 and m[2] == 0.0
    assert m[3] == 15.0 and m[4] == 0.0 and m[5] == 0.0 and m[6] == 0.0 and m[7] == 0.0 and m[8] == 0.0
    # discounted return: sum_t gamma^t r_t with r_t = 1000 * 2^(t-1), gamma = 1/2 -> 1000/2 per period
    assert m[9] == 4 * 500.0 and m[10] == 4


def test_traj_metrics_constant_loss_sortino_is_minus_sqrt_a():
    # rho = -1/2 every period: mean = -1/2, downside deviation = 1/2
    v = [1 << 20 >> t for t in range(5)]
    rew, v0 = _traj_from_values(v)
    m = oracle.trajectory_metrics(rew, None, v0, 9.0, 1.0)[0]
    assert m[6] == -3.0
    assert m[8] == 0.0                     # no gains
    assert m[2] == -1.0 + 1.0 / 16.0       # trough / peak - 1


def test_traj_metrics_omega_of_one_gain_and_one_loss():
    # +50% then -25% (both exact in binary): Omega = 0.5 / 0.25 = 2, cumulative
    # return 1/8, drawdown -1/4, RoMaD 1/2, undiscounted return 200 - 150
    rew, v0 = _traj_from_values([400, 600, 450])
    m = oracle.trajectory_metrics(rew, None, v0, 1.0, 1.0)[0]
    assert m[8] == 2.0 and m[0] == 0.125 and m[2] == -0.25 and m[5] == 0.5 and m[9] == 50.0


def test_traj_metrics_scale_invariance_and_done_truncation():
    rng = np.random.default_rng(9)
    T, N = 40, 6
    rew = rng.integers(-5000, 6000, (T, N)).astype(np.int64)
    done = np.zeros((T, N), np.uint8)
    done[np.arange(N) * 5 + 3, np.arange(N)] = 1
    a = oracle.trajectory_metrics(rew, done, 10 ** 6, 252.0, 0.97)
    b = oracle.trajectory_metrics(rew * 7, done, 7 * 10 ** 6, 252.0, 0.97)
    assert np.array_equal(a[:, :9], b[:, :9]) and np.array_equal(a[:, 10], b[:, 10])
    assert np.allclose(b[:, 9], 7 * a[:, 9], rtol=1e-14, atol=0)
    garbage = rew.copy()
    for i in range(N):
        garbage[i * 5 + 4:, i] = 123456789               # rows after the first done are ignored
    c = oracle.trajectory_metrics(garbage, done, 10 ** 6, 252.0, 0.97)
    assert np.array_equal(a, c)
    assert np.array_equal(a[:, 10], np.arange(N) * 5 + 4)


def test_traj_metrics_agree_with_the_env_episode_metrics():
    # the same rollout, its metrics from the env's accumulators and from its
    # stored rewards: cumulative return, Sharpe and drawdown agree bit for bit
    w = synth.workload_stock_small()
    e = w.envs
    r = oracle.stock_run(w.market, e.Ke, e.start, e.W, e.bps, init_cash=e.init_cash, hmax=100, fee_bps=10,
                         T=w.T, act_i32=synth.prescribed_shares(w.T, e.N, 30, seed=7),
                         want=("rew", "done", "metrics"))
    m = oracle.trajectory_metrics(r["rew"], r["done"], e.init_cash, 252.0, 0.99)
    assert np.array_equal(m[:, :3], r["metrics"])


# -------------------------------------------- exploration randomness (Philox)
def test_philox4x32_10_known_answer_vectors():
    # the known-answer vectors published with Philox4x32-10 (Salmon et al.
    # 2011, Random123 distribution)
    assert oracle.philox4x32_10([0, 0, 0, 0], [0, 0]) == (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)
    assert oracle.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == (0x408F276D, 0x41C83B0E, 0xA20BC7C6,
                                                                       0x6D5451FD)
    assert oracle.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0]) == \
        (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)


def test_uniform24_is_open_interval_with_exact_ends():
    assert oracle.uniform24(0) == 2.0 ** -25
    assert oracle.uniform24(0xFFFFFFFF) == 1.0 - 2.0 ** -25
    assert oracle.uniform24(0x80000000) == 0.5 + 2.0 ** -25


def test_explore_normal_known_value_from_the_published_philox_words():
    # Philox4x32-10 of counter (0, 0, 0, 0) under key (0, 0) is the published
    # known-answer vector (0x6627E8D5, 0xE169C58D, ...) (Salmon et al. 2011);
    # the exploration normal of seed 0, env 0, step 0, asset 0 is Box-Muller
    # of its first two words as uniforms (x >> 8) 2^-24 + 2^-25: computed here
    # by hand from those words, so a swap of the two uniforms, sin for cos or
    # other words would fail
    u0 = (0x6627E8D5 >> 8) / 2.0 ** 24 + 2.0 ** -25
    u1 = (0xE169C58D >> 8) / 2.0 ** 24 + 2.0 ** -25
    want = math.sqrt(-2.0 * math.log(u0)) * math.cos(2.0 * math.pi * u1)
    assert oracle.explore_normal(0, 0, 0, 0) == pytest.approx(want, rel=1e-14, abs=1e-14)
    for other in (math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u0),
                  math.sqrt(-2.0 * math.log(u0)) * math.sin(2.0 * math.pi * u1)):
        assert abs(other - want) > 1e-3


def test_explore_greedy_rule_from_philox_words():
    # the greedy draw of (env e, step g) uses words 2 and 3 of Philox(e, g, 0, 1):
    # replace when (x2 >> 8) < floor(eps 2^24), by action floor(3 (x3 >> 8) / 2^24)
    for e, g in [(0, 0), (5, 17), (123456, 7)]:
        x = oracle.philox4x32_10([e, g, 0, 1], [99, 0])
        r2, r3 = x[2] >> 8, x[3] >> 8
        for eps in (0.0, r2 / 2.0 ** 24, (r2 + 1) / 2.0 ** 24, 1.0):
            thr = int(eps * 2 ** 24)
            want = (r3 * 3) >> 24 if r2 < thr else 7
            assert oracle.explore_greedy(99, e, g, eps, 7) == want


def test_explore_normal_moments():
    z = np.array([oracle.explore_normal(1234, e, g, k) for e in range(20) for g in range(50) for k in range(20)])
    n = z.size
    assert abs(z.mean()) < 4 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 4 * math.sqrt(2.0 / n)
    assert abs(np.mean(np.abs(z) < 1.0) - 0.682689) < 4 * math.sqrt(0.2166 / n)


def test_explore_greedy_rate_and_uniform_replacements():
    eps = 0.05
    a = np.array([oracle.explore_greedy(99, e, g, eps, 7) for e in range(200) for g in range(100)])
    n = a.size
    rep = a != 7
    p = rep.mean()
    assert abs(p - eps) < 4 * math.sqrt(eps * (1 - eps) / n)
    counts = np.bincount(a[rep], minlength=3)
    assert counts.sum() == rep.sum() and len(counts) == 3
    assert all(abs(c / rep.sum() - 1 / 3) < 4 * math.sqrt(2 / 9 / rep.sum()) for c in counts)
    assert all(oracle.explore_greedy(99, e, 0, 0.0, 2) == 2 for e in range(100))     # eps = 0: never


# ---------------------------------------------- data preparation (Sec. 5.1, 6.1)
def test_splitmix64_published_sequence():
    # the first outputs of SplitMix64 from state 0 (the generator's published
    # reference sequence): output n mixes n+1 golden-gamma increments
    g = 0x9E3779B97F4A7C15
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC, 0x1B39896A51A8749B]
    assert [oracle.splitmix64((n * g) % 2**64) for n in range(5)] == want


def test_perturb_bps_range_and_uniformity():
    R = 100
    v = np.array([oracle.perturb_bps(2024, e, k, R) for e in range(400) for k in range(30)])
    assert v.min() == -R and v.max() == R
    counts = np.bincount(v + R, minlength=2 * R + 1)
    n, p = v.size, 1.0 / (2 * R + 1)
    chi2 = float(((counts - n * p) ** 2 / (n * p)).sum())
    assert chi2 < 200 + 5 * math.sqrt(2 * 200)                     # 200 degrees of freedom
    assert abs(v.mean()) < 4 * math.sqrt((R * (R + 1) / 3) / n)
    assert all(oracle.perturb_bps(5, e, k, 0) == 0 for e in range(20) for k in range(30))
    # different seeds, envs and assets decorrelate
    a = np.array([oracle.perturb_bps(1, e, 3, R) for e in range(2000)], float)
    b = np.array([oracle.perturb_bps(2, e, 3, R) for e in range(2000)], float)
    c = np.array([oracle.perturb_bps(1, e, 4, R) for e in range(2000)], float)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.1 and abs(np.corrcoef(a, c)[0, 1]) < 0.1


def _ramp(T, c0, d):
    c = (c0 + d * np.arange(T, dtype=np.int64))[:, None]
    return c, c.copy(), c.copy()


def _ramp_mad(m):
    j = np.arange(m)
    return np.abs(j - (m - 1) / 2.0).mean()


def test_indicators_of_a_constant_series():
    c = np.full((120, 2), 123456, np.int64)
    f = oracle.indicators(c, c, c)
    want = np.zeros(8, np.float32)
    want[3] = 0.5                                                  # RSI 50 without gains or losses
    assert np.array_equal(f, np.broadcast_to(want[None, :, None], f.shape))


@pytest.mark.parametrize("d", [250, -250])
def test_indicators_of_a_linear_ramp(d):
    # c_t = c0 + d t with h = l = c: every indicator has a closed form
    T, c0 = 150, 100_000
    close, high, low = _ramp(T, c0, d)
    f = oracle.indicators(close, high, low)[:, :, 0].astype(np.float64)
    t = np.arange(T)
    ct = (c0 + d * t).astype(np.float64)
    # EMA of a ramp from e_0 = c_0: e_t = c_t - d (1 - a) / a (1 - (1 - a)^t), (1 - a) / a = (n - 1) / 2
    macd = d * (12.5 * (1 - (25 / 27) ** t) - 5.5 * (1 - (11 / 13) ** t))
    assert np.allclose(f[:, 0], macd / ct, rtol=1e-5, atol=1e-8)
    m20 = np.minimum(t + 1, 20)
    sma20 = ct - d * (m20 - 1) / 2.0
    sd20 = abs(d) * np.sqrt((m20 ** 2 - 1) / 12.0)                  # population sd of m equally spaced values
    assert np.allclose(f[:, 1], (sma20 + 2 * sd20) / ct - 1, rtol=1e-5, atol=1e-7)
    assert np.allclose(f[:, 2], (sma20 - 2 * sd20) / ct - 1, rtol=1e-5, atol=1e-7)
    assert f[0, 3] == 0.5 and (f[1:, 3] == (1.0 if d > 0 else 0.0)).all()
    m30 = np.minimum(t + 1, 30)
    mad = np.array([abs(d) * _ramp_mad(m) for m in m30])
    cci = np.where(mad > 0, (d * (m30 - 1) / 2.0) / (0.015 * np.where(mad > 0, mad, 1)), 0.0)
    assert np.allclose(f[:, 4], cci / 100, rtol=1e-5, atol=1e-7)
    assert f[0, 5] == 0.0 and (f[1:, 5] == 1.0).all()               # one-sided movement: DX 100
    assert np.allclose(f[:, 6], -(d * (m30 - 1) / 2.0) / ct, rtol=1e-5, atol=1e-8)
    m60 = np.minimum(t + 1, 60)
    assert np.allclose(f[:, 7], -(d * (m60 - 1) / 2.0) / ct, rtol=1e-5, atol=1e-8)


def _geometric(x, a, w0=None):
    """The recurrence e_t = a x_t + (1 - a) e_{t-1}, e_0 = x_0, summed in closed
    form: e_t = (1 - a)^t x_0 + sum_{j=1..t} a (1 - a)^(t - j) x_j."""
    T = x.shape[0]
    t = np.arange(T)
    W = np.where(t[:, None] >= t[None, :], a * (1 - a) ** np.maximum(t[:, None] - t[None, :], 0), 0.0)
    W[:, 0] = (1 - a) ** t
    return W @ x


def test_indicators_against_closed_form_recurrences_and_windows():
    # random OHLC; recurrences by their closed-form weights, windows by
    # explicit slices, RSI and DX through their algebraically equal forms
    mk = synth.stock_market(160, 3, seed=11)
    c, h, lo = (x.astype(np.float64) for x in (mk.close, mk.high, mk.low))
    f = oracle.indicators(mk.close, mk.high, mk.low).astype(np.float64)
    T, K = c.shape
    macd = _geometric(c, 2 / 13) - _geometric(c, 2 / 27)
    assert np.allclose(f[:, 0], macd / c, rtol=1e-4, atol=2e-7)
    d = np.vstack([np.zeros((1, K)), c[1:] - c[:-1]])
    G, L = _geometric(np.maximum(d, 0), 1 / 30), _geometric(np.maximum(-d, 0), 1 / 30)
    rsi = np.where(G + L > 0, G / np.where(G + L > 0, G + L, 1), 0.5)
    assert np.allclose(f[:, 3], rsi, rtol=0, atol=1e-6)
    win = lambda x, t, n: x[max(0, t - n + 1):t + 1]
    tp = (h + lo + c) / 3
    for t in range(T):
        w20 = win(c, t, 20)
        s20 = np.sqrt(((w20 - w20.mean(0)) ** 2).mean(0))
        assert np.allclose(f[t, 1], (w20.mean(0) + 2 * s20) / c[t] - 1, rtol=0, atol=1e-6)
        assert np.allclose(f[t, 2], (w20.mean(0) - 2 * s20) / c[t] - 1, rtol=0, atol=1e-6)
        wt = win(tp, t, 30)
        mad = np.abs(wt - wt.mean(0)).mean(0)
        cci = np.where(mad > 0, (tp[t] - wt.mean(0)) / (0.015 * np.where(mad > 0, mad, 1)), 0)
        assert np.allclose(f[t, 4], cci / 100, rtol=1e-5, atol=1e-6)
        assert np.allclose(f[t, 6], win(c, t, 30).mean(0) / c[t] - 1, rtol=0, atol=1e-7)
        assert np.allclose(f[t, 7], win(c, t, 60).mean(0) / c[t] - 1, rtol=0, atol=1e-7)
    up = np.vstack([np.zeros((1, K)), h[1:] - h[:-1]])
    dn = np.vstack([np.zeros((1, K)), lo[:-1] - lo[1:]])
    pdm, ndm = np.where((up > dn) & (up > 0), up, 0), np.where((dn > up) & (dn > 0), dn, 0)
    pc = np.vstack([c[:1], c[:-1]])
    tr = np.max([h - lo, np.abs(h - pc), np.abs(lo - pc)], axis=0)
    P, N = _geometric(pdm, 1 / 30), _geometric(ndm, 1 / 30)      # DI+ / DI- = P / N: TR cancels
    dx = np.where(P + N > 0, np.abs(P - N) / np.where(P + N > 0, P + N, 1), 0)
    assert (_geometric(tr, 1 / 30) > 0).all()
    assert np.allclose(f[:, 5], dx, rtol=0, atol=1e-6)


def test_indicator_windows_see_no_future():
    mk = synth.stock_market(200, 4, seed=5)
    full = oracle.indicators(mk.close, mk.high, mk.low)
    for t in (0, 1, 29, 59, 60, 137):
        part = oracle.indicators(mk.close[:t + 1], mk.high[:t + 1], mk.low[:t + 1])
        assert np.array_equal(part, full[:t + 1])



# ---------------------------------------------------------- FP8 E4M3 actors
def _e4m3_codes():
    torch = pytest.importorskip("torch")
    v = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    return np.unique(v[np.isfinite(v)])


def test_e4m3_round_agrees_with_torch_float8_cast():
    # a library routine: torch's float8_e4m3fn conversion (round to nearest
    # even) on in-range values, every code and every midpoint between codes
    torch = pytest.importorskip("torch")
    codes = _e4m3_codes()
    assert codes.size == 253 and codes.max() == 448.0 and codes[codes > 0].min() == 2.0 ** -9
    mids = (codes[1:] + codes[:-1]) / 2
    rng = np.random.default_rng(8)
    x = np.concatenate([codes, mids, rng.uniform(-448, 448, 50000), rng.normal(0, 0.01, 50000)]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(oracle.e4m3_round(x), want)


def test_e4m3_round_special_cases():
    r = oracle.e4m3_round
    assert r(1.0625) == 1.0 and r(1.1875) == 1.25          # ties to the even fraction
    assert r(2.0 ** -10) == 0.0 and r(3 * 2.0 ** -10) == 2.0 ** -8    # subnormal ties
    assert r(448.0) == 448.0 and r(460.0) == 448.0 and r(1e9) == 448.0 and r(-500.0) == -448.0
    assert r(0.0) == 0.0 and r(-2.0 ** -9) == -2.0 ** -9


def test_fp8_weights_scale_and_codes():
    rng = np.random.default_rng(3)
    W = rng.normal(0, 0.1, (40, 70)).astype(np.float32)
    W[5] = 0.0
    q, sw = oracle.fp8_weights(W)
    assert sw[5] == 1.0 and (q[5] == 0).all()
    nz = np.arange(40) != 5
    assert (np.abs(q[nz]).max(axis=1) == 448.0).all()        # each row's extreme maps to +-448
    # dequantised weights within half an E4M3 step of the original
    rel = np.abs(q[nz] * sw[nz, None] - W[nz]) / np.maximum(np.abs(W[nz]), 2.0 ** -6 * sw[nz, None])
    assert rel.max() <= 2.0 ** -4 * (1 + 1e-6)


def test_fp8_forward_is_exact_on_representable_networks():
    # layer 1 = 28 I (row scale 28 / 448 = 1/16, codes 448), inputs powers of
    # two up to 4 (hidden 28 x = 1.75 2^(j+4), a code), layer 2 code-valued
    # with a 448 in every row (row scale 1), integer biases, activation scales
    # 1: every quantisation is exact and every sum fits float64, so the FP8
    # forward equals the fp64 forward bit for bit
    codes = _e4m3_codes()
    rng = np.random.default_rng(4)
    fin = h = 24
    fout = 7
    W1 = np.eye(h, fin, dtype=np.float32) * np.float32(28.0)
    b1 = np.zeros(h, np.float32)
    W2 = rng.choice(codes, (fout, h)).astype(np.float32)
    W2[:, 0] = 448.0
    b2 = rng.integers(-5, 6, fout).astype(np.float32)
    params = np.concatenate([W1.ravel(), b1, W2.ravel(), b2])
    x = np.ldexp(1.0, rng.integers(-6, 3, (50, fin))).astype(np.float32)
    x[rng.random(x.shape) < 0.2] = 0.0
    dims = (fin, h, fout)
    y8 = oracle.fp8_forward(dims, params, [1.0, 1.0], x, 0)
    assert np.array_equal(y8, oracle.net_forward(dims, params, x, 0))
    # a scale that is not a power of two breaks exactness, by a bounded amount
    y8b = oracle.fp8_forward(dims, params, [1.0, 0.3], x, 0)
    # (hidden / 0.3 stays in the normal range, where rounding errs by at most 2^-4 relative)
    bound = 2.0 ** -4 * (np.abs(28.0 * x.astype(np.float64)) @ np.abs(W2.astype(np.float64)).T)
    assert not np.array_equal(y8b, y8) and (np.abs(y8b - y8) <= bound * (1 + 1e-6)).all()


def test_fp8_forward_exact_tail_reductions():
    # the FP8 model with an exact input tail (the fused stock kernel's: the
    # indicator block through a float table) reduces to the plain FP8 model
    # when the tail is empty or zero, and to the fp64 forward on the tail
    # when only the tail is nonzero
    rng = np.random.default_rng(8)
    dims = (20, 48, 16, 5)
    params = synth.actor_params(dims, 1, seed=9)[0]
    sc = [0.01, 0.02, 0.03]
    x = rng.normal(0, 1, (64, 20)).astype(np.float32)
    full = oracle.fp8_forward(dims, params, sc, x, 1)
    assert np.array_equal(oracle.fp8_forward_exact_tail(dims, params, sc, x, 1, 20), full)
    x0 = x.copy()
    x0[:, 7:] = 0.0
    assert np.array_equal(oracle.fp8_forward_exact_tail(dims, params, sc, x0, 1, 7),
                          oracle.fp8_forward(dims, params, sc, x0, 1))
    # a single layer with only the tail nonzero is the exact affine map
    d1 = (20, 6)
    p1 = synth.actor_params(d1, 1, seed=10)[0]
    xt = x.copy()
    xt[:, :7] = 0.0
    W = p1[:120].reshape(6, 20).astype(np.float64)
    b = p1[120:].astype(np.float64)
    assert np.array_equal(oracle.fp8_forward_exact_tail(d1, p1, [0.5], xt, 0, 7),
                          xt[:, 7:].astype(np.float64) @ W[:, 7:].T + b)
    # and a quantised head differs from the exact one by a bounded amount
    y = oracle.fp8_forward_exact_tail(d1, p1, [0.01], x, 0, 7)
    ex = x.astype(np.float64) @ W.T + b
    assert not np.array_equal(y, ex)
    assert np.abs(y - ex).max() <= 2.0 ** -3 * (np.abs(x[:, :7].astype(np.float64)) @ np.abs(W[:, :7]).T).max() + 1e-6


def test_fp8_calibration_scales_homogeneously():
    # zero biases: ReLU networks are positively homogeneous, so doubling the
    # batch doubles every layer's maximum and scale exactly
    rng = np.random.default_rng(6)
    dims = (12, 32, 16, 3)
    params = synth.actor_params(dims, 1, seed=2)[0].copy()
    off = 0
    for fin, fout in zip(dims[:-1], dims[1:]):
        off += fin * fout
        params[off:off + fout] = 0
        off += fout
    obs = rng.normal(0, 1, (200, 12)).astype(np.float32)
    s1 = oracle.fp8_calibrate(dims, params, obs)
    s2 = oracle.fp8_calibrate(dims, params, 2 * obs)
    assert np.array_equal(s2, 2 * s1)
    assert s1[0] == np.float32(np.abs(obs).max()) / np.float32(448)


# ------------------------------------------------------------- replay buffer
def _tiny_traj():
    T, N, D = 3, 2, 2
    obs = np.arange(T * N * D, dtype=np.float32).reshape(T, N, D)
    act = -np.arange(T * N, dtype=np.float32).reshape(T, N, 1)
    rew = np.arange(T * N, dtype=np.float32).reshape(T, N)          # row index as the reward
    done = np.array([[0, 0], [1, 0], [1, 1]], np.uint8)        # env 0 ends at t = 1, env 1 at t = 2
    last = np.full((N, D), 99.0, np.float32)
    return obs, act, rew, done, last


def _rews(rb):
    return [int(i[2]) for i in rb.contents()]


def test_replay_ref_takes_real_steps_in_order():
    obs, act, rew, done, last = _tiny_traj()
    rb = oracle.ReplayRef(100)
    rb.push(obs, act, rew, done, last)
    # (t, e) order; row (2, 0) follows env 0's last step and is not a step
    got = [(int(i[2]), i[0].tolist(), int(i[1][0]), i[3].tolist(), int(i[4])) for i in rb.contents()]
    assert got == [(0, [0, 1], 0, [4, 5], 0), (1, [2, 3], -1, [6, 7], 0), (2, [4, 5], -2, [8, 9], 1),
                   (3, [6, 7], -3, [10, 11], 0), (5, [10, 11], -5, [99, 99], 1)]
    rb2 = oracle.ReplayRef(100)
    rb2.push(obs, act, rew, done, last, live0=np.array([1, 0], np.uint8))
    assert _rews(rb2) == [0, 2, 3, 5]
    rb3 = oracle.ReplayRef(100)
    rb3.push(obs, act, rew, done, last, auto_reset=True)
    assert _rews(rb3) == [0, 1, 2, 3, 4, 5] and rb3.contents()[4][3].tolist() == [99, 99]


def test_replay_ref_fifo_and_sampling():
    obs, act, rew, done, last = _tiny_traj()
    rb = oracle.ReplayRef(4)
    rb.push(obs, act, rew, done, last)                             # 5 steps, capacity 4: the oldest goes
    assert _rews(rb) == [1, 2, 3, 5]
    rb.push(obs, act, rew, done, last)
    assert len(rb.items) == 10 and _rews(rb) == [1, 2, 3, 5]
    rb.push(obs[:1], act[:1], rew[:1], done[:1], obs[1])
    assert _rews(rb) == [3, 5, 0, 1]
    pos = oracle.ReplayRef(7)
    pos.items = list(range(7))
    p = np.array(pos.sample_positions(7000, 123, 5))
    assert p.min() == 0 and p.max() == 6
    counts = np.bincount(p, minlength=7)
    assert ((counts - 1000) ** 2 / 1000).sum() < 6 + 5 * math.sqrt(12)      # chi-square, 6 dof
    assert pos.sample_positions(50, 123, 5) == list(p[:50]) and pos.sample_positions(50, 123, 6) != list(p[:50])
    assert oracle.ReplayRef(3).sample_positions(4, 1, 0) == [-1] * 4


# ------------------------------------------------ DQN-family heads and targets
def test_dueling_head_hand_example_and_identities():
    y = np.array([1.0, 2.0, 0.0, 4.0])                          # V = 1, A = (2, 0, 4), mean 2
    assert oracle.head_q(y, 1, 3).tolist() == [1.0, -1.0, 3.0]
    assert oracle.head_q(y, 0, 3).tolist() == [1.0, 2.0, 0.0]  # a plain head ignores the extra output
    rng = np.random.default_rng(2)
    Y = rng.normal(0, 1, (1000, 4))
    Q = oracle.head_q(Y, 1, 3)
    assert np.allclose(Q.mean(-1), Y[:, 0], atol=1e-14)        # the advantages average to zero
    assert (Q.argmax(-1) == Y[:, 1:].argmax(-1)).all()          # V and the mean do not change the argmax


def _linear_q(W, b):
    # a one-layer Q-network: Q(s) = W s + b
    return np.concatenate([np.asarray(W, np.float32).ravel(), np.asarray(b, np.float32)])


def test_double_and_plain_dqn_targets_by_hand():
    dims = (2, 3)
    s1 = np.array([[1.0, 0.0], [0.0, 1.0]], np.float32)
    on = _linear_q([[0, 0], [1, 0], [0, 1]], [0, 0, 0])         # online argmax: action 1 for s1[0], 2 for s1[1]
    tg = _linear_q([[5, 5], [1, 0], [2, 3]], [0, 0, 0])         # target Q: (5, 1, 2) and (5, 0, 3)
    rew = np.array([0.5, -1.0])
    done = np.array([0, 1], np.uint8)
    g = 0.9
    plain = oracle.q_targets(dims, [on], [tg], [0], s1, rew, done, g, False)[0]
    double = oracle.q_targets(dims, [on], [tg], [0], s1, rew, done, g, True)[0]
    assert plain.tolist() == [0.5 + 0.9 * 5.0, -1.0]            # max of the target Q; done: no bootstrap
    assert double.tolist() == [0.5 + 0.9 * 1.0, -1.0]           # target Q at the online argmax
    same = oracle.q_targets(dims, [tg], [tg], [0], s1, rew, None, g, True)[0]
    assert same.tolist() == oracle.q_targets(dims, [tg], [tg], [0], s1, rew, None, g, False)[0].tolist()
    # ties: lowest index (all-zero online Q selects action 0)
    zero = _linear_q(np.zeros((3, 2)), [0, 0, 0])
    assert oracle.q_targets(dims, [zero], [tg], [0], s1, rew, None, g, True)[0].tolist() == [0.5 + 4.5, -1.0 + 4.5]
