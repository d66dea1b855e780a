/*
 * finrl_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU restatement of the trading MDP and
 * ensemble rules of "Revisiting Ensemble Methods for Stock Trading and Crypto
 * Trading Tasks at ACM ICAIF FinRL Contests 2023/2024" (arXiv 2501.10709).
 * It exists so that tests, the smoke check and the benchmark's CPU baseline can
 * check the CUDA library against something written independently from the
 * paper.  No product code links, loads or calls it; it shares no source with
 * the CUDA library.
 *
 * Arithmetic: accounting in int64 cents / int32 shares, every floating-point
 * quantity in IEEE fp64, compiled with -ffp-contract=off so that no FMA is
 * formed.  OpenMP is used only across independent environments (Sec. 4.2.1:
 * every trajectory is an independent simulation).
 *
 * Passages followed (paper section / equation):
 *   state  s_t = [b_t, p_t, h_t, f_t]          Sec. 3.1 (MDP, State)
 *   action a_t = change of holdings            Sec. 3.1 (MDP, Action)
 *   reward v_{t+1} - v_t, v_t = b_t + p_t^T h_t Sec. 3.1 (MDP, Reward)
 *   transaction costs as a market constraint   Sec. 3.2
 *   reset / step / reward of every SubEnv      Sec. 4.2.2
 *   T x N x D sample tensors                   Sec. 4.3.2
 *   +-1% per-asset price change                Sec. 5.1 (dataset diversity)
 *   weighted average of agent actions          Sec. 5.2.1
 *   majority vote of discrete actions          Sec. 5.2.2
 *   Sharpe ratio (r_p - r_f) / sigma_p         Sec. 5.2.1, Sharpe equation
 *   cumulative return, maximum drawdown        Sec. 6.1 (performance metrics)
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   prices and cash are integer cents, holdings integer shares >= 0;
 *   an action in [-1,1] becomes trunc(a * hmax) shares (round toward zero);
 *   sells execute before buys; buys fill greedily in ascending asset order
 *   (or, as an option, largest requested count first), partially when cash
 *   runs short; the fee is ceil(notional * fee_bps / 1e4)
 *   per order on both sides; the perturbed price is
 *   max(1, round-half-up(close * (1e4 + bps) / 1e4)); a W-day window has W-1
 *   steps; argmax ties go to the lowest index; a vote with no strict winner
 *   holds; Sharpe uses per-period returns, ddof = 1, r_f = 0 and an
 *   annualisation factor sqrt(A).
 *
 * Pins: every function here is checked in tests/test_oracle_*.py against
 * something other than itself (exact rationals, linear search, brute force
 * with Python fractions, torch float64 matmul, the Condorcet binomial sum of
 * Sec. 3.3.1, hand-computed series).  Parity of the financial result tables
 * (trained agents on real data) is out of scope and unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_BPS_ONE 10000

/* ---------------------------------------------------------------- prices */

/* Sec. 5.1 dataset diversity: a per-asset change of -1%..+1%, held as an
 * integer number of basis points, rounded half up to the cent, floor 1 cent. */
int64_t orc_perturb(int64_t close, int32_t bps)
{
    int64_t num = close * (int64_t)(ORC_BPS_ONE + bps) + ORC_BPS_ONE / 2;
    int64_t p = num / ORC_BPS_ONE;            /* num > 0: division is floor */
    return p < 1 ? 1 : p;
}

/* Transaction cost (Sec. 3.2): ceil(notional * fee_bps / 1e4), notional >= 0 */
int64_t orc_fee(int64_t notional, int32_t fee_bps)
{
    int64_t x = notional * (int64_t)fee_bps;
    return (x + ORC_BPS_ONE - 1) / ORC_BPS_ONE;
}

/* Cost of buying n shares at price p, fee included. */
int64_t orc_buy_cost(int64_t n, int64_t p, int32_t fee_bps)
{
    int64_t g = n * p;
    return g + orc_fee(g, fee_bps);
}

/* Largest affordable share count: floor(cash * 1e4 / (p * (1e4 + fee))),
 * then one step down if the rounded-up fee still breaks the budget. */
int64_t orc_buy_max(int64_t cash, int64_t p, int32_t fee_bps)
{
    if (cash <= 0) return 0;
    int64_t n0 = (cash * ORC_BPS_ONE) / (p * (int64_t)(ORC_BPS_ONE + fee_bps));
    if (n0 > 0 && orc_buy_cost(n0, p, fee_bps) > cash) n0 -= 1;
    return n0;
}

/* Action -> integer share change (Sec. 3.1 action = change of holdings):
 * a non-finite action (NaN, +-Inf) counts as 0; otherwise clip to [-1,1],
 * scale by hmax, truncate toward zero. */
int32_t orc_discretise(double a, int32_t hmax)
{
    if (!isfinite(a)) a = 0.0;
    if (a > 1.0) a = 1.0;
    if (a < -1.0) a = -1.0;
    double y = a * (double)hmax;
    return (int32_t)y;                        /* C conversion truncates */
}

/* ------------------------------------------------------------- MLP forward */

/* One actor (Sec. 6.1 agent networks): L dense layers, parameters packed per
 * layer as W_l[out][in] row-major followed by b_l[out] (fp32 master copy).
 * Hidden layers apply ReLU; the output applies tanh (out_act = 1, stock
 * actor) or nothing (out_act = 0, crypto Q-network).  fp64 throughout. */
static int64_t net_param_count(int L, const int32_t *dims)
{
    int64_t c = 0;
    for (int l = 0; l < L; ++l) c += (int64_t)dims[l + 1] * dims[l] + dims[l + 1];
    return c;
}

int64_t orc_net_param_count(int32_t L, const int32_t *dims)
{
    return net_param_count(L, dims);
}

static void net_forward_row(int L, const int32_t *dims, const float *params,
                            int out_act, const float *x, double *y,
                            double *buf_a, double *buf_b)
{
    const float *pw = params;
    for (int k = 0; k < dims[0]; ++k) buf_a[k] = (double)x[k];
    double *in = buf_a, *out = buf_b;
    for (int l = 0; l < L; ++l) {
        int fi = dims[l], fo = dims[l + 1];
        const float *W = pw;
        const float *b = pw + (int64_t)fo * fi;
        for (int o = 0; o < fo; ++o) {
            double acc = 0.0;
            for (int k = 0; k < fi; ++k) acc += (double)W[(int64_t)o * fi + k] * in[k];
            acc += (double)b[o];
            if (l + 1 < L) acc = acc > 0.0 ? acc : 0.0;          /* ReLU */
            else if (out_act == 1) acc = tanh(acc);
            out[o] = acc;
        }
        pw = b + fo;
        double *t = in; in = out; out = t;
    }
    for (int o = 0; o < dims[L]; ++o) y[o] = in[o];
}

static int max_width(int L, const int32_t *dims)
{
    int w = 0;
    for (int l = 0; l <= L; ++l) if (dims[l] > w) w = dims[l];
    return w;
}

/* y[n][dims[L]] = net(x[n][.]) with row stride ldx for x. */
void orc_net_forward(int32_t L, const int32_t *dims, const float *params,
                     int32_t out_act, const float *x, int32_t ldx, int32_t n,
                     double *y, int32_t nthreads)
{
    int w = max_width(L, dims);
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        double *ba = (double *)malloc(sizeof(double) * w);
        double *bb = (double *)malloc(sizeof(double) * w);
#pragma omp for schedule(static)
        for (int r = 0; r < n; ++r)
            net_forward_row(L, dims, params, out_act, x + (int64_t)r * ldx,
                            y + (int64_t)r * dims[L], ba, bb);
        free(ba);
        free(bb);
    }
}

/* ------------------------------------------------------- ensemble combine */

/* Sec. 5.2.1: weighted average of the agents' actions, written anchored on
 * agent 0 so that identical agents reproduce agent 0 exactly:
 *   a = a_0 + sum_{j>=1} w_j (a_j - a_0).
 * This equals sum_j w_j a_j whenever the weights sum to one.  w == NULL
 * means uniform weights 1/M. */
void orc_ensemble_mean(int32_t M, int32_t K, const double *a, const double *w,
                       double *out)
{
    for (int k = 0; k < K; ++k) {
        double acc = a[k];
        for (int j = 1; j < M; ++j) {
            double wj = w ? w[j] : 1.0 / (double)M;
            acc += wj * (a[(int64_t)j * K + k] - a[k]);
        }
        out[k] = acc;
    }
}

/* argmax with ties to the lowest index */
int32_t orc_argmax(const double *q, int32_t n)
{
    int best = 0;
    for (int i = 1; i < n; ++i) if (q[i] > q[best]) best = i;
    return best;
}

/* Sec. 5.2.2 majority vote over M discrete ballots in {0 sell, 1 hold,
 * 2 buy}: the action with the strictly largest count; any tie for the top
 * count holds. */
int32_t orc_vote(int32_t M, const uint8_t *ballots)
{
    int cnt[3] = {0, 0, 0};
    for (int j = 0; j < M; ++j) if (ballots[j] < 3) cnt[ballots[j]]++;
    int best = -1, bestc = -1, tie = 0;
    for (int a = 0; a < 3; ++a) {
        if (cnt[a] > bestc) { bestc = cnt[a]; best = a; tie = 0; }
        else if (cnt[a] == bestc) tie = 1;
    }
    return tie ? 1 : best;
}

/* ------------------------------------------------ exploration randomness */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw 2011): ten rounds of two 32x32
 * multiplications; each round maps (c0, c1, c2, c3) with key (k0, k1) to
 * (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)), and the
 * key is bumped by the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A uniform in (0, 1) from the top 24 bits: (x >> 8) 2^-24 + 2^-25 (exact in
 * float32 and double). */
double orc_uniform24(uint32_t x)
{
    return (double)(x >> 8) * (1.0 / 16777216.0) + 1.0 / 33554432.0;
}

/* Exploration draws of env e at global step g, component k (seed = key):
 * z = sqrt(-2 ln u0) cos(2 pi u1), Box-Muller (double) from the first two
 * words of Philox(ctr = (e, g, k, 0)); greedy replacement when
 * (x2 >> 8) < floor(eps 2^24) -- probability floor(eps 2^24) / 2^24 -- by
 * the action floor(3 (x3 >> 8) / 2^24), from Philox(ctr = (e, g, 0, 1)). */
double orc_explore_normal(uint64_t seed, uint32_t e, uint32_t g, uint32_t k)
{
    const uint32_t ctr[4] = {e, g, k, 0u}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    const double u0 = orc_uniform24(x[0]), u1 = orc_uniform24(x[1]);
    return sqrt(-2.0 * log(u0)) * cos(2.0 * 3.14159265358979323846 * u1);
}

int32_t orc_explore_greedy(uint64_t seed, uint32_t e, uint32_t g, double eps, int32_t action)
{
    const uint32_t ctr[4] = {e, g, 0u, 1u}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    const uint32_t thr = (uint32_t)(eps * 16777216.0);
    if ((x[2] >> 8) < thr) return (int32_t)(((uint64_t)(x[3] >> 8) * 3u) >> 24);
    return action;
}

/* ----------------------------------------------- on-device data preparation */
/* SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014; Stafford's
 * mix13 finaliser): add the golden gamma, then three xor-shift / multiply
 * steps.  Written from the published definition. */
uint64_t orc_splitmix64(uint64_t x)
{
    x = x + 0x9E3779B97F4A7C15ull;
    x = x ^ (x >> 30);
    x = x * 0xBF58476D1CE4E5B9ull;
    x = x ^ (x >> 27);
    x = x * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

/* Sec. 5.1 per-env +-1% price change (R = 100 bps): env e, asset k draws
 * z = splitmix64(seed ^ splitmix64(e * 256 + k)) and takes z mod (2R + 1) - R. */
int32_t orc_perturb_bps(uint64_t seed, uint32_t e, uint32_t k, int32_t R)
{
    const uint64_t z = orc_splitmix64(seed ^ orc_splitmix64((uint64_t)e * 256u + (uint64_t)k));
    return (int32_t)(z % (uint64_t)(2 * R + 1)) - R;
}

/* mean of x[t-m+1 .. t] (m = min(n, t + 1)), summed from the oldest */
static double win_mean(const double *x, int t, int n, int K, int k)
{
    const int t0 = t - n + 1 > 0 ? t - n + 1 : 0;
    double s = 0.0;
    for (int u = t0; u <= t; ++u) s += x[(int64_t)u * K + k];
    return s / (double)(t - t0 + 1);
}

/* The 8 technical indicators of Sec. 6.1 (textbook forms) from data up to
 * each day, stored scale-free as float32 ind[day][8][K]:
 *   MACD(12, 26) / c, (SMA20 + 2 sd20) / c - 1, (SMA20 - 2 sd20) / c - 1,
 *   RSI-30 / 100, CCI-30 / 100, DX-30 / 100, SMA30 / c - 1, SMA60 / c - 1.
 * In double: windows over up to n trailing days (shorter at the start),
 * summed from the oldest; sd population; EMA e_t = a c_t + (1 - a) e_{t-1},
 * a = 2 / (n + 1), e_0 = c_0; Wilder w_t = w_{t-1} + (x_t - w_{t-1}) / 30,
 * w_0 = x_0; RSI from Wilder gains / losses of c_t - c_{t-1} (100 without
 * losses, 50 without either); CCI = (tp - SMA30(tp)) / (0.015 MAD), tp =
 * (h + l + c) / 3, 0 when MAD = 0; DX = 100 |DI+ - DI-| / (DI+ + DI-) from
 * Wilder DM+ / DM- / TR (TR with c_{-1} = c_0), 0 when DI+ + DI- = 0. */
void orc_indicators(int32_t T, int32_t K, const int64_t *close, const int64_t *high, const int64_t *low,
                    float *ind)
{
    double *c = (double *)malloc(sizeof(double) * (size_t)T * K);
    double *tp = (double *)malloc(sizeof(double) * (size_t)T * K);
    for (int64_t i = 0; i < (int64_t)T * K; ++i) {
        c[i] = (double)close[i];
        tp[i] = ((double)high[i] + (double)low[i] + (double)close[i]) / 3.0;
    }
    for (int k = 0; k < K; ++k) {
        double e12 = c[k], e26 = c[k];
        const double a12 = 2.0 / 13.0, a26 = 2.0 / 27.0;
        double gain = 0.0, loss = 0.0, str = 0.0, spd = 0.0, snd = 0.0;
        for (int t = 0; t < T; ++t) {
            const double ct = c[(int64_t)t * K + k];
            const double ht = (double)high[(int64_t)t * K + k], lt = (double)low[(int64_t)t * K + k];
            const double cp = t > 0 ? c[(int64_t)(t - 1) * K + k] : ct;
            if (t > 0) {
                e12 = a12 * ct + (1.0 - a12) * e12;
                e26 = a26 * ct + (1.0 - a26) * e26;
            }
            const double d = ct - cp;
            const double g = d > 0.0 ? d : 0.0, l = d < 0.0 ? -d : 0.0;
            const double up = t > 0 ? ht - (double)high[(int64_t)(t - 1) * K + k] : 0.0;
            const double dn = t > 0 ? (double)low[(int64_t)(t - 1) * K + k] - lt : 0.0;
            const double pdm = (up > dn && up > 0.0) ? up : 0.0, ndm = (dn > up && dn > 0.0) ? dn : 0.0;
            double tr = ht - lt;
            if (fabs(ht - cp) > tr) tr = fabs(ht - cp);
            if (fabs(lt - cp) > tr) tr = fabs(lt - cp);
            if (t == 0) {
                gain = g; loss = l; str = tr; spd = pdm; snd = ndm;
            } else {
                gain = gain + (g - gain) / 30.0;
                loss = loss + (l - loss) / 30.0;
                str = str + (tr - str) / 30.0;
                spd = spd + (pdm - spd) / 30.0;
                snd = snd + (ndm - snd) / 30.0;
            }
            const double rsi = (gain == 0.0 && loss == 0.0) ? 50.0
                               : (loss > 0.0 ? 100.0 - 100.0 / (1.0 + gain / loss) : 100.0);
            const double sma20 = win_mean(c, t, 20, K, k);
            const int t20 = t - 19 > 0 ? t - 19 : 0;
            double v20 = 0.0;
            for (int u = t20; u <= t; ++u) {
                const double z = c[(int64_t)u * K + k] - sma20;
                v20 += z * z;
            }
            const double sd20 = sqrt(v20 / (double)(t - t20 + 1));
            const double smatp = win_mean(tp, t, 30, K, k);
            const int t30 = t - 29 > 0 ? t - 29 : 0;
            double mad = 0.0;
            for (int u = t30; u <= t; ++u) mad += fabs(tp[(int64_t)u * K + k] - smatp);
            mad = mad / (double)(t - t30 + 1);
            const double cci = mad > 0.0 ? (tp[(int64_t)t * K + k] - smatp) / (0.015 * mad) : 0.0;
            const double pdi = 100.0 * spd / (str > 0.0 ? str : 1.0), ndi = 100.0 * snd / (str > 0.0 ? str : 1.0);
            const double dx = pdi + ndi > 0.0 ? 100.0 * fabs(pdi - ndi) / (pdi + ndi) : 0.0;
            const double sma30 = win_mean(c, t, 30, K, k), sma60 = win_mean(c, t, 60, K, k);
            float *o = ind + (int64_t)t * 8 * K + k;
            o[0 * K] = (float)((e12 - e26) / ct);
            o[1 * K] = (float)((sma20 + 2.0 * sd20) / ct - 1.0);
            o[2 * K] = (float)((sma20 - 2.0 * sd20) / ct - 1.0);
            o[3 * K] = (float)(rsi / 100.0);
            o[4 * K] = (float)(cci / 100.0);
            o[5 * K] = (float)(dx / 100.0);
            o[6 * K] = (float)(sma30 / ct - 1.0);
            o[7 * K] = (float)(sma60 / ct - 1.0);
        }
    }
    free(c);
    free(tp);
}

/* ----------------------------------------------------------- episode metrics */

typedef struct {
    int64_t n;       /* periods seen */
    double mu, m2;   /* Welford running mean / sum of squared deviations */
    int64_t v0;      /* value at reset */
    int64_t peak;    /* running maximum of the value */
    double mdd;      /* running min of v / peak - 1 (<= 0) */
    int64_t vlast;   /* latest value */
} orc_acc;

static void acc_reset(orc_acc *a, int64_t v0)
{
    a->n = 0; a->mu = 0.0; a->m2 = 0.0;
    a->v0 = v0; a->peak = v0; a->mdd = 0.0; a->vlast = v0;
}

/* One period: rho = v1 / v0 - 1, Welford update, running peak and drawdown. */
static void acc_push(orc_acc *a, int64_t vprev, int64_t v1)
{
    double rho = (double)v1 / (double)vprev - 1.0;
    a->n += 1;
    double delta = rho - a->mu;
    a->mu += delta / (double)a->n;
    a->m2 += delta * (rho - a->mu);
    if (v1 > a->peak) a->peak = v1;
    double dd = (double)v1 / (double)a->peak - 1.0;
    if (dd < a->mdd) a->mdd = dd;
    a->vlast = v1;
}

/* out = {cumulative return, Sharpe, maximum drawdown}.
 * Sharpe (Sec. 5.2.1) = (mean - r_f) / std * sqrt(A), ddof 1, r_f = 0;
 * 0 when fewer than two periods or zero variance. */
static void acc_final(const orc_acc *a, double ann, double *out)
{
    out[0] = (double)a->vlast / (double)a->v0 - 1.0;
    double sharpe = 0.0;
    if (a->n >= 2 && a->m2 != 0.0) {
        double sd = sqrt(a->m2 / (double)(a->n - 1));
        sharpe = (a->mu - 0.0) / sd * sqrt(ann);
    }
    out[1] = sharpe;
    out[2] = a->mdd;
}

/* Metrics of a plain value series v[0..n-1] (v[0] = value at reset). */
void orc_metrics_series(int32_t n, const int64_t *v, double ann, double *out)
{
    orc_acc a;
    acc_reset(&a, v[0]);
    for (int i = 1; i < n; ++i) acc_push(&a, v[i - 1], v[i]);
    acc_final(&a, ann, out);
}

/* Sec. 6.1 metric list and Sec. 4.3 discounted trajectory return, from a
 * stored trajectory: rew[T][N] int64 rewards (v_t - v_{t-1}), done[T][N] (or
 * NULL); env i's periods are its rows up to and including its first done row
 * (all T rows when it has none), its values v_0 = v0, v_t = v_{t-1} + rew.
 * out[N][11]:
 *   0 cumulative return v_n / v_0 - 1      1 Sharpe (as the episode metrics)
 *   2 maximum drawdown (<= 0)               3 annual return (v_n/v_0)^(A/n) - 1
 *   4 annual volatility sd * sqrt(A)        5 RoMaD = cumulative return / |MDD|
 *   6 Sortino = mean / DD * sqrt(A), DD = sqrt(sum min(rho, 0)^2 / n)
 *   7 Calmar = annual return / |MDD|
 *   8 Omega = sum max(rho, 0) / sum max(-rho, 0) (threshold return 0)
 *   9 discounted return sum_{t=1..n} gamma^t r_t (cents)   10 n
 * with r_f = 0, sd with ddof 1 (0 below two periods), and every ratio whose
 * denominator is 0 reported as 0. */
void orc_trajectory_metrics(int32_t T, int32_t N, const int64_t *rew, const uint8_t *done,
                            int64_t v0, double ann, double gamma, double *out)
{
    for (int i = 0; i < N; ++i) {
        orc_acc a;
        acc_reset(&a, v0);
        double down2 = 0.0, up = 0.0, dn = 0.0, disc = 0.0, g = 1.0;
        int64_t v = v0;
        for (int t = 0; t < T; ++t) {
            const int64_t r = rew[(int64_t)t * N + i];
            const int64_t v1 = v + r;
            const double rho = (double)v1 / (double)v - 1.0;
            acc_push(&a, v, v1);
            if (rho < 0.0) {
                down2 += rho * rho;
                dn += -rho;
            } else {
                up += rho;
            }
            g *= gamma;
            disc += g * (double)r;
            v = v1;
            if (done && done[(int64_t)t * N + i]) break;
        }
        double *o = out + (int64_t)i * 11;
        acc_final(&a, ann, o);
        const double n = (double)a.n;
        const double cr = o[0], mdd = -o[2];
        o[3] = a.n > 0 ? pow((double)a.vlast / (double)a.v0, ann / n) - 1.0 : 0.0;
        o[4] = a.n >= 2 ? sqrt(a.m2 / (n - 1.0)) * sqrt(ann) : 0.0;
        o[5] = mdd != 0.0 ? cr / mdd : 0.0;
        const double dd = a.n > 0 ? sqrt(down2 / n) : 0.0;
        o[6] = dd != 0.0 ? a.mu / dd * sqrt(ann) : 0.0;
        o[7] = mdd != 0.0 ? o[3] / mdd : 0.0;
        o[8] = dn != 0.0 ? up / dn : 0.0;
        o[9] = disc;
        o[10] = n;
    }
}

/* ------------------------------------------------------------ stock task */

typedef struct {
    int64_t cash;
    int32_t *h;     /* [K] */
    int32_t t;      /* steps taken in this episode */
    uint8_t done;
    orc_acc acc;
} stock_env;

static void stock_prices(const int64_t *close, const int16_t *bps, int K,
                         int Ke, int d, int64_t *p)
{
    for (int k = 0; k < K; ++k)
        p[k] = k < Ke ? orc_perturb(close[(int64_t)d * K + k], bps ? bps[k] : 0) : 0;
}

static int64_t stock_value(int64_t cash, const int32_t *h, const int64_t *p, int Ke)
{
    int64_t v = cash;
    for (int k = 0; k < Ke; ++k) v += p[k] * (int64_t)h[k];
    return v;
}

/* Sec. 3.1 state [b, p, h, f]: cash*1e-8, p*1e-4, h*1e-2, indicators
 * indicator-major (i outer, asset inner); assets k >= Ke are zero.  Each
 * scaled entry is the float32 product of the value rounded to float32 and
 * the float32 constant. */
static void stock_obs(const stock_env *e, const int64_t *p, const float *ind,
                      int K, int I, int Ke, int d, float *o)
{
    o[0] = (float)e->cash * 1e-8f;
    for (int k = 0; k < K; ++k) {
        o[1 + k] = k < Ke ? (float)p[k] * 1e-4f : 0.0f;
        o[1 + K + k] = k < Ke ? (float)e->h[k] * 1e-2f : 0.0f;
    }
    for (int i = 0; i < I; ++i)
        for (int k = 0; k < K; ++k)
            o[1 + 2 * K + i * K + k] =
                k < Ke ? ind[((int64_t)d * I + i) * K + k] : 0.0f;
}

static void stock_reset(stock_env *e, int K, int64_t init_cash)
{
    e->cash = init_cash;
    for (int k = 0; k < K; ++k) e->h[k] = 0;
    e->t = 0;
    e->done = 0;
    acc_reset(&e->acc, init_cash);
}

/* Execute integer share changes q[0..Ke) at prices p: sells first (capped at
 * holdings), then greedy buys under the cash, in ascending asset order
 * (buy_order 0) or largest requested count first with ties in ascending
 * asset order (buy_order 1); each buy fills as far as the cash allows. */
static void stock_trade(stock_env *e, const int32_t *q, const int64_t *p,
                        int Ke, int32_t fee_bps, int32_t buy_order)
{
    int order[Ke];
    for (int k = 0; k < Ke; ++k) order[k] = k;
    if (buy_order == 1) {
        /* stable insertion sort by decreasing q: equal counts keep their
         * ascending asset order */
        for (int i = 1; i < Ke; ++i) {
            const int k = order[i];
            int j = i;
            while (j > 0 && q[order[j - 1]] < q[k]) {
                order[j] = order[j - 1];
                --j;
            }
            order[j] = k;
        }
    }
    for (int k = 0; k < Ke; ++k) {
        if (q[k] < 0) {
            int64_t n = -(int64_t)q[k];
            if (n > e->h[k]) n = e->h[k];
            int64_t g = n * p[k];
            e->h[k] -= (int32_t)n;
            e->cash += g - orc_fee(g, fee_bps);
        }
    }
    for (int i = 0; i < Ke; ++i) {
        const int k = order[i];
        if (q[k] > 0) {
            int64_t n0 = orc_buy_max(e->cash, p[k], fee_bps);
            int64_t n = q[k] < n0 ? q[k] : n0;
            if (n > 0) {
                e->h[k] += (int32_t)n;
                e->cash -= orc_buy_cost(n, p[k], fee_bps);
            }
        }
    }
}

/*
 * Run T steps of N stock environments from reset.
 *
 * Market: close[n_days][K] (int64 cents), ind[n_days][I][K] (float32).
 * Env e trades its first Ke[e] assets over the window start[e] ..
 * start[e] + W[e] - 1 (W[e] days, W[e] - 1 steps), with per-asset basis-point
 * perturbation bps[e][K] (NULL = none).
 *
 * mode 0: prescribed integer share changes act_i32[T][N][K];
 * mode 1: prescribed unit actions act_f32[T][N][K] in [-1,1];
 * mode 2: ensemble of M actors (L layers, dims[L+1], params[M][P]) with
 *         weights wts[M] (NULL = uniform) combined as orc_ensemble_mean.
 *
 * Outputs (any may be NULL): obs[T][N][D] with D = 1 + 2K + I K (the
 * observation the step acted on), act[T][N][K] (combined action, mode 2 only),
 * q[T][N][K] (executed share orders before caps), rew[T][N], rew_f32[T][N],
 * done[T][N], cash[T][N] and hold[T][N][K] after the step, metrics[N][3]
 * (cumulative return, Sharpe with A = 252, MDD) after the last step.
 * buy_order: 0 ascending asset order, 1 largest requested count first
 * (see stock_trade).
 */
int32_t orc_stock_run(int32_t n_days, int32_t K, int32_t I,
                      const int64_t *close, const float *ind,
                      int32_t N, const int32_t *Ke, const int32_t *start,
                      const int32_t *W, const int16_t *bps,
                      int64_t init_cash, int32_t hmax, int32_t fee_bps,
                      int32_t auto_reset, int32_t T, int32_t mode,
                      const int32_t *act_i32, const float *act_f32,
                      int32_t M, int32_t L, const int32_t *dims,
                      const float *params, const double *wts,
                      float *obs, double *act_out, int32_t *q_out,
                      int64_t *rew, float *rew_f32, uint8_t *done_out,
                      int64_t *cash_out, int32_t *hold_out, double *metrics,
                      int32_t nthreads, int32_t buy_order)
{
    const int D = 1 + 2 * K + I * K;
    if (buy_order != 0 && buy_order != 1) return -3;
    for (int e = 0; e < N; ++e) {
        if (Ke[e] < 1 || Ke[e] > K || W[e] < 2 || start[e] < 0 ||
            start[e] + W[e] > n_days)
            return -1;
    }
    if (mode == 2 && (dims[0] != D || dims[L] != K)) return -2;
    const int64_t P = mode == 2 ? net_param_count(L, dims) : 0;
    const int wmax = mode == 2 ? max_width(L, dims) : 1;

#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        int32_t *h = (int32_t *)malloc(sizeof(int32_t) * K);
        int64_t *p = (int64_t *)malloc(sizeof(int64_t) * K);
        int64_t *p1 = (int64_t *)malloc(sizeof(int64_t) * K);
        int32_t *q = (int32_t *)malloc(sizeof(int32_t) * K);
        float *o = (float *)malloc(sizeof(float) * D);
        double *ya = (double *)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1) * K);
        double *a = (double *)malloc(sizeof(double) * K);
        double *ba = (double *)malloc(sizeof(double) * wmax);
        double *bb = (double *)malloc(sizeof(double) * wmax);

#pragma omp for schedule(dynamic, 1)
        for (int e = 0; e < N; ++e) {
            stock_env env;
            env.h = h;
            stock_reset(&env, K, init_cash);
            const int16_t *eb = bps ? bps + (int64_t)e * K : NULL;
            const int ke = Ke[e];
            for (int t = 0; t < T; ++t) {
                const int64_t row = (int64_t)t * N + e;
                int d = start[e] + env.t;
                stock_prices(close, eb, K, ke, d, p);
                stock_obs(&env, p, ind, K, I, ke, d, o);
                if (obs) memcpy(obs + row * D, o, sizeof(float) * D);
                /* the action the step receives */
                for (int k = 0; k < K; ++k) q[k] = 0;
                if (mode == 0) {
                    for (int k = 0; k < ke; ++k) q[k] = act_i32[row * K + k];
                } else if (mode == 1) {
                    for (int k = 0; k < ke; ++k)
                        q[k] = orc_discretise((double)act_f32[row * K + k], hmax);
                } else {
                    for (int j = 0; j < M; ++j)
                        net_forward_row(L, dims, params + (int64_t)j * P, 1, o,
                                        ya + (int64_t)j * K, ba, bb);
                    orc_ensemble_mean(M, K, ya, wts, a);
                    if (act_out) memcpy(act_out + row * K, a, sizeof(double) * K);
                    for (int k = 0; k < ke; ++k) q[k] = orc_discretise(a[k], hmax);
                }
                if (q_out) memcpy(q_out + row * K, q, sizeof(int32_t) * K);

                int64_t r = 0;
                uint8_t dn;
                if (env.done) {                      /* frozen after its window */
                    dn = 1;
                } else {
                    int64_t v0 = stock_value(env.cash, env.h, p, ke);
                    stock_trade(&env, q, p, ke, fee_bps, buy_order);
                    env.t += 1;
                    stock_prices(close, eb, K, ke, d + 1, p1);
                    int64_t v1 = stock_value(env.cash, env.h, p1, ke);
                    r = v1 - v0;
                    acc_push(&env.acc, v0, v1);
                    dn = env.t == W[e] - 1;
                    env.done = dn;
                }
                if (rew) rew[row] = r;
                if (rew_f32) rew_f32[row] = (float)r * 1e-6f;
                if (done_out) done_out[row] = dn;
                if (dn && auto_reset) {
                    if (metrics) acc_final(&env.acc, 252.0, metrics + (int64_t)e * 3);
                    stock_reset(&env, K, init_cash);
                }
                if (cash_out) cash_out[row] = env.cash;
                if (hold_out) memcpy(hold_out + row * K, env.h, sizeof(int32_t) * K);
            }
            if (metrics && !(auto_reset && env.t == 0 && T > 0))
                acc_final(&env.acc, 252.0, metrics + (int64_t)e * 3);
        }
        free(h); free(p); free(p1); free(q); free(o); free(ya); free(a);
        free(ba); free(bb);
    }
    return 0;
}

/* ----------------------------------------------------------- crypto task */

/*
 * Run T steps of N single-asset crypto environments from reset.
 *
 * Market: mid[S] (int64 cents per lot), spread[S] (cents, 1..5),
 * fac[S][8] (float32).  Env e covers seconds start[e] .. start[e]+W[e]-1.
 * Observation (Sec. 3.1 with K = 1, factors in place of indicators):
 *   [cash*1e-8, pos/pmax, fac_0..fac_7].
 * Action u in {0 sell, 1 hold, 2 buy} of one lot: buy at ask = bid + s when
 * pos < pmax and cash >= ask; sell at bid = mid - s/2 when pos > 0; no fee.
 * Value = cash + pos * mid.
 *
 * mode 0: prescribed act_u8[T][N] (values > 2 hold);
 * mode 2: M Q-networks, per-agent argmax, majority vote (Sec. 5.2.2).
 * Outputs (NULL allowed): obs[T][N][10], act_out[T][N] (executed action),
 * agent_act[T][N][M] (mode 2), rew, rew_f32, done, cash, pos per step, and
 * metrics[N][3] with A = 1.
 */
int32_t orc_crypto_run(int32_t S, const int64_t *mid, const uint8_t *spread,
                       const float *fac, int32_t N, const int32_t *start,
                       const int32_t *W, int64_t init_cash, int32_t pmax,
                       int32_t auto_reset, int32_t T, int32_t mode,
                       const uint8_t *act_u8, int32_t M, int32_t L,
                       const int32_t *dims, const float *params,
                       float *obs, uint8_t *act_out, uint8_t *agent_act,
                       int64_t *rew, float *rew_f32, uint8_t *done_out,
                       int64_t *cash_out, int32_t *pos_out, double *metrics,
                       int32_t nthreads)
{
    const int D = 10;
    for (int e = 0; e < N; ++e)
        if (W[e] < 2 || start[e] < 0 || start[e] + W[e] > S) return -1;
    if (pmax < 1) return -1;
    if (mode == 2 && (dims[0] != D || dims[L] != 3 || M > 255)) return -2;
    const int64_t P = mode == 2 ? net_param_count(L, dims) : 0;
    const int wmax = mode == 2 ? max_width(L, dims) : 1;

#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        float o[10];
        double qv[3];
        uint8_t *ballots = (uint8_t *)malloc((size_t)(M > 0 ? M : 1));
        double *ba = (double *)malloc(sizeof(double) * wmax);
        double *bb = (double *)malloc(sizeof(double) * wmax);
#pragma omp for schedule(dynamic, 1)
        for (int e = 0; e < N; ++e) {
            int64_t cash = init_cash;
            int32_t pos = 0, tt = 0;
            uint8_t done = 0;
            orc_acc acc;
            acc_reset(&acc, init_cash);
            for (int t = 0; t < T; ++t) {
                const int64_t row = (int64_t)t * N + e;
                int d = start[e] + tt;
                o[0] = (float)cash * 1e-8f;
                o[1] = (float)pos / (float)pmax;
                for (int i = 0; i < 8; ++i) o[2 + i] = fac[(int64_t)d * 8 + i];
                if (obs) memcpy(obs + row * D, o, sizeof(o));
                int u = 1;
                if (mode == 0) {
                    u = act_u8[row];
                    if (u > 2) u = 1;
                } else {
                    for (int j = 0; j < M; ++j) {
                        net_forward_row(L, dims, params + (int64_t)j * P, 0, o, qv, ba, bb);
                        ballots[j] = (uint8_t)orc_argmax(qv, 3);
                        if (agent_act) agent_act[row * M + j] = ballots[j];
                    }
                    u = orc_vote(M, ballots);
                }
                if (act_out) act_out[row] = (uint8_t)u;
                int64_t r = 0;
                uint8_t dn;
                if (done) {
                    dn = 1;
                } else {
                    int64_t m0 = mid[d];
                    int64_t v0 = cash + (int64_t)pos * m0;
                    int64_t s = spread[d];
                    int64_t bid = m0 - s / 2, ask = bid + s;
                    if (u == 2 && pos < pmax && cash >= ask) { pos += 1; cash -= ask; }
                    else if (u == 0 && pos > 0) { pos -= 1; cash += bid; }
                    tt += 1;
                    int64_t v1 = cash + (int64_t)pos * mid[d + 1];
                    r = v1 - v0;
                    acc_push(&acc, v0, v1);
                    dn = tt == W[e] - 1;
                    done = dn;
                }
                if (rew) rew[row] = r;
                if (rew_f32) rew_f32[row] = (float)r * 1e-6f;
                if (done_out) done_out[row] = dn;
                if (dn && auto_reset) {
                    if (metrics) acc_final(&acc, 1.0, metrics + (int64_t)e * 3);
                    cash = init_cash; pos = 0; tt = 0; done = 0;
                    acc_reset(&acc, init_cash);
                }
                if (cash_out) cash_out[row] = cash;
                if (pos_out) pos_out[row] = pos;
            }
            if (metrics && !(auto_reset && tt == 0 && T > 0))
                acc_final(&acc, 1.0, metrics + (int64_t)e * 3);
        }
        free(ballots); free(ba); free(bb);
    }
    return 0;
}

/* ---------------------------------------------- vectorised helpers (tests) */

void orc_discretise_many(const float *a, int64_t n, int32_t hmax, int32_t *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_discretise((double)a[i], hmax);
}

void orc_buy_max_many(const int64_t *cash, const int64_t *p, const int32_t *fee,
                      int64_t n, int64_t *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_buy_max(cash[i], p[i], fee[i]);
}

void orc_perturb_many(const int64_t *close, const int32_t *bps, int64_t n,
                      int64_t *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_perturb(close[i], bps[i]);
}

int32_t orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
