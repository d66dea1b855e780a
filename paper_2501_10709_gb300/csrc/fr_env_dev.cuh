// fr_env_dev.cuh -- device-side accounting of the trading MDP (Sec. 3.1):
// integer-cent prices with the Sec. 5.1 per-asset perturbation, sells then
// greedy buys with a rounded-up fee (Sec. 3.2 transaction costs), the
// total-asset value v = b + p^T h and the reward v_{t+1} - v_t, and the FP64
// episode accumulators behind the Sharpe ratio (Sec. 5.2.1) and the maximum
// drawdown (Sec. 6.1).  Every floating-point step uses an explicitly rounded
// intrinsic so that no FMA contraction changes a result.
#pragma once

#include "fr_common.cuh"

namespace fr {

constexpr unsigned FULL_MASK = 0xffffffffu;

// Per-asset price after the basis-point change, rounded half up, >= 1 cent.
// close >= 1 (checked at market creation) and bps >= -100, so the numerator
// is positive and the division is done unsigned (fewer instructions than the
// signed one, same quotient).
__device__ __forceinline__ int64_t perturb(int64_t close, int bps)
{
    const uint64_t num = (uint64_t)close * (uint64_t)(BPS_ONE + bps) + (uint64_t)(BPS_ONE / 2);
    const int64_t p = (int64_t)(num / (uint64_t)BPS_ONE);
    return p < 1 ? 1 : p;
}

// The same three rules in 32-bit unsigned arithmetic, exact when the caller
// has proven that every intermediate fits (EnvView::narrow): the same
// quotients and sums, far fewer instructions than the 64-bit forms.
__device__ __forceinline__ uint32_t perturb32(uint32_t close, int bps)
{
    const uint32_t num = close * (uint32_t)(BPS_ONE + bps) + (uint32_t)(BPS_ONE / 2);
    const uint32_t p = num / (uint32_t)BPS_ONE;
    return p < 1u ? 1u : p;
}

__device__ __forceinline__ uint32_t fee_of32(uint32_t g, int fee_bps)
{
    return (g * (uint32_t)fee_bps + (uint32_t)(BPS_ONE - 1)) / (uint32_t)BPS_ONE;
}

__device__ __forceinline__ uint32_t cost_of32(uint32_t n, uint32_t p, int fee_bps)
{
    const uint32_t g = n * p;
    return g + fee_of32(g, fee_bps);
}

// ceil(g * fee_bps / 1e4) for g >= 0, fee_bps >= 0 (unsigned division)
__device__ __forceinline__ int64_t fee_of(int64_t g, int fee_bps)
{
    return (int64_t)(((uint64_t)g * (uint64_t)fee_bps + (uint64_t)(BPS_ONE - 1)) / (uint64_t)BPS_ONE);
}

__device__ __forceinline__ int64_t cost_of(int64_t n, int64_t p, int fee_bps)
{
    const int64_t g = n * p;
    return g + fee_of(g, fee_bps);
}

// Largest n with cost_of(n) <= c, for c >= 0, when the caller knows the
// answer is small (below the order it could not fully fill).  The quotient
// floor(c*1e4 / (p*(1e4+fee))) is estimated in fp32 and corrected exactly
// with integer products; the correction loops are bounded because the
// estimate is within one of the true quotient for quotients below 2^20.
__device__ __forceinline__ int64_t afford(int64_t c, int64_t p, int fee_bps)
{
    if (c <= 0) return 0;
    const int64_t X = c * BPS_ONE;
    const int64_t Dn = p * (int64_t)(BPS_ONE + fee_bps);
    int64_t n = (int64_t)__fdiv_rn((float)X, (float)Dn);
#pragma unroll 1
    for (int i = 0; i < 8 && n > 0 && n * Dn > X; ++i) --n;
#pragma unroll 1
    for (int i = 0; i < 8 && (n + 1) * Dn <= X; ++i) ++n;
    if (n > 0 && cost_of(n, p, fee_bps) > c) --n;
    return n;
}

// afford() for an order whose full cost fits 32 bits (EnvView::narrow): the
// largest n < want with cost_of32(n) <= c, given c below cost_of32(want).
// With D = p (1 + fee/1e4), cost_of32(n) lies in [n D, n D + 1) and D >= 1,
// so the answer is floor(c / D) or one less.  The fp32 quotient q is within
// 2^-21 relative of c / D, i.e. within one of it below 2^20 (hmax <= 1e6
// keeps every answer there), so trunc(q) exceeds the answer by -1 to 2: two
// conditional decrements and one conditional increment, all exact 32-bit
// comparisons of costs at most cost_of32(want), settle it without branches.
__device__ __forceinline__ uint32_t afford32(uint32_t c, uint32_t p, int fee_bps, uint32_t want)
{
    const float q = __fdividef((float)c, __fmul_rn((float)p, __fmaf_rn((float)fee_bps, 1e-4f, 1.0f)));
    uint32_t n = min((uint32_t)fminf(fmaxf(q, 0.0f), 1048576.0f), want - 1u);
    n -= (n > 0u && cost_of32(n, p, fee_bps) > c) ? 1u : 0u;
    n -= (n > 0u && cost_of32(n, p, fee_bps) > c) ? 1u : 0u;
    n += (n + 1u < want && cost_of32(n + 1u, p, fee_bps) <= c) ? 1u : 0u;
    return n;
}

// Action in [-1,1] -> share change trunc(a * hmax).  __fmul_rz keeps the
// product on the zero side of the exact value and integers up to hmax are
// representable, so the truncation equals that of the exact product.
__device__ __forceinline__ int32_t discretise(float a, int hmax, bool &bad)
{
    bad = !isfinite(a);
    if (bad) a = 0.0f;
    a = fminf(fmaxf(a, -1.0f), 1.0f);
    return (int32_t)__fmul_rz(a, (float)hmax);
}

__device__ __forceinline__ int64_t warp_sum(int64_t x)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(FULL_MASK, x, o);
    return x;
}

// Exact int64 warp sum (mod 2^64, like the serial sum) from three 32-bit
// hardware reductions: x = hi 2^42 + mid 2^21 + lo with lo, mid in [0, 2^21)
// and hi in [-2^21, 2^21), so none of the 32-lane partial sums overflows.
// The three reductions are independent, unlike the five dependent shuffle
// rounds of a butterfly sum.
__device__ __forceinline__ int64_t warp_sum_redux(int64_t x)
{
    const unsigned lo = (unsigned)x & 0x1fffffu;
    const unsigned mid = (unsigned)(x >> 21) & 0x1fffffu;
    const int hi = (int)(x >> 42);
    const unsigned slo = __reduce_add_sync(FULL_MASK, lo);
    const unsigned smid = __reduce_add_sync(FULL_MASK, mid);
    const int shi = __reduce_add_sync(FULL_MASK, hi);
    return (int64_t)(((uint64_t)(int64_t)shi << 42) + ((uint64_t)smid << 21) + (uint64_t)slo);
}

__device__ __forceinline__ int64_t warp_incl_scan(int64_t x, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// int64 -> float32, round to nearest.  Values that fit in 32 bits take the
// 32-bit conversion (the 64-bit one is a slow path on this GPU); both give
// the same correctly rounded result.
__device__ __forceinline__ float ll2f(int64_t x)
{
    return (x >= INT32_MIN && x <= INT32_MAX) ? __int2float_rn((int)x) : __ll2float_rn(x);
}

// Observation / learner scaling: the value rounded to float32 times a
// float32 constant, one rounding each, no FP64 on the step path.
__device__ __forceinline__ float obs_scale(int64_t x, float c)
{
    return __fmul_rn(ll2f(x), c);
}

__device__ __forceinline__ float reward_f32(int64_t r)
{
    return __fmul_rn(ll2f(r), 1e-6f);
}

// ---------------------------------------------------- FP64 episode metrics
// One period: rho = v1/v0 - 1, Welford mean / sum of squared deviations,
// running peak and drawdown min(v/peak - 1).  n is the period count after
// this one.
__device__ __forceinline__ void acc_push(double &mu, double &m2, double &mdd,
                                         int64_t &peak, int64_t &vlast, int n,
                                         int64_t v0, int64_t v1)
{
    const double rho = __dsub_rn(__ddiv_rn((double)v1, (double)v0), 1.0);
    const double delta = __dsub_rn(rho, mu);
    mu = __dadd_rn(mu, __ddiv_rn(delta, (double)n));
    m2 = __dadd_rn(m2, __dmul_rn(delta, __dsub_rn(rho, mu)));
    if (v1 > peak) peak = v1;
    // at a new peak the drawdown is exactly 0 and cannot lower mdd (<= 0):
    // the division is needed only below the peak
    if (v1 < peak) {
        const double dd = __dsub_rn(__ddiv_rn((double)v1, (double)peak), 1.0);
        if (dd < mdd) mdd = dd;
    }
    vlast = v1;
}

// {cumulative return, Sharpe = (mu - r_f) / sd * sqrt(A), max drawdown}
__device__ __forceinline__ void acc_final(double mu, double m2, double mdd,
                                          int64_t vlast, int64_t v0, int n,
                                          double ann, double *out)
{
    out[0] = __dsub_rn(__ddiv_rn((double)vlast, (double)v0), 1.0);
    double sh = 0.0;
    if (n >= 2 && m2 != 0.0) {
        const double sd = __dsqrt_rn(__ddiv_rn(m2, (double)(n - 1)));
        sh = __dmul_rn(__ddiv_rn(__dsub_rn(mu, 0.0), sd), __dsqrt_rn(ann));
    }
    out[1] = sh;
    out[2] = mdd;
}

// Episode bookkeeping after a step of env e (one thread): stores the new
// accumulators, or -- when the window is finished and auto_reset is on --
// latches the finished episode's metrics and restarts the env.
__device__ __forceinline__ void finish_step(const EnvView &v, int e, int64_t cash,
                                            int t1, bool done, int64_t v0, int64_t v1)
{
    double mu = v.mu[e], m2 = v.m2[e], mdd = v.mdd[e];
    int64_t peak = v.peak[e], vlast = v.vlast[e];
    acc_push(mu, m2, mdd, peak, vlast, t1, v0, v1);
    if (done && v.auto_reset) {
        double *L = v.latched + (int64_t)e * 4;
        acc_final(mu, m2, mdd, vlast, v.init_cash, t1, v.ann, L);
        L[3] = 1.0;
        v.cash[e] = v.init_cash;
        v.t[e] = 0;
        v.done[e] = 0;
        v.mu[e] = 0.0;
        v.m2[e] = 0.0;
        v.mdd[e] = 0.0;
        v.peak[e] = v.init_cash;
        v.vlast[e] = v.init_cash;
    } else {
        v.cash[e] = cash;
        v.t[e] = t1;
        v.done[e] = done ? 1 : 0;
        v.mu[e] = mu;
        v.m2[e] = m2;
        v.mdd[e] = mdd;
        v.peak[e] = peak;
        v.vlast[e] = vlast;
    }
}

// ------------------------------------------------------------ stock, warp
// The episode bookkeeping a stock step leaves for finish_step: deferred so
// that one thread per env can run the FP64 updates of many envs in one warp
// instruction (the FP64 pipe is narrow on this GPU).
struct StepFin {
    int64_t cash, v0, v1;
    int t1;
    int done;
    int valid;                  // 0: the env was already done, nothing to finish
};

// Observation of stock env e's current state into o[0..D), lane = asset:
// [cash*1e-8, p_k*1e-4, h_k*1e-2, f_{i,k} indicator-major], zero beyond Ke.
__device__ __forceinline__ void stock_obs_warp(const EnvView &v, int e, int lane, float *o)
{
    const int K = v.K, I = v.I;
    const int Ke = v.Ke[e];
    const int d = v.start[e] + v.t[e];
    const bool act = lane < Ke;
    if (lane == 0) o[0] = obs_scale(v.cash[e], 1e-8f);
    if (lane < K) {
        float pv = 0.0f, hv = 0.0f;
        if (act) {
            const int64_t p = perturb(__ldg(v.close + (int64_t)d * K + lane),
                                      v.bps[(int64_t)e * KP + lane]);
            pv = obs_scale(p, 1e-4f);
            hv = obs_scale(v.hold[(int64_t)e * KP + lane], 1e-2f);
        }
        o[1 + lane] = pv;
        o[1 + K + lane] = hv;
        const float *f = v.ind + (int64_t)d * I * K;
        float *oi = o + 1 + 2 * K + lane;
        if (I == 8) {                                    // the usual count: every load in flight
            float fv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) fv[i] = act ? __ldg(f + i * K + lane) : 0.0f;
#pragma unroll
            for (int i = 0; i < 8; ++i) oi[i * K] = fv[i];
        } else {
            for (int i = 0; i < I; ++i) oi[i * K] = act ? __ldg(f + i * K + lane) : 0.0f;
        }
    }
}

// ---------------------------------------------------------- crypto, thread
// One step of crypto env e by one thread; u in {0 sell, 1 hold, 2 buy}.
__device__ __forceinline__ int64_t crypto_step_thread(const EnvView &v, int e, int u,
                                                      bool &done_out)
{
    if (v.done[e]) {
        done_out = true;
        return 0;
    }
    const int t0 = v.t[e];
    const int d = v.start[e] + t0;
    int64_t cash = v.cash[e];
    int pos = v.hold[e];
    const int64_t m0 = __ldg(v.mid + d);
    const int64_t s = (int64_t)__ldg(v.spread + d);
    const int64_t v0 = cash + (int64_t)pos * m0;
    const int64_t bid = m0 - s / 2, ask = bid + s;
    if (u == 2) {
        if (pos < v.pmax && cash >= ask) { pos += 1; cash -= ask; }
    } else if (u == 0) {
        if (pos > 0) { pos -= 1; cash += bid; }
    }
    const int t1 = t0 + 1;
    const int64_t v1 = cash + (int64_t)pos * __ldg(v.mid + d + 1);
    const bool done = t1 == v.W[e] - 1;
    v.hold[e] = (done && v.auto_reset) ? 0 : pos;
    finish_step(v, e, cash, t1, done, v0, v1);
    done_out = done;
    return v1 - v0;
}

// [cash*1e-8, pos/pmax, fac_0..7] of crypto env e's current state
__device__ __forceinline__ void crypto_obs_thread(const EnvView &v, int e, float *o)
{
    const int d = v.start[e] + v.t[e];
    o[0] = obs_scale(v.cash[e], 1e-8f);
    o[1] = __fdiv_rn(__int2float_rn(v.hold[e]), __int2float_rn(v.pmax));
    const float *f = v.fac + (int64_t)d * FR_CRYPTO_FACTORS;
#pragma unroll
    for (int i = 0; i < FR_CRYPTO_FACTORS; ++i) o[2 + i] = __ldg(f + i);
}

}  // namespace fr
