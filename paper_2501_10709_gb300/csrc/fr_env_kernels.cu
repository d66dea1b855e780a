// fr_env_kernels.cu -- the reset / step / reward operations of every SubEnv
// (Sec. 4.2.2), one launch over the whole VecEnv.  Stock envs are stepped by
// one warp per env (lane = asset, warp-shuffle int64 reductions for the
// total-asset value); crypto envs by one thread per env.
#include "fr_env_dev.cuh"

namespace fr {

namespace {

constexpr int kBlock = 256;
constexpr int kStepEnvs = 8;           // envs (warps) per block of the stock step kernel (<= 32)
constexpr int kStepBlocks = 8;          // its resident blocks per SM (register bound)

__global__ void k_env_reset(EnvView v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int hs = v.task == FR_TASK_STOCK ? KP : 1;
    if (i < (int64_t)v.N * hs) v.hold[i] = 0;
    if (i < v.N) {
        const int e = (int)i;
        v.cash[e] = v.init_cash;
        v.t[e] = 0;
        v.done[e] = 0;
        v.mu[e] = 0.0;
        v.m2[e] = 0.0;
        v.mdd[e] = 0.0;
        v.peak[e] = v.init_cash;
        v.vlast[e] = v.init_cash;
        v.latched[(int64_t)e * 4 + 0] = 0.0;
        v.latched[(int64_t)e * 4 + 1] = 0.0;
        v.latched[(int64_t)e * 4 + 2] = 0.0;
        v.latched[(int64_t)e * 4 + 3] = 0.0;
    }
}

// One warp per env (lane = asset): every independent load is issued first,
// then sells (capped at the holding), greedy buys in ascending asset order
// (one sum settles them when every order fits; otherwise rounds that drop
// the assets that cannot afford one share, fill every order in full up to the
// first whose prefix cost exceeds the cash, fill that one as far as the cash
// allows and continue after it), the value at the next day's prices and the
// next observation from registers.  BYSIZE: the buys execute largest
// requested count first (equal counts in ascending asset order): when not
// every order fits, the orders are moved to the lanes of their execution
// positions, filled by the same rounds, and the fills moved back.
// The FP64 episode bookkeeping is deferred: the last warp of the block to
// finish runs it for all the block's envs, one thread per env, so that one
// instruction of the narrow FP64 pipe serves several envs and no warp waits
// at a block barrier.  Blocks are small (8 envs, 8 blocks per SM at 32
// registers): measured at 1,048,576 envs, 879 us per step against 1,148 us
// with 32-env blocks (2 per SM), 945 us with 16-env and 979 us with 4-env
// blocks -- a block's slot is held until its slowest warp and its
// bookkeeping finish, and small blocks turn over sooner.
// NARROW: the prices, orders and a step's sums of sells and buys run in
// 32-bit arithmetic (env_create proved the ranges; same results).  FIXED:
// the market has K = 30 assets and I = 8 indicators (the paper's shape), so
// every row offset of the state, action, price and observation rows is a
// compile-time constant.
template <int KIND, bool BYSIZE, bool NARROW, bool FIXED>
__global__ void __launch_bounds__(kStepEnvs * 32, kStepBlocks) k_stock_step(EnvView v, const void *act, int64_t *rew,
                                                                float *rew_f32, uint8_t *done_out,
                                                                float *obs, int ld)
{
    static_assert(kStepEnvs <= 32, "one lane per env of the block in the bookkeeping warp");
    __shared__ StepFin fin_sm[kStepEnvs];
    __shared__ unsigned arrived;
    if (threadIdx.x == 0) arrived = 0u;
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int e = blockIdx.x * kStepEnvs + w;
    const int K = FIXED ? 30 : v.K;
    const int NI = FIXED ? 8 : v.I;
    StepFin fin;
    fin.valid = 0;
    if (e < v.N) {                                       // uniform per warp
        const bool was_done = v.done[e] != 0;
        const int Ke = v.Ke[e], t0 = v.t[e], start = v.start[e], W = v.W[e];
        const int64_t cash0 = v.cash[e];
        const bool live = lane < Ke;
        const int bps = lane < K ? (int)v.bps[(int64_t)e * KP + lane] : 0;
        int64_t h = live ? (int64_t)v.hold[(int64_t)e * KP + lane] : 0;
        int32_t q = 0;
        if (live) {
            if (KIND == FR_ACT_I32_SHARES) {
                q = ((const int32_t *)act)[(int64_t)e * K + lane];
            } else {
                bool bad;
                q = discretise(((const float *)act)[(int64_t)e * K + lane], v.hmax, bad);
                if (bad) atomicAdd(v.err, 1ull);
            }
        }
        const int d = start + t0;
        const int64_t c0 = live ? __ldg(v.close + (int64_t)d * K + lane) : 0;
        const int64_t c1 = (live && !was_done) ? __ldg(v.close + (int64_t)(d + 1) * K + lane) : 0;
        int64_t cash = cash0, r = 0;
        int t_obs = t0;
        bool dn = true;
        int64_t p_obs = live ? (NARROW ? (int64_t)perturb32((uint32_t)c0, bps) : perturb(c0, bps)) : 0;
        if (!was_done) {
            const int fee = v.fee_bps;
            const int64_t p = p_obs;
            // holdings are int32 >= 0 and prices below 2^32: one 32 x 32 -> 64-bit product
            const int64_t v0 = cash + warp_sum_redux(NARROW ? (int64_t)((uint64_t)(uint32_t)p * (uint32_t)h) : p * h);
            int64_t net = 0;
            uint32_t net32 = 0u;
            if (q < 0) {
                int64_t n = -(int64_t)q;
                if (n > h) n = h;
                h -= n;
                if (NARROW) {
                    const uint32_t g = (uint32_t)n * (uint32_t)p;
                    net32 = g - fee_of32(g, fee);
                } else {
                    const int64_t g = n * p;
                    net = g - fee_of(g, fee);
                }
            }
            cash += NARROW ? (int64_t)__reduce_add_sync(FULL_MASK, net32) : warp_sum_redux(net);
            const int64_t want = q > 0 ? (int64_t)q : 0;
            int64_t full = 0, nb = 0;
            if (want > 0) full = NARROW ? (int64_t)cost_of32((uint32_t)want, (uint32_t)p, fee) : cost_of(want, p, fee);
            unsigned pending = __ballot_sync(FULL_MASK, want > 0);
            const int64_t all = NARROW ? (int64_t)__reduce_add_sync(FULL_MASK, (uint32_t)full) : warp_sum_redux(full);
            if (all <= cash) {
                nb = want;
                cash -= all;
                pending = 0u;
            }
            int rank = lane;                     // execution position of this lane's order
            // the one-share cost only matters when not every order fits
            const int64_t one = pending && want > 0
                                    ? (NARROW ? (int64_t)cost_of32(1u, (uint32_t)p, fee) : cost_of(1, p, fee))
                                    : 0;
            int64_t bw = want, bf = full, bo = one, bp = p;
            if (BYSIZE && pending) {
                // rank: orders with a larger count, or an equal count at a
                // lower asset index, go first (a permutation of 0..31: the
                // lanes without a buy follow in lane order)
                rank = 0;
#pragma unroll 1
                for (int j = 0; j < 32; ++j) {
                    const int64_t wj = __shfl_sync(FULL_MASK, want, j);
                    rank += (wj > want || (wj == want && j < lane)) ? 1 : 0;
                }
                int src = 0;                     // the lane whose order executes at position `lane`
#pragma unroll 1
                for (int j = 0; j < 32; ++j)
                    if (__shfl_sync(FULL_MASK, rank, j) == lane) src = j;
                bw = __shfl_sync(FULL_MASK, want, src);
                bf = __shfl_sync(FULL_MASK, full, src);
                bo = __shfl_sync(FULL_MASK, one, src);
                bp = __shfl_sync(FULL_MASK, p, src);
                pending = __ballot_sync(FULL_MASK, bw > 0);
            }
            int64_t bn = nb;                     // fill at this lane's position
#pragma unroll 1
            while (pending) {
                bool mine = (pending >> lane) & 1u;
                pending &= ~__ballot_sync(FULL_MASK, mine && bo > cash);
                if (!pending) break;
                mine = (pending >> lane) & 1u;
                const int64_t x = mine ? bf : 0;
                int64_t pre;
                if (NARROW) {
                    // every order's cost and their sum fit 32 bits
                    uint32_t y = (uint32_t)x;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t z = __shfl_up_sync(FULL_MASK, y, o);
                        y += lane >= o ? z : 0u;
                    }
                    pre = (int64_t)y;
                } else {
                    pre = warp_incl_scan(x, lane);
                }
                const unsigned fail = __ballot_sync(FULL_MASK, mine && pre > cash);
                if (fail == 0u) {
                    if (mine) bn = bw;
                    cash -= __shfl_sync(FULL_MASK, pre, 31);
                    break;
                }
                const int f = __ffs(fail) - 1;
                if (mine && lane < f) bn = bw;
                int64_t cf = cash - (pre - x);
                if (lane == f) {
                    // the failing order: cf is below its cost, so (NARROW) below 2^32
                    const int64_t n = NARROW ? (int64_t)afford32((uint32_t)cf, (uint32_t)bp, fee, (uint32_t)bw)
                                             : afford(cf, bp, fee);
                    bn = n;
                    cf -= NARROW ? (int64_t)cost_of32((uint32_t)n, (uint32_t)bp, fee) : cost_of(n, bp, fee);
                }
                cash = __shfl_sync(FULL_MASK, cf, f);
                pending &= ~((2u << f) - 1u);
            }
            nb = BYSIZE ? __shfl_sync(FULL_MASK, bn, rank) : bn;
            h += nb;
            const int t1 = t0 + 1;
            const int64_t p1 = live ? (NARROW ? (int64_t)perturb32((uint32_t)c1, bps) : perturb(c1, bps)) : 0;
            const int64_t v1 = cash + warp_sum_redux(NARROW ? (int64_t)((uint64_t)(uint32_t)p1 * (uint32_t)h) : p1 * h);
            dn = t1 == W - 1;
            r = v1 - v0;
            fin.cash = cash;
            fin.v0 = v0;
            fin.v1 = v1;
            fin.t1 = t1;
            fin.done = dn ? 1 : 0;
            fin.valid = 1;
            const bool reset = dn && v.auto_reset;
            if (live) v.hold[(int64_t)e * KP + lane] = reset ? 0 : (int32_t)h;
            if (reset) {
                cash = v.init_cash;
                t_obs = 0;
                h = 0;
                p_obs = live ? perturb(__ldg(v.close + (int64_t)start * K + lane), bps) : 0;
            } else {
                t_obs = t1;
                p_obs = p1;
            }
        }
        if (lane == 0) {
            if (rew) rew[e] = r;
            if (rew_f32) rew_f32[e] = reward_f32(r);
            if (done_out) done_out[e] = dn ? 1 : 0;
            fin_sm[w] = fin;
        }
        if (obs) {
            // [cash*1e-8, p_k*1e-4, h_k*1e-2, f_{i,k} indicator-major], zero beyond Ke
            float *o = obs + (int64_t)e * ld;
            if (lane == 0) o[0] = obs_scale(cash, 1e-8f);
            if (lane < K) {
                // NARROW prices are below 2^31 and holdings are int32: the
                // 32-bit conversion gives the same correctly rounded float
                o[1 + lane] = live ? (NARROW ? __fmul_rn(__int2float_rn((int)p_obs), 1e-4f) : obs_scale(p_obs, 1e-4f))
                                   : 0.0f;
                o[1 + K + lane] = live ? __fmul_rn(__int2float_rn((int)h), 1e-2f) : 0.0f;
                const float *f = v.ind + (int64_t)(start + t_obs) * NI * K;
                float *oi = o + 1 + 2 * K + lane;
                if (NI == 8) {                           // the usual count: every load in flight
                    float fv[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) fv[i] = live ? __ldg(f + i * K + lane) : 0.0f;
#pragma unroll
                    for (int i = 0; i < 8; ++i) oi[i * K] = fv[i];
                } else {
                    for (int i = 0; i < NI; ++i) oi[i * K] = live ? __ldg(f + i * K + lane) : 0.0f;
                }
            }
        }
    } else if (lane == 0) {
        fin_sm[w].valid = 0;
    }
    __syncwarp();
    unsigned last = 0;
    if (lane == 0) {
        __threadfence_block();
        last = atomicAdd(&arrived, 1u) == (unsigned)(kStepEnvs - 1) ? 1u : 0u;
    }
    last = __shfl_sync(FULL_MASK, last, 0);
    if (last) {
        __threadfence_block();
        if (lane < kStepEnvs) {
            const StepFin f = fin_sm[lane];
            if (f.valid) finish_step(v, blockIdx.x * kStepEnvs + lane, f.cash, f.t1, f.done != 0, f.v0, f.v1);
        }
    }
}

// ------------------------------------------------ stock, two envs per warp
// Sums over each half-warp (lanes 0-15, 16-31), every lane receiving its own
// half's sum: one full-warp hardware reduction per half of the values masked
// to that half.  32-bit (mod 2^32) and exact int64 (mod 2^64, from 21-bit
// pieces as in warp_sum_redux: no partial sum of 16 lanes overflows).
__device__ __forceinline__ uint32_t half_sum32(uint32_t x, int half)
{
    const uint32_t s0 = __reduce_add_sync(FULL_MASK, half ? 0u : x);
    const uint32_t s1 = __reduce_add_sync(FULL_MASK, half ? x : 0u);
    return half ? s1 : s0;
}

__device__ __forceinline__ int64_t half_sum64(int64_t x, int half)
{
    const unsigned lo = (unsigned)x & 0x1fffffu;
    const unsigned mid = (unsigned)(x >> 21) & 0x1fffffu;
    const int hi = (int)(x >> 42);
    const unsigned slo = half_sum32(lo, half), smid = half_sum32(mid, half);
    const int shi = (int)half_sum32((uint32_t)hi, half);
    return (int64_t)(((uint64_t)(int64_t)shi << 42) + ((uint64_t)smid << 21) + (uint64_t)slo);
}

// The stock step of k_stock_step for the paper's shape (K = 30, I = 8) with
// 32-bit accounting (EnvView::narrow) and ascending buy order, two envs per
// warp: a half-warp per env, lane l of a half holding assets 2l and 2l + 1
// (lane 15 none).  The per-env work -- the state loads, index arithmetic
// and control -- serves two envs per warp instruction, the per-asset rows
// load as 4-, 8- and 16-byte vectors, and each warp keeps two envs' loads
// in flight.  Every sum, fill and rounding is that of k_stock_step, in the
// same asset order, so the results are identical.  Both halves run every
// warp-wide step: an env past N, or one already done, takes part with no
// orders and writes nothing it must not.  The caller guarantees that the
// action rows are 8-byte aligned.
constexpr int kHEnvs = 16;             // envs per block (8 warps)
constexpr int kHBlocks = kStepBlocks;  // resident blocks per SM (register bound)

template <int KIND>
__global__ void __launch_bounds__(kHEnvs * 16, kHBlocks) k_stock_step_h(EnvView v, const void *act, int64_t *rew,
                                                                  float *rew_f32, uint8_t *done_out,
                                                                  float *obs, int ld)
{
    constexpr int K = 30, NI = 8;
    __shared__ StepFin fin_sm[kHEnvs];
    __shared__ unsigned arrived;
    if (threadIdx.x == 0) arrived = 0u;
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int half = lane >> 4, hl = lane & 15;
    const int slot = 2 * w + half;                  // this half's env within the block
    const int e = blockIdx.x * kHEnvs + slot;
    const bool in = e < v.N;                        // uniform per half
    const int a0 = 2 * hl;                          // this lane's assets a0, a0 + 1 (none at hl = 15)
    const bool has = in && hl < 15;

    bool was_done = true;
    int Ke = 0, t0 = 0, start = 0, W = 2;
    int64_t cash0 = 0;
    if (in) {
        was_done = v.done[e] != 0;
        Ke = v.Ke[e];
        t0 = v.t[e];
        start = v.start[e];
        W = v.W[e];
        cash0 = v.cash[e];
    }
    const bool live0 = has && a0 < Ke, live1 = has && a0 + 1 < Ke;
    int b0 = 0, b1 = 0;
    int32_t h0 = 0, h1 = 0, q0 = 0, q1 = 0;
    if (has) {
        const short2 bb = *(const short2 *)(v.bps + (int64_t)e * KP + a0);
        b0 = bb.x;
        b1 = bb.y;
        const int2 hh = *(const int2 *)(v.hold + (int64_t)e * KP + a0);
        h0 = live0 ? hh.x : 0;
        h1 = live1 ? hh.y : 0;
        if (KIND == FR_ACT_I32_SHARES) {
            const int2 qq = *(const int2 *)((const int32_t *)act + (int64_t)e * K + a0);
            q0 = live0 ? qq.x : 0;
            q1 = live1 ? qq.y : 0;
        } else {
            const float2 aa = *(const float2 *)((const float *)act + (int64_t)e * K + a0);
            bool bad0 = false, bad1 = false;
            if (live0) q0 = discretise(aa.x, v.hmax, bad0);
            if (live1) q1 = discretise(aa.y, v.hmax, bad1);
            if (bad0 || bad1) atomicAdd(v.err, (unsigned long long)((bad0 ? 1 : 0) + (bad1 ? 1 : 0)));
        }
    }
    const int d = start + t0;
    uint32_t c00 = 0u, c01 = 0u, c10 = 0u, c11 = 0u;   // closes of the day and the next day (below 2^31)
    if (has) {
        const longlong2 x0 = __ldg((const longlong2 *)(v.close + (int64_t)d * K + a0));
        c00 = live0 ? (uint32_t)x0.x : 0u;
        c01 = live1 ? (uint32_t)x0.y : 0u;
        if (!was_done) {
            const longlong2 x1 = __ldg((const longlong2 *)(v.close + (int64_t)(d + 1) * K + a0));
            c10 = live0 ? (uint32_t)x1.x : 0u;
            c11 = live1 ? (uint32_t)x1.y : 0u;
        }
    }
    const int fee = v.fee_bps;
    // prices of the day (also the observation's when the env is done)
    uint32_t p0 = live0 ? perturb32(c00, b0) : 0u, p1 = live1 ? perturb32(c01, b1) : 0u;
    if (was_done) {                                // uniform per half: no orders
        q0 = 0;
        q1 = 0;
    }
    int64_t cash = cash0;
    // holdings are int32 >= 0 and prices below 2^31: 32 x 32 -> 64-bit products
    const int64_t v0 =
        cash + half_sum64((int64_t)((uint64_t)p0 * (uint32_t)h0 + (uint64_t)p1 * (uint32_t)h1), half);
    // sells, capped at the holding
    uint32_t net = 0u;
    if (q0 < 0) {
        const uint32_t n = (uint32_t)min(-(int64_t)q0, (int64_t)h0);
        h0 -= (int32_t)n;
        const uint32_t g = n * p0;
        net += g - fee_of32(g, fee);
    }
    if (q1 < 0) {
        const uint32_t n = (uint32_t)min(-(int64_t)q1, (int64_t)h1);
        h1 -= (int32_t)n;
        const uint32_t g = n * p1;
        net += g - fee_of32(g, fee);
    }
    cash += (int64_t)half_sum32(net, half);
    // buys in ascending asset order: one sum settles them when every order fits
    const uint32_t want0 = q0 > 0 ? (uint32_t)q0 : 0u, want1 = q1 > 0 ? (uint32_t)q1 : 0u;
    const uint32_t full0 = want0 ? cost_of32(want0, p0, fee) : 0u, full1 = want1 ? cost_of32(want1, p1, fee) : 0u;
    const uint32_t all = half_sum32(full0 + full1, half);
    uint32_t nb0 = 0u, nb1 = 0u;
    bool pend0 = want0 > 0u, pend1 = want1 > 0u;
    if ((int64_t)all <= cash) {
        nb0 = want0;
        nb1 = want1;
        cash -= (int64_t)all;
        pend0 = false;
        pend1 = false;
    }
    // otherwise rounds per half: drop the orders that cannot buy one share,
    // fill every order in full up to the first whose prefix cost exceeds the
    // cash, fill that one as far as the cash allows, continue after it
    const uint32_t one0 = pend0 ? cost_of32(1u, p0, fee) : 0u, one1 = pend1 ? cost_of32(1u, p1, fee) : 0u;
#pragma unroll 1
    while (__any_sync(FULL_MASK, pend0 || pend1)) {
        pend0 = pend0 && (int64_t)one0 <= cash;
        pend1 = pend1 && (int64_t)one1 <= cash;
        const uint32_t x0 = pend0 ? full0 : 0u, x1 = pend1 ? full1 : 0u;
        uint32_t y = x0 + x1;                       // inclusive prefix through asset a0 + 1
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
            const uint32_t z = __shfl_up_sync(FULL_MASK, y, o, 16);
            y += hl >= o ? z : 0u;
        }
        const uint32_t pre0 = y - x1;               // through asset a0
        const bool fail0 = pend0 && (int64_t)pre0 > cash, fail1 = pend1 && (int64_t)y > cash;
        const uint32_t fm = fail0 ? (uint32_t)a0 : (fail1 ? (uint32_t)a0 + 1u : 64u);
        const uint32_t f0 = __reduce_min_sync(FULL_MASK, half ? 64u : fm);
        const uint32_t f1 = __reduce_min_sync(FULL_MASK, half ? fm : 64u);
        const uint32_t f = half ? f1 : f0;          // the half's first failing order (64: none)
        const uint32_t total = __shfl_sync(FULL_MASK, y, 16 * half + 15);
        // the failing order: the cash before it is below its cost, so below 2^32
        int64_t cf = cash;
        const bool own0 = (uint32_t)a0 == f, own1 = (uint32_t)a0 + 1u == f;
        if (own0 || own1) {
            const uint32_t pp = own0 ? p0 : p1, ww = own0 ? want0 : want1;
            cf = cash - (int64_t)(own0 ? pre0 - x0 : y - x1);
            const uint32_t n = afford32((uint32_t)cf, pp, fee, ww);
            if (own0)
                nb0 = n;
            else
                nb1 = n;
            cf -= (int64_t)cost_of32(n, pp, fee);
        }
        const int64_t cf_f = __shfl_sync(FULL_MASK, cf, 16 * half + (int)min(f >> 1, 15u));
        if (f == 64u) {
            if (pend0) nb0 = want0;
            if (pend1) nb1 = want1;
            cash -= (int64_t)total;
            pend0 = false;
            pend1 = false;
        } else {
            if (pend0 && (uint32_t)a0 < f) nb0 = want0;
            if (pend1 && (uint32_t)a0 + 1u < f) nb1 = want1;
            cash = cf_f;
            pend0 = pend0 && (uint32_t)a0 > f;
            pend1 = pend1 && (uint32_t)a0 + 1u > f;
        }
    }
    h0 += (int32_t)nb0;
    h1 += (int32_t)nb1;
    const int t1 = t0 + 1;
    const uint32_t p10 = live0 ? perturb32(c10, b0) : 0u, p11 = live1 ? perturb32(c11, b1) : 0u;
    const int64_t v1 =
        cash + half_sum64((int64_t)((uint64_t)p10 * (uint32_t)h0 + (uint64_t)p11 * (uint32_t)h1), half);

    StepFin fin;
    fin.valid = 0;
    bool dn = true;
    int64_t r = 0;
    int t_obs = t0;
    if (in && !was_done) {                          // uniform per half
        dn = t1 == W - 1;
        r = v1 - v0;
        fin.cash = cash;
        fin.v0 = v0;
        fin.v1 = v1;
        fin.t1 = t1;
        fin.done = dn ? 1 : 0;
        fin.valid = 1;
        const bool reset = dn && v.auto_reset;
        int32_t *hp = v.hold + (int64_t)e * KP + a0;
        if (live1)
            *(int2 *)hp = reset ? make_int2(0, 0) : make_int2(h0, h1);
        else if (live0)
            *hp = reset ? 0 : h0;
        if (reset) {
            cash = v.init_cash;
            t_obs = 0;
            h0 = 0;
            h1 = 0;
            p0 = live0 ? (uint32_t)perturb(__ldg(v.close + (int64_t)start * K + a0), b0) : 0u;
            p1 = live1 ? (uint32_t)perturb(__ldg(v.close + (int64_t)start * K + a0 + 1), b1) : 0u;
        } else {
            t_obs = t1;
            p0 = p10;
            p1 = p11;
        }
    }
    if (hl == 0) {
        if (in) {
            if (rew) rew[e] = r;
            if (rew_f32) rew_f32[e] = reward_f32(r);
            if (done_out) done_out[e] = dn ? 1 : 0;
        }
        fin_sm[slot] = fin;
    }
    if (obs && in) {
        // [cash*1e-8, p_k*1e-4, h_k*1e-2, f_{i,k} indicator-major], zero beyond Ke
        float *o = obs + (int64_t)e * ld;
        if (hl == 0) o[0] = obs_scale(cash, 1e-8f);
        if (hl < 15) {
            // prices below 2^31 and int32 holdings: the 32-bit conversion
            // gives the same correctly rounded float
            o[1 + a0] = live0 ? __fmul_rn(__int2float_rn((int)p0), 1e-4f) : 0.0f;
            o[2 + a0] = live1 ? __fmul_rn(__int2float_rn((int)p1), 1e-4f) : 0.0f;
            o[1 + K + a0] = live0 ? __fmul_rn(__int2float_rn((int)h0), 1e-2f) : 0.0f;
            o[2 + K + a0] = live1 ? __fmul_rn(__int2float_rn((int)h1), 1e-2f) : 0.0f;
            const float *f = v.ind + (int64_t)(start + t_obs) * NI * K + a0;
            float2 fv[NI];
#pragma unroll
            for (int i = 0; i < NI; ++i) fv[i] = __ldg((const float2 *)(f + i * K));
            float *oi = o + 1 + 2 * K + a0;
#pragma unroll
            for (int i = 0; i < NI; ++i) {
                oi[i * K] = live0 ? fv[i].x : 0.0f;
                oi[i * K + 1] = live1 ? fv[i].y : 0.0f;
            }
        }
    }
    __syncwarp();
    unsigned last = 0;
    if (lane == 0) {
        __threadfence_block();
        last = atomicAdd(&arrived, 1u) == (unsigned)(kHEnvs / 2 - 1) ? 1u : 0u;
    }
    last = __shfl_sync(FULL_MASK, last, 0);
    if (last) {
        __threadfence_block();
        if (lane < kHEnvs) {
            const StepFin f = fin_sm[lane];
            if (f.valid) finish_step(v, blockIdx.x * kHEnvs + lane, f.cash, f.t1, f.done != 0, f.v0, f.v1);
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_crypto_step(EnvView v, const uint8_t *act, int64_t *rew,
                                                         float *rew_f32, uint8_t *done_out,
                                                         float *obs, int ld)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= v.N) return;
    int u = act[e];
    if (u > 2) {
        atomicAdd(v.err, 1ull);
        u = 1;
    }
    bool done;
    const int64_t r = crypto_step_thread(v, e, u, done);
    if (rew) rew[e] = r;
    if (rew_f32) rew_f32[e] = reward_f32(r);
    if (done_out) done_out[e] = done ? 1 : 0;
    if (obs) crypto_obs_thread(v, e, obs + (int64_t)e * ld);
}

__global__ void __launch_bounds__(kBlock) k_stock_observe(EnvView v, float *obs, int ld)
{
    const int e = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= v.N) return;
    stock_obs_warp(v, e, lane, obs + (int64_t)e * ld);
}

__global__ void k_crypto_observe(EnvView v, float *obs, int ld)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= v.N) return;
    crypto_obs_thread(v, e, obs + (int64_t)e * ld);
}

__global__ void k_env_metrics(EnvView v, double *out)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= v.N) return;
    const double *L = v.latched + (int64_t)e * 4;
    double *o = out + (int64_t)e * 3;
    if (v.t[e] == 0 && L[3] != 0.0) {
        o[0] = L[0];
        o[1] = L[1];
        o[2] = L[2];
    } else {
        acc_final(v.mu[e], v.m2[e], v.mdd[e], v.vlast[e], v.init_cash, v.t[e], v.ann, o);
    }
}

__global__ void k_env_get_state(EnvView v, int64_t *cash, int32_t *hold, int32_t *steps,
                                uint8_t *done)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int K = v.task == FR_TASK_STOCK ? v.K : 1;
    if (hold && i < (int64_t)v.N * K) {
        const int64_t e = i / K, k = i % K;
        hold[i] = v.task == FR_TASK_STOCK ? v.hold[e * KP + k] : v.hold[e];
    }
    if (i < v.N) {
        if (cash) cash[i] = v.cash[i];
        if (steps) steps[i] = v.t[i];
        if (done) done[i] = v.done[i];
    }
}

}  // namespace

cudaError_t launch_env_reset(const EnvView &v, cudaStream_t s)
{
    const int64_t n = (int64_t)v.N * (v.task == FR_TASK_STOCK ? KP : 1);
    k_env_reset<<<ceil_div(n, kBlock), kBlock, 0, s>>>(v);
    return cudaGetLastError();
}

namespace {
__global__ void k_explore_stock(float *act, int N, int K, Explore x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)N * K) return;
    const int e = (int)(i / K), k = (int)(i % K);
    act[i] = __fadd_rn(act[i], __fmul_rn(x.sigma, explore_normal(x, (uint32_t)e, x.g0, (uint32_t)k)));
}

__global__ void k_explore_crypto(uint8_t *act, int N, Explore x)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < N) act[e] = (uint8_t)explore_greedy(x, (uint32_t)e, x.g0, act[e]);
}
}  // namespace

cudaError_t launch_explore(const EnvView &v, void *act, const Explore &x, cudaStream_t s)
{
    if (x.kind == FR_EXPLORE_GAUSSIAN) {
        const int64_t n = (int64_t)v.N * v.K;
        k_explore_stock<<<ceil_div(n, kBlock), kBlock, 0, s>>>((float *)act, v.N, v.K, x);
    } else if (x.kind == FR_EXPLORE_EPS_GREEDY) {
        k_explore_crypto<<<ceil_div(v.N, kBlock), kBlock, 0, s>>>((uint8_t *)act, v.N, x);
    }
    return cudaGetLastError();
}

cudaError_t launch_env_step(const EnvView &v, int kind, const void *act, int64_t *rew,
                            float *rew_f32, uint8_t *done, float *obs, int ld, cudaStream_t s)
{
    if (v.task == FR_TASK_STOCK) {
        const unsigned grid = ceil_div(v.N, kStepEnvs);
        const bool by_size = v.buy_order == FR_BUY_LARGEST_FIRST;
        const unsigned bs = kStepEnvs * 32;
        const bool fixed = v.K == 30 && v.I == 8;
#define FR_STEP(K_, B_, N_, F_) k_stock_step<K_, B_, N_, F_><<<grid, bs, 0, s>>>(v, act, rew, rew_f32, done, obs, ld)
#define FR_STEP2(K_, B_)                                                                 \
    (fixed ? (v.narrow ? FR_STEP(K_, B_, true, true) : FR_STEP(K_, B_, false, true))     \
           : (v.narrow ? FR_STEP(K_, B_, true, false) : FR_STEP(K_, B_, false, false)))
        // the paper's shape with 32-bit accounting and ascending buys: two
        // envs per warp (vector loads of the action rows need 8-byte alignment)
        if (fixed && v.narrow && !by_size && ((uintptr_t)act & 7u) == 0) {
            const unsigned gh = ceil_div(v.N, kHEnvs);
            if (kind == FR_ACT_I32_SHARES)
                k_stock_step_h<FR_ACT_I32_SHARES><<<gh, kHEnvs * 16, 0, s>>>(v, act, rew, rew_f32, done, obs, ld);
            else
                k_stock_step_h<FR_ACT_F32_UNIT><<<gh, kHEnvs * 16, 0, s>>>(v, act, rew, rew_f32, done, obs, ld);
        } else if (kind == FR_ACT_I32_SHARES) {
            if (by_size)
                FR_STEP2(FR_ACT_I32_SHARES, true);
            else
                FR_STEP2(FR_ACT_I32_SHARES, false);
        } else {
            if (by_size)
                FR_STEP2(FR_ACT_F32_UNIT, true);
            else
                FR_STEP2(FR_ACT_F32_UNIT, false);
        }
#undef FR_STEP2
#undef FR_STEP
    } else {
        k_crypto_step<<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v, (const uint8_t *)act, rew, rew_f32,
                                                               done, obs, ld);
    }
    return cudaGetLastError();
}

cudaError_t launch_env_observe(const EnvView &v, float *obs, int ld, cudaStream_t s)
{
    if (v.task == FR_TASK_STOCK)
        k_stock_observe<<<ceil_div((int64_t)v.N * 32, kBlock), kBlock, 0, s>>>(v, obs, ld);
    else
        k_crypto_observe<<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v, obs, ld);
    return cudaGetLastError();
}

cudaError_t launch_env_metrics(const EnvView &v, double *out, cudaStream_t s)
{
    k_env_metrics<<<ceil_div(v.N, kBlock), kBlock, 0, s>>>(v, out);
    return cudaGetLastError();
}

cudaError_t launch_env_get_state(const EnvView &v, int64_t *cash, int32_t *hold, int32_t *steps,
                                 uint8_t *done, cudaStream_t s)
{
    const int64_t n = (int64_t)v.N * (v.task == FR_TASK_STOCK ? v.K : 1);
    k_env_get_state<<<ceil_div(n > v.N ? n : v.N, kBlock), kBlock, 0, s>>>(v, cash, hold, steps, done);
    return cudaGetLastError();
}

}  // namespace fr
