// fr_prep.cu -- on-device data preparation: the technical indicators of the
// state (Sec. 3.1 f_t; the Sec. 6.1 list: MACD, Bollinger bands, RSI-30,
// CCI-30, DX-30, SMA-30 and SMA-60) computed from daily OHLC on the GPU, and
// the per-env +-1% price perturbations of Sec. 5.1 drawn on the GPU.
//
// The indicators are computed in FP64 with every operation explicitly
// rounded (no contraction into FMA), in the order of their definitions:
// windows summed from the oldest day, recurrences in day order.  So the table
// is a pure function of the price series, identical on any launch shape.
//
// Two roles share the first launch.  Recurrence blocks (two per 32 assets;
// one lane per asset) run the six serial chains, one warp each: EMA-12 /
// EMA-26 together, and one each for the Wilder-smoothed gains, losses, TR,
// DM+ and DM-, storing each day's states.  Window blocks (one per asset and 128-day tile, one thread per
// day) stage the tile plus a 59-day halo of closes and typical prices in
// shared memory and compute the windowed means, the standard deviation and
// the mean absolute deviation.  A second launch, one thread per (day, asset),
// turns the states into MACD, RSI and DX, so the chains carry only their own
// recurrences (at most one FP64 division per day).
#include "fr_common.cuh"

namespace fr {
namespace {

constexpr int PREP_TILE = 128;     // days per window block
constexpr int PREP_HALO = 59;      // longest window (60 days) minus one
constexpr int N_IND = 8;

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

// Wilder smoothing with n = 30: w + (x - w) / 30.
__device__ __forceinline__ double wilder30(double w, double x) { return dadd(w, ddiv(dsub(x, w), 30.0)); }

__device__ __forceinline__ void put(float *ind, int K, int t, int col, int k, double v)
{
    ind[((int64_t)t * N_IND + col) * K + k] = __double2float_rn(v);
}

// Chain `role` for asset k over all T days: only a recurrence runs here, one
// value per day into plane `role` of st[6][T][K]: 0 e12 - e26, 1 / 2 the
// Wilder-smoothed gains / losses, 3 / 4 / 5 the Wilder-smoothed TR, DM+, DM-
// (each role derives its own inputs, so every chain carries at most one
// division per day); the divisions that turn the states into MACD, RSI and
// DX are off the chains, in k_ind_final, one thread per (day, asset).
__device__ void indicator_chain(int role, int k, const int64_t *close, const int64_t *high, const int64_t *low,
                                int T, int K, double *st)
{
    double *out = st + (int64_t)role * T * K;
    const double c0 = (double)close[k];
    if (role == 0) {
        // e_t = a c_t + (1 - a) e_{t-1}, a = 2 / (n + 1), e_0 = c_0
        const double a12 = ddiv(2.0, 13.0), a26 = ddiv(2.0, 27.0);
        const double b12 = dsub(1.0, a12), b26 = dsub(1.0, a26);
        double e12 = c0, e26 = c0;
#pragma unroll 4
        for (int t = 0; t < T; ++t) {
            const double ct = (double)close[(int64_t)t * K + k];
            if (t > 0) {
                e12 = dadd(dmul(a12, ct), dmul(b12, e12));
                e26 = dadd(dmul(a26, ct), dmul(b26, e26));
            }
            out[(int64_t)t * K + k] = dsub(e12, e26);
        }
    } else if (role <= 2) {
        // Wilder-smoothed gains (role 1) or losses (role 2) of c_t - c_{t-1}
        double w = 0.0, cp = c0;
#pragma unroll 4
        for (int t = 0; t < T; ++t) {
            const double ct = (double)close[(int64_t)t * K + k];
            const double d = dsub(ct, cp);
            const double x = role == 1 ? (d > 0.0 ? d : 0.0) : (d < 0.0 ? -d : 0.0);
            w = t == 0 ? x : wilder30(w, x);
            out[(int64_t)t * K + k] = w;
            cp = ct;
        }
    } else {
        // Wilder-smoothed true range (3), DM+ (4) or DM- (5), c_{-1} = c_0
        double w = 0.0, cp = c0;
        double hp = (double)high[k], lp = (double)low[k];
#pragma unroll 4
        for (int t = 0; t < T; ++t) {
            const int64_t i = (int64_t)t * K + k;
            const double ct = (double)close[i], ht = (double)high[i], lt = (double)low[i];
            double x;
            if (role == 3) {
                double tr = dsub(ht, lt);
                const double th = fabs(dsub(ht, cp)), tl = fabs(dsub(lt, cp));
                if (th > tr) tr = th;
                if (tl > tr) tr = tl;
                x = tr;
            } else {
                const double up = t > 0 ? dsub(ht, hp) : 0.0;
                const double dn = t > 0 ? dsub(lp, lt) : 0.0;
                x = role == 4 ? ((up > dn && up > 0.0) ? up : 0.0) : ((dn > up && dn > 0.0) ? dn : 0.0);
            }
            w = t == 0 ? x : wilder30(w, x);
            out[i] = w;
            cp = ct;
            hp = ht;
            lp = lt;
        }
    }
}

// MACD / c, RSI-30 / 100 and DX-30 / 100 of (day, asset) from the chains'
// states, the same operations as if they ran on the chain.
__global__ void k_ind_final(const int64_t *__restrict__ close, int T, int K, const double *__restrict__ st,
                            float *__restrict__ ind)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t TK = (int64_t)T * K;
    if (i >= TK) return;
    const int t = (int)(i / K), k = (int)(i % K);
    const double ct = (double)close[i];
    put(ind, K, t, 0, k, ddiv(st[i], ct));
    const double gain = st[TK + i], loss = st[2 * TK + i];
    double rsi;
    if (gain == 0.0 && loss == 0.0) rsi = 50.0;
    else if (loss > 0.0) rsi = dsub(100.0, ddiv(100.0, dadd(1.0, ddiv(gain, loss))));
    else rsi = 100.0;
    put(ind, K, t, 3, k, ddiv(rsi, 100.0));
    const double str = st[3 * TK + i], spd = st[4 * TK + i], snd = st[5 * TK + i];
    const double den = str > 0.0 ? str : 1.0;
    const double pdi = ddiv(dmul(100.0, spd), den), ndi = ddiv(dmul(100.0, snd), den);
    const double s = dadd(pdi, ndi);
    const double dx = s > 0.0 ? ddiv(dmul(100.0, fabs(dsub(pdi, ndi))), s) : 0.0;
    put(ind, K, t, 5, k, ddiv(dx, 100.0));
}

// Mean of x[j - m + 1 .. j] in shared memory, m = min(n, t + 1) days ending at
// day t (local index j), summed from the oldest.
__device__ __forceinline__ double win_mean(const double *x, int j, int t, int n, int &m)
{
    m = t + 1 < n ? t + 1 : n;
    double s = 0.0;
    for (int u = j - m + 1; u <= j; ++u) s = dadd(s, x[u]);
    return ddiv(s, (double)m);
}

__global__ void __launch_bounds__(PREP_TILE) k_indicators(const int64_t *__restrict__ close,
                                                          const int64_t *__restrict__ high,
                                                          const int64_t *__restrict__ low, int T, int K,
                                                          float *__restrict__ ind, int n_chain, int n_tiles,
                                                          double *__restrict__ st)
{
    if ((int)blockIdx.x < n_chain) {
        // two recurrence blocks per 32 assets, three chains (warps) each
        const int role = (blockIdx.x & 1) * 3 + (threadIdx.x >> 5);
        const int k = (blockIdx.x >> 1) * 32 + (threadIdx.x & 31);
        if ((threadIdx.x >> 5) < 3 && k < K) indicator_chain(role, k, close, high, low, T, K, st);
        return;
    }
    __shared__ double c_s[PREP_TILE + PREP_HALO], tp_s[PREP_TILE + PREP_HALO];
    const int b = blockIdx.x - n_chain;
    const int k = b / n_tiles, t0 = (b % n_tiles) * PREP_TILE;
    for (int j = threadIdx.x; j < PREP_TILE + PREP_HALO; j += PREP_TILE) {
        const int u = t0 - PREP_HALO + j;
        if (u >= 0 && u < T) {
            const int64_t i = (int64_t)u * K + k;
            const double c = (double)close[i];
            c_s[j] = c;
            tp_s[j] = ddiv(dadd(dadd((double)high[i], (double)low[i]), c), 3.0);
        }
    }
    __syncthreads();
    const int t = t0 + threadIdx.x;
    if (t >= T) return;
    const int j = PREP_HALO + threadIdx.x;
    const double ct = c_s[j];
    int m;
    // Bollinger(20, 2): SMA20 +- 2 population standard deviations
    const double sma20 = win_mean(c_s, j, t, 20, m);
    double v = 0.0;
    for (int u = j - m + 1; u <= j; ++u) {
        const double z = dsub(c_s[u], sma20);
        v = dadd(v, dmul(z, z));
    }
    const double sd20 = __dsqrt_rn(ddiv(v, (double)m));
    put(ind, K, t, 1, k, dsub(ddiv(dadd(sma20, dmul(2.0, sd20)), ct), 1.0));
    put(ind, K, t, 2, k, dsub(ddiv(dsub(sma20, dmul(2.0, sd20)), ct), 1.0));
    // CCI-30 = (tp - SMA30(tp)) / (0.015 MAD30(tp))
    const double smatp = win_mean(tp_s, j, t, 30, m);
    double mad = 0.0;
    for (int u = j - m + 1; u <= j; ++u) mad = dadd(mad, fabs(dsub(tp_s[u], smatp)));
    mad = ddiv(mad, (double)m);
    const double cci = mad > 0.0 ? ddiv(dsub(tp_s[j], smatp), dmul(0.015, mad)) : 0.0;
    put(ind, K, t, 4, k, ddiv(cci, 100.0));
    // SMA30 / c - 1, SMA60 / c - 1
    put(ind, K, t, 6, k, dsub(ddiv(win_mean(c_s, j, t, 30, m), ct), 1.0));
    put(ind, K, t, 7, k, dsub(ddiv(win_mean(c_s, j, t, 60, m), ct), 1.0));
}

__global__ void k_perturb(EnvView v, uint64_t seed, int R)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)v.N * KP) return;
    const int e = (int)(i / KP), k = (int)(i % KP);
    ((int16_t *)v.bps)[i] = (k < v.K && R > 0) ? perturb_bps(seed, (uint32_t)e, (uint32_t)k, R) : (int16_t)0;
}

}  // namespace

cudaError_t launch_indicators(const int64_t *close, const int64_t *high, const int64_t *low, int T, int K,
                              float *ind, cudaStream_t s)
{
    const int n_chain = 2 * ((K + 31) / 32), n_tiles = (T + PREP_TILE - 1) / PREP_TILE;
    const long long blocks = (long long)n_chain + (long long)K * n_tiles;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    // the chains' states, stream-ordered scratch: 6 doubles per (day, asset)
    double *st = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&st, 48ull * (uint64_t)T * K, s);
    if (e != cudaSuccess) return e;
    k_indicators<<<(unsigned)blocks, PREP_TILE, 0, s>>>(close, high, low, T, K, ind, n_chain, n_tiles, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_ind_final<<<ceil_div((int64_t)T * K, 256), 256, 0, s>>>(close, T, K, st, ind);
        e = cudaGetLastError();
    }
    const cudaError_t f = cudaFreeAsync(st, s);
    return e != cudaSuccess ? e : f;
}

}  // namespace fr

using namespace fr;

extern "C" {

int market_indicators(const int64_t *close, const int64_t *high, const int64_t *low, int32_t n_days,
                      int32_t n_assets, float *ind, void *stream)
{
    FR_NVTX("market_indicators");
    FR_CHECK(close && high && low && ind, FR_EINVAL, "market_indicators: NULL table");
    FR_CHECK(n_days >= 1 && n_assets >= 1 && (int64_t)n_days * n_assets <= ((int64_t)1 << 40), FR_EINVAL,
             "market_indicators: n_days %d and n_assets %d must be >= 1", n_days, n_assets);
    FR_CUDA(launch_indicators(close, high, low, n_days, n_assets, ind, (cudaStream_t)stream));
    return FR_OK;
}

int env_perturb(fr_env *env, uint64_t seed, int32_t bps_range, void *stream)
{
    FR_NVTX("env_perturb");
    FR_CHECK(env, FR_EINVAL, "env_perturb: NULL env");
    FR_CHECK(env->v.task == FR_TASK_STOCK, FR_EINVAL, "env_perturb: stock envs only");
    FR_CHECK(bps_range >= 0 && bps_range <= 100, FR_EINVAL, "env_perturb: bps_range %d not in 0..100",
             bps_range);
    FR_CUDA(cudaSetDevice(env->ctx->device));
    const int64_t n = (int64_t)env->v.N * KP;
    k_perturb<<<ceil_div(n, 256), 256, 0, (cudaStream_t)stream>>>(env->v, seed, bps_range);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

}  // extern "C"
