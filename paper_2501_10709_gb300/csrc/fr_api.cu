// fr_api.cu -- the C ABI: contexts with an HBM budget, device-resident market
// tables, env batches in structure-of-arrays layout, ensembles, and the
// rollout driver that strings observe -> ensemble -> step together
// (the simulation phase of Sec. 3.2, parallel over trajectories, Sec. 4.2.1).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "fr_common.cuh"

namespace fr {

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what)
{
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return FR_ECUDA;
}

// ------------------------------------------------------------------ budget
static std::mutex g_budget_mu;

int ctx_reserve(fr_ctx *ctx, uint64_t bytes)
{
    std::lock_guard<std::mutex> lk(g_budget_mu);
    if (ctx->budget && ctx->used + bytes > ctx->budget) {
        set_error("HBM budget exceeded: %llu in use + %llu requested > %llu",
                  (unsigned long long)ctx->used, (unsigned long long)bytes,
                  (unsigned long long)ctx->budget);
        return FR_ENOMEM;
    }
    ctx->used += bytes;
    return FR_OK;
}

void ctx_release(fr_ctx *ctx, uint64_t bytes)
{
    std::lock_guard<std::mutex> lk(g_budget_mu);
    ctx->used = ctx->used >= bytes ? ctx->used - bytes : 0;
}

// Host fault injection: per kind, events to let through, then events to fail.
static std::mutex g_fault_mu;
static std::atomic<int> g_fault_armed{0};
static int32_t g_fault_skip[4], g_fault_count[4];

bool fault_hit(int kind)
{
    if (g_fault_armed.load(std::memory_order_relaxed) == 0) return false;
    std::lock_guard<std::mutex> lk(g_fault_mu);
    if (kind < 1 || kind > 3 || g_fault_count[kind] <= 0) return false;
    if (g_fault_skip[kind] > 0) {
        --g_fault_skip[kind];
        return false;
    }
    if (--g_fault_count[kind] == 0 && g_fault_count[1] + g_fault_count[2] + g_fault_count[3] == 0)
        g_fault_armed.store(0, std::memory_order_relaxed);
    return true;
}

int dev_alloc(fr_ctx *ctx, void **p, uint64_t bytes)
{
    *p = nullptr;
    if (bytes == 0) return FR_OK;
    if (fault_hit(FR_FAULT_ALLOC)) {
        set_error("device allocation of %llu bytes failed (injected fault)", (unsigned long long)bytes);
        return FR_ENOMEM;
    }
    int rc = ctx_reserve(ctx, bytes);
    if (rc) return rc;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        ctx_release(ctx, bytes);
        *p = nullptr;
        (void)cudaGetLastError();
        set_error("cudaMalloc of %llu bytes failed: %s", (unsigned long long)bytes,
                  cudaGetErrorString(e));
        return FR_ENOMEM;
    }
    return FR_OK;
}

void dev_free(fr_ctx *ctx, void *p, uint64_t bytes)
{
    if (!p) return;
    cudaFree(p);
    ctx_release(ctx, bytes);
}

static int use_device(const fr_ctx *ctx)
{
    FR_CUDA(cudaSetDevice(ctx->device));
    return FR_OK;
}

// ------------------------------------------------------- plain fp32 forward
cudaError_t forward_plain(const fr_ensemble *e, const float *obs, int ld, int n, float *y,
                          float *scratch, cudaStream_t s)
{
    int wmax = 0;
    for (int l = 1; l < e->L; ++l) wmax = std::max(wmax, e->dims[l]);
    const float *in = obs;
    int64_t in_stride = 0;
    int in_ld = ld;
    for (int l = 0; l < e->L; ++l) {
        const bool last = l == e->L - 1;
        const int fin = e->dims[l], fout = e->dims[l + 1];
        float *out = last ? y : scratch + (int64_t)(l & 1) * e->M * n * wmax;
        const int64_t out_stride = (int64_t)n * fout;
        const int act = last ? (e->out_act ? 1 : 2) : 0;
        cudaError_t err = launch_dense_f32(in, in_stride, in_ld, e->params, e->P, e->w_off[l],
                                           e->b_off[l], out, out_stride, fout, n, fin, fout,
                                           act, e->M, s);
        if (err != cudaSuccess) return err;
        in = out;
        in_stride = out_stride;
        in_ld = fout;
    }
    return cudaSuccess;
}

namespace {
struct Carve {
    char *base;
    uint64_t off = 0;
    template <class T>
    T *take(uint64_t count)
    {
        off = (off + 255) & ~255ull;
        T *p = (T *)(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
};

// Lay out every per-env array in one block; with base NULL only sizes it.
uint64_t carve_env(EnvView &v, char *base)
{
    Carve c{base};
    const int64_t N = v.N;
    const int64_t hs = v.task == FR_TASK_STOCK ? KP : 1;
    v.Ke = c.take<int32_t>(N);
    v.start = c.take<int32_t>(N);
    v.W = c.take<int32_t>(N);
    v.bps = c.take<int16_t>(v.task == FR_TASK_STOCK ? N * KP : 1);
    // state (contiguous from here: the snapshot covers it all)
    v.cash = c.take<int64_t>(N);
    v.hold = c.take<int32_t>(N * hs);
    v.t = c.take<int32_t>(N);
    v.done = c.take<uint8_t>(N);
    v.mu = c.take<double>(N);
    v.m2 = c.take<double>(N);
    v.mdd = c.take<double>(N);
    v.peak = c.take<int64_t>(N);
    v.vlast = c.take<int64_t>(N);
    v.latched = c.take<double>(N * 4);
    v.err = c.take<unsigned long long>(1);
    return (c.off + 255) & ~255ull;
}
}  // namespace

namespace {
struct SnapHeader {
    uint32_t magic, version;
    int32_t task, N, K, I;
    uint64_t state_off, state_bytes;
};
constexpr uint32_t kSnapMagic = 0x4e534652u;  // "FRSN"
}  // namespace

namespace {
// per-agent outputs into y[M][n][out]; plain path scratch from the stream-
// ordered allocator so that calls on different streams never share it
int forward_any(const fr_ensemble *e, const float *obs, int ld, int n, float *y, cudaStream_t s)
{
    if (e->precision != FR_PREC_FP32) {
        const uint64_t tb = tc_tiled_scratch_bytes(e, n);
        if (tb == 0) return tc_forward(e, obs, ld, n, y, s);
        void *tiles = nullptr;
        FR_CUDA(cudaMallocAsync(&tiles, tb, s));
        const int rc = tc_forward_tiled(e, obs, ld, n, y, tiles, s);
        cudaFreeAsync(tiles, s);
        if (rc == FR_EINVAL) return tc_forward(e, obs, ld, n, y, s);   // plan too large for the tiled kernel
        return rc;
    }
    void *scratch = nullptr;
    const uint64_t sb = plain_scratch_bytes(e, n);
    if (sb) FR_CUDA(cudaMallocAsync(&scratch, sb, s));
    cudaError_t err = forward_plain(e, obs, ld, n, y, (float *)scratch, s);
    if (scratch) cudaFreeAsync(scratch, s);
    FR_CUDA(err);
    return FR_OK;
}
}  // namespace

}  // namespace fr

using namespace fr;

// =================================================================== C ABI
extern "C" {

const char *fr_last_error(void) { return g_err; }

const char *fr_version(void) { return "finrl_gb300 0.1 (sm_103a)"; }

int fr_fault_inject(int32_t kind, int32_t skip, int32_t count)
{
    FR_CHECK(kind >= FR_FAULT_ALLOC && kind <= FR_FAULT_POLL && skip >= 0 && count >= 0, FR_EINVAL,
             "fr_fault_inject: kind %d, skip %d, count %d", kind, skip, count);
    std::lock_guard<std::mutex> lk(g_fault_mu);
    g_fault_skip[kind] = skip;
    g_fault_count[kind] = count;
    g_fault_armed.store(g_fault_count[1] + g_fault_count[2] + g_fault_count[3] > 0 ? 1 : 0,
                        std::memory_order_relaxed);
    return FR_OK;
}

// ---------------------------------------------------------------- context
int fr_ctx_create(int device, uint64_t hbm_budget_bytes, fr_ctx **out)
{
    FR_NVTX("fr_ctx_create");
    FR_CHECK(out, FR_EINVAL, "fr_ctx_create: out is NULL");
    *out = nullptr;
    int n = 0;
    FR_CUDA(cudaGetDeviceCount(&n));
    FR_CHECK(device >= 0 && device < n, FR_EINVAL, "fr_ctx_create: device %d of %d", device, n);
    FR_CUDA(cudaSetDevice(device));
    fr_ctx *c = new (std::nothrow) fr_ctx();
    FR_CHECK(c, FR_ENOMEM, "fr_ctx_create: out of host memory");
    c->device = device;
    c->budget = hbm_budget_bytes;
    c->used = 0;
    cudaError_t e1 = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    cudaError_t e2 = cudaDeviceGetAttribute(&c->cc_major, cudaDevAttrComputeCapabilityMajor, device);
    cudaError_t e3 = cudaDeviceGetAttribute(&c->cc_minor, cudaDevAttrComputeCapabilityMinor, device);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        delete c;
        return cuda_fail(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3), "device attributes");
    }
    *out = c;
    return FR_OK;
}

void fr_ctx_destroy(fr_ctx *ctx) { delete ctx; }

uint64_t fr_ctx_bytes_in_use(const fr_ctx *ctx) { return ctx ? ctx->used : 0; }

int fr_ctx_sm_count(const fr_ctx *ctx) { return ctx ? ctx->sm_count : 0; }

// ----------------------------------------------------------------- market
int fr_market_create(fr_ctx *ctx, const fr_market_desc *d, fr_market **out)
{
    FR_NVTX("fr_market_create");
    FR_CHECK(ctx && d && out, FR_EINVAL, "fr_market_create: NULL argument");
    *out = nullptr;
    int rc = use_device(ctx);
    if (rc) return rc;
    fr_market *m = new (std::nothrow) fr_market();
    FR_CHECK(m, FR_ENOMEM, "fr_market_create: out of host memory");
    m->ctx = ctx;
    m->task = d->task;
    if (d->task == FR_TASK_STOCK) {
        const bool prep = !d->ind && d->n_ind == 8 && d->high && d->low;
        if (!(d->n_days >= 2 && d->n_assets >= 1 && d->n_assets <= FR_MAX_ASSETS &&
              d->n_ind >= 0 && d->n_ind <= FR_MAX_INDICATORS && d->close &&
              (d->ind || d->n_ind == 0 || prep))) {
            delete m;
            set_error("fr_market_create: stock market needs n_days >= 2, 1 <= n_assets <= 32, "
                      "0 <= n_ind <= 16 and host tables");
            return FR_EINVAL;
        }
        m->close_max = 1;
        for (int64_t i = 0; i < (int64_t)d->n_days * d->n_assets; ++i) {
            if (d->close[i] < 1) {
                delete m;
                set_error("fr_market_create: close[%lld] = %lld < 1 cent", (long long)i,
                          (long long)d->close[i]);
                return FR_EINVAL;
            }
            m->close_max = std::max(m->close_max, d->close[i]);
        }
        m->n_days = d->n_days;
        m->K = d->n_assets;
        m->I = d->n_ind;
        const uint64_t cb = (uint64_t)m->n_days * m->K * 8;
        const uint64_t ib = (uint64_t)m->n_days * m->I * m->K * 4;
        if ((rc = dev_alloc(ctx, (void **)&m->close, cb)) ||
            (rc = dev_alloc(ctx, (void **)&m->ind, ib ? ib : 16))) {
            fr_market_destroy(m);
            return rc;
        }
        m->bytes = cb + (ib ? ib : 16);
        cudaError_t e = cudaMemcpy(m->close, d->close, cb, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && ib && !prep) e = cudaMemcpy(m->ind, d->ind, ib, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            fr_market_destroy(m);
            return cuda_fail(e, "fr_market_create upload");
        }
        if (prep) {
            for (int64_t i = 0; i < (int64_t)d->n_days * d->n_assets; ++i) {
                if (!(d->low[i] <= d->close[i] && d->close[i] <= d->high[i])) {
                    fr_market_destroy(m);
                    set_error("fr_market_create: low <= close <= high fails at %lld", (long long)i);
                    return FR_EINVAL;
                }
            }
            // high / low staged in one temporary allocation, freed after the launch completes
            int64_t *hl = nullptr;
            if ((rc = dev_alloc(ctx, (void **)&hl, 2 * cb))) {
                fr_market_destroy(m);
                return rc;
            }
            e = cudaMemcpy(hl, d->high, cb, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(hl + cb / 8, d->low, cb, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = launch_indicators(m->close, hl, hl + cb / 8, m->n_days, m->K, m->ind, 0);
            if (e == cudaSuccess) e = cudaStreamSynchronize(0);
            dev_free(ctx, hl, 2 * cb);
            if (e != cudaSuccess) {
                fr_market_destroy(m);
                return cuda_fail(e, "fr_market_create indicators");
            }
        }
    } else if (d->task == FR_TASK_CRYPTO) {
        if (!(d->n_seconds >= 2 && d->mid && d->spread && d->fac)) {
            delete m;
            set_error("fr_market_create: crypto market needs n_seconds >= 2 and host tables");
            return FR_EINVAL;
        }
        for (int64_t i = 0; i < d->n_seconds; ++i) {
            if (d->mid[i] < 1 || (int64_t)d->spread[i] >= 2 * d->mid[i]) {
                delete m;
                set_error("fr_market_create: mid/spread at second %lld out of range", (long long)i);
                return FR_EINVAL;
            }
        }
        m->S = d->n_seconds;
        m->K = 1;
        const uint64_t mb = (uint64_t)m->S * 8, sb = (uint64_t)m->S, fb = (uint64_t)m->S * 32;
        if ((rc = dev_alloc(ctx, (void **)&m->mid, mb)) ||
            (rc = dev_alloc(ctx, (void **)&m->spread, sb)) ||
            (rc = dev_alloc(ctx, (void **)&m->fac, fb))) {
            fr_market_destroy(m);
            return rc;
        }
        m->bytes = mb + sb + fb;
        cudaError_t e = cudaMemcpy(m->mid, d->mid, mb, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(m->spread, d->spread, sb, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(m->fac, d->fac, fb, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            fr_market_destroy(m);
            return cuda_fail(e, "fr_market_create upload");
        }
    } else {
        delete m;
        set_error("fr_market_create: unknown task %d", d->task);
        return FR_EINVAL;
    }
    *out = m;
    return FR_OK;
}

int fr_market_copy_indicators(const fr_market *m, float *dst)
{
    FR_NVTX("fr_market_copy_indicators");
    FR_CHECK(m && dst, FR_EINVAL, "fr_market_copy_indicators: NULL argument");
    FR_CHECK(m->task == FR_TASK_STOCK, FR_EINVAL, "fr_market_copy_indicators: stock markets only");
    int rc = use_device(m->ctx);
    if (rc) return rc;
    const uint64_t ib = (uint64_t)m->n_days * m->I * m->K * 4;
    if (ib) FR_CUDA(cudaMemcpy(dst, m->ind, ib, cudaMemcpyDefault));
    return FR_OK;
}

void fr_market_destroy(fr_market *m)
{
    FR_NVTX("fr_market_destroy");
    if (!m) return;
    cudaSetDevice(m->ctx->device);
    if (m->task == FR_TASK_STOCK) {
        dev_free(m->ctx, m->close, (uint64_t)m->n_days * m->K * 8);
        uint64_t ib = (uint64_t)m->n_days * m->I * m->K * 4;
        dev_free(m->ctx, m->ind, ib ? ib : 16);
    } else {
        dev_free(m->ctx, m->mid, (uint64_t)m->S * 8);
        dev_free(m->ctx, m->spread, (uint64_t)m->S);
        dev_free(m->ctx, m->fac, (uint64_t)m->S * 32);
    }
    delete m;
}

// -------------------------------------------------------------------- env

int env_create(fr_ctx *ctx, const fr_env_desc *d, const fr_market *m, fr_env **out)
{
    FR_NVTX("env_create");
    FR_CHECK(ctx && d && m && out, FR_EINVAL, "env_create: NULL argument");
    *out = nullptr;
    FR_CHECK(d->task == m->task, FR_EINVAL, "env_create: env task %d on a market of task %d",
             d->task, m->task);
    FR_CHECK(d->n_envs >= 1 && d->window && d->start, FR_EINVAL,
             "env_create: need n_envs >= 1, window[] and start[]");
    FR_CHECK(d->init_cash >= 0, FR_EINVAL, "env_create: init_cash < 0");
    const int N = d->n_envs;
    const bool stock = d->task == FR_TASK_STOCK;
    if (stock) {
        FR_CHECK(d->hmax >= 1 && d->hmax <= 1000000, FR_EINVAL, "env_create: hmax %d not in 1..1e6",
                 d->hmax);
        FR_CHECK(d->fee_bps >= 0 && d->fee_bps <= BPS_ONE, FR_EINVAL,
                 "env_create: fee_bps %d not in 0..10000", d->fee_bps);
    } else {
        FR_CHECK(d->pmax >= 1, FR_EINVAL, "env_create: pmax < 1");
    }
    FR_CHECK(d->buy_order == FR_BUY_ASCENDING || (stock && d->buy_order == FR_BUY_LARGEST_FIRST), FR_EINVAL,
             "env_create: buy_order %d not valid for this task", d->buy_order);
    const int64_t horizon = stock ? m->n_days : m->S;
    std::vector<int32_t> Ke(N, stock ? m->K : 1);
    for (int e = 0; e < N; ++e) {
        if (stock && d->n_assets) Ke[e] = d->n_assets[e];
        FR_CHECK(Ke[e] >= 1 && Ke[e] <= m->K, FR_EINVAL, "env_create: n_assets[%d] = %d not in 1..%d",
                 e, Ke[e], m->K);
        FR_CHECK(d->window[e] >= 2, FR_EINVAL, "env_create: window[%d] = %d < 2", e, d->window[e]);
        FR_CHECK(d->start[e] >= 0 && (int64_t)d->start[e] + d->window[e] <= horizon, FR_EINVAL,
                 "env_create: env %d window %d..%d runs past the market end %lld", e,
                 d->start[e], d->start[e] + d->window[e] - 1, (long long)horizon);
        if (stock && d->bps) {
            for (int k = 0; k < m->K; ++k) {
                const int b = d->bps[(int64_t)e * m->K + k];
                FR_CHECK(b >= -100 && b <= 100, FR_EINVAL, "env_create: bps[%d][%d] = %d not in -100..100",
                         e, k, b);
            }
        }
    }
    int rc = use_device(ctx);
    if (rc) return rc;
    fr_env *env = new (std::nothrow) fr_env();
    FR_CHECK(env, FR_ENOMEM, "env_create: out of host memory");
    env->ctx = ctx;
    env->mkt = m;
    EnvView &v = env->v;
    v.task = d->task;
    v.N = N;
    v.K = stock ? m->K : 1;
    v.I = stock ? m->I : 0;
    v.D = stock ? 1 + 2 * m->K + m->I * m->K : FR_CRYPTO_OBS_DIM;
    v.hmax = d->hmax;
    v.fee_bps = d->fee_bps;
    v.pmax = d->pmax;
    v.auto_reset = d->auto_reset ? 1 : 0;
    v.buy_order = d->buy_order;
    // The step kernel's 32-bit accounting is exact when, for every price the
    // env can see (perturbed by at most +100 bps): the perturbation's
    // numerator close * (1e4 + bps) + 5e3 fits 32 bits; an order's notional
    // (at most hmax shares) plus its fee fits 31 bits and notional * fee_bps
    // + 9,999 fits 32 bits; and K such amounts (a step's sell proceeds or buy
    // costs) sum within 32 bits.
    if (stock) {
        const uint64_t cmax = (uint64_t)m->close_max;
        const uint64_t pmax = (cmax * (uint64_t)(BPS_ONE + 100) + BPS_ONE / 2) / BPS_ONE;
        const uint64_t gmax = pmax * (uint64_t)d->hmax;
        const uint64_t fmax = (gmax * (uint64_t)d->fee_bps + BPS_ONE - 1) / BPS_ONE;
        v.narrow = cmax * (uint64_t)(BPS_ONE + 100) + BPS_ONE / 2 < (1ull << 32) &&
                   gmax * (uint64_t)d->fee_bps + BPS_ONE < (1ull << 32) && gmax + fmax < (1ull << 31) &&
                   (uint64_t)m->K * (gmax + fmax) < (1ull << 32);
    }
    v.init_cash = d->init_cash;
    v.ann = stock ? 252.0 : 1.0;
    v.n_days = m->n_days;
    v.S = m->S;
    v.close = m->close;
    v.ind = m->ind;
    v.mid = m->mid;
    v.spread = m->spread;
    v.fac = m->fac;
    const uint64_t bytes = carve_env(v, nullptr);
    rc = dev_alloc(ctx, &env->block, bytes);
    if (rc) {
        delete env;
        return rc;
    }
    env->bytes = bytes;
    carve_env(v, (char *)env->block);
    // host staging of the per-env constants
    std::vector<int16_t> bps(stock ? (size_t)N * KP : 1, 0);
    if (stock && d->bps)
        for (int e = 0; e < N; ++e)
            for (int k = 0; k < m->K; ++k) bps[(size_t)e * KP + k] = d->bps[(int64_t)e * m->K + k];
    cudaError_t err = cudaMemcpy((void *)v.Ke, Ke.data(), 4ull * N, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy((void *)v.start, d->start, 4ull * N, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy((void *)v.W, d->window, 4ull * N, cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy((void *)v.bps, bps.data(), bps.size() * 2, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemset(v.err, 0, 8);
    if (err == cudaSuccess) err = launch_env_reset(v, 0);
    if (err == cudaSuccess) err = cudaDeviceSynchronize();
    if (err != cudaSuccess) {
        env_destroy(env);
        return cuda_fail(err, "env_create upload");
    }
    *out = env;
    return FR_OK;
}

void env_destroy(fr_env *env)
{
    FR_NVTX("env_destroy");
    if (!env) return;
    cudaSetDevice(env->ctx->device);
    dev_free(env->ctx, env->block, env->bytes);
    dev_free(env->ctx, env->scratch, env->scratch_bytes);
    dev_free(env->ctx, env->slot_of_env, 4ull * env->v.N + 4ull * 32);
    dev_free(env->ctx, env->zbuf, env->zbuf_bytes);
    const uint64_t tiles = ceil_div(env->v.N, 128);
    dev_free(env->ctx, env->pack_perm, 4ull * tiles * 128);
    dev_free(env->ctx, env->pack_tile_w, 4ull * tiles);
    for (int i = 0; i < 2; ++i)
        if (env->k_ev[i]) cudaEventDestroy(env->k_ev[i]);
    for (int i = 0; i < 5; ++i)
        if (env->split_ev[i]) cudaEventDestroy(env->split_ev[i]);
    if (env->split_stream) cudaStreamDestroy(env->split_stream);
    delete env;
}

int env_dims(const fr_env *env, int32_t *n_envs, int32_t *obs_dim, int32_t *n_assets)
{
    FR_NVTX("env_dims");
    FR_CHECK(env, FR_EINVAL, "env_dims: NULL env");
    if (n_envs) *n_envs = env->v.N;
    if (obs_dim) *obs_dim = env->v.D;
    if (n_assets) *n_assets = env->v.K;
    return FR_OK;
}

int env_reset(fr_env *env, void *stream)
{
    FR_NVTX("env_reset");
    FR_CHECK(env, FR_EINVAL, "env_reset: NULL env");
    int rc = use_device(env->ctx);
    if (rc) return rc;
    FR_CUDA(launch_env_reset(env->v, (cudaStream_t)stream));
    return FR_OK;
}

int env_step(fr_env *env, const fr_action *a, const fr_step_out *o, void *stream)
{
    FR_NVTX("env_step");
    FR_CHECK(env && a && a->data, FR_EINVAL, "env_step: NULL env or action");
    const bool stock = env->v.task == FR_TASK_STOCK;
    FR_CHECK(stock ? (a->kind == FR_ACT_I32_SHARES || a->kind == FR_ACT_F32_UNIT)
                   : a->kind == FR_ACT_U8_DISCRETE,
             FR_EINVAL, "env_step: action kind %d does not fit task %d", a->kind, env->v.task);
    int rc = use_device(env->ctx);
    if (rc) return rc;
    fr_step_out none = {nullptr, nullptr, nullptr, nullptr};
    if (!o) o = &none;
    FR_CUDA(launch_env_step(env->v, a->kind, a->data, o->rew, o->rew_f32, o->done, o->obs,
                            env->v.D, (cudaStream_t)stream));
    return FR_OK;
}

int env_observe(fr_env *env, float *obs, int32_t ld, void *stream)
{
    FR_NVTX("env_observe");
    FR_CHECK(env && obs && ld >= env->v.D, FR_EINVAL, "env_observe: need obs and ld >= D");
    int rc = use_device(env->ctx);
    if (rc) return rc;
    FR_CUDA(launch_env_observe(env->v, obs, ld, (cudaStream_t)stream));
    return FR_OK;
}

int env_get_state(fr_env *env, int64_t *cash, int32_t *hold, int32_t *steps, uint8_t *done,
                  void *stream)
{
    FR_NVTX("env_get_state");
    FR_CHECK(env, FR_EINVAL, "env_get_state: NULL env");
    int rc = use_device(env->ctx);
    if (rc) return rc;
    FR_CUDA(launch_env_get_state(env->v, cash, hold, steps, done, (cudaStream_t)stream));
    return FR_OK;
}

int env_metrics(fr_env *env, double *metrics, void *stream)
{
    FR_NVTX("env_metrics");
    FR_CHECK(env && metrics, FR_EINVAL, "env_metrics: NULL argument");
    int rc = use_device(env->ctx);
    if (rc) return rc;
    FR_CUDA(launch_env_metrics(env->v, metrics, (cudaStream_t)stream));
    return FR_OK;
}


int env_snapshot(fr_env *env, void *host_buf, size_t cap, size_t *len)
{
    FR_NVTX("env_snapshot");
    FR_CHECK(env && len, FR_EINVAL, "env_snapshot: NULL argument");
    const uint64_t off = (uint64_t)((char *)env->v.cash - (char *)env->block);
    const uint64_t sb = env->bytes - off;
    *len = sizeof(SnapHeader) + sb;
    if (!host_buf) return FR_OK;
    FR_CHECK(cap >= *len, FR_EINVAL, "env_snapshot: buffer of %zu bytes < %zu needed", cap, *len);
    int rc = use_device(env->ctx);
    if (rc) return rc;
    SnapHeader h{kSnapMagic, 1u, env->v.task, env->v.N, env->v.K, env->v.I, off, sb};
    FR_CUDA(cudaDeviceSynchronize());
    memcpy(host_buf, &h, sizeof(h));
    FR_CUDA(cudaMemcpy((char *)host_buf + sizeof(h), env->v.cash, sb, cudaMemcpyDeviceToHost));
    return FR_OK;
}

int env_restore(fr_env *env, const void *host_buf, size_t len)
{
    FR_NVTX("env_restore");
    FR_CHECK(env && host_buf && len >= sizeof(SnapHeader), FR_EINVAL, "env_restore: bad buffer");
    SnapHeader h;
    memcpy(&h, host_buf, sizeof(h));
    const uint64_t off = (uint64_t)((char *)env->v.cash - (char *)env->block);
    FR_CHECK(h.magic == kSnapMagic && h.version == 1u && h.task == env->v.task && h.N == env->v.N &&
                 h.K == env->v.K && h.I == env->v.I && h.state_off == off &&
                 h.state_bytes == env->bytes - off && len == sizeof(h) + h.state_bytes,
             FR_EINVAL, "env_restore: snapshot does not match this env's task and shape");
    int rc = use_device(env->ctx);
    if (rc) return rc;
    FR_CUDA(cudaDeviceSynchronize());
    FR_CUDA(cudaMemcpy(env->v.cash, (const char *)host_buf + sizeof(h), h.state_bytes,
                       cudaMemcpyHostToDevice));
    return FR_OK;
}

int env_set_rollout_path(fr_env *env, int32_t path)
{
    FR_NVTX("env_set_rollout_path");
    FR_CHECK(env && (path == FR_PATH_AUTO || path == FR_PATH_UNFUSED), FR_EINVAL,
             "env_set_rollout_path: bad argument");
    env->path = path;
    return FR_OK;
}

int env_set_exploration(fr_env *env, const fr_explore *x)
{
    FR_NVTX("env_set_exploration");
    FR_CHECK(env, FR_EINVAL, "env_set_exploration: NULL env");
    if (!x || x->kind == FR_EXPLORE_NONE) {
        env->explore_kind = FR_EXPLORE_NONE;
        return FR_OK;
    }
    const bool stock = env->v.task == FR_TASK_STOCK;
    FR_CHECK(stock ? x->kind == FR_EXPLORE_GAUSSIAN : x->kind == FR_EXPLORE_EPS_GREEDY, FR_EINVAL,
             "env_set_exploration: %s envs take %s exploration", stock ? "stock" : "crypto",
             stock ? "Gaussian" : "epsilon-greedy");
    FR_CHECK(x->sigma >= 0.0f && isfinite(x->sigma) && x->eps >= 0.0f && x->eps <= 1.0f, FR_EINVAL,
             "env_set_exploration: need finite sigma >= 0 and eps in [0, 1]");
    env->explore_kind = x->kind;
    env->explore_sigma = x->sigma;
    env->explore_thr = (uint32_t)((double)x->eps * 16777216.0);
    env->explore_seed = x->seed;
    return FR_OK;
}

int env_set_tile_packing(fr_env *env, int32_t on)
{
    FR_NVTX("env_set_tile_packing");
    FR_CHECK(env, FR_EINVAL, "env_set_tile_packing: NULL env");
    env->pack_off = on ? 0 : 1;
    return FR_OK;
}

int env_set_table_cache(fr_env *env, int32_t on)
{
    FR_NVTX("env_set_table_cache");
    FR_CHECK(env, FR_EINVAL, "env_set_table_cache: NULL env");
    env->z_cache_off = on ? 0 : 1;
    return FR_OK;
}

int env_set_rollout_split(fr_env *env, int32_t on)
{
    FR_NVTX("env_set_rollout_split");
    FR_CHECK(env, FR_EINVAL, "env_set_rollout_split: NULL env");
    env->split_off = on ? 0 : 1;
    return FR_OK;
}

int env_tile_packing_efficiency(const fr_env *env, float *eff)
{
    FR_NVTX("env_tile_packing_efficiency");
    FR_CHECK(env && eff, FR_EINVAL, "env_tile_packing_efficiency: NULL argument");
    *eff = env->pack_state == 2 && !env->pack_off ? env->pack_efficiency : 1.0f;
    return FR_OK;
}

int env_set_kernel_timing(fr_env *env, int32_t on)
{
    FR_NVTX("env_set_kernel_timing");
    FR_CHECK(env, FR_EINVAL, "env_set_kernel_timing: NULL env");
    int rc = use_device(env->ctx);
    if (rc) return rc;
    for (int i = 0; i < 2 && on; ++i)
        if (!env->k_ev[i]) FR_CUDA(cudaEventCreate(&env->k_ev[i]));
    env->k_timing = on ? 1 : 0;
    env->k_recorded = 0;
    return FR_OK;
}

int env_last_launch_shape(fr_env *env, int32_t *ctas, int32_t *tile_envs)
{
    FR_NVTX("env_last_launch_shape");
    FR_CHECK(env && ctas && tile_envs, FR_EINVAL, "env_last_launch_shape: NULL argument");
    FR_CHECK(env->last_ctas > 0, FR_EINVAL, "env_last_launch_shape: no fused stock rollout launched yet");
    *ctas = env->last_ctas;
    *tile_envs = env->last_tile;
    return FR_OK;
}

int env_last_kernel_ms(fr_env *env, float *ms)
{
    FR_NVTX("env_last_kernel_ms");
    FR_CHECK(env && ms, FR_EINVAL, "env_last_kernel_ms: NULL argument");
    FR_CHECK(env->k_recorded, FR_EINVAL, "env_last_kernel_ms: no kernel timed since timing was switched on");
    int rc = use_device(env->ctx);
    if (rc) return rc;
    FR_CUDA(cudaEventSynchronize(env->k_ev[1]));
    FR_CUDA(cudaEventElapsedTime(ms, env->k_ev[0], env->k_ev[1]));
    return FR_OK;
}

extern "C++" {
namespace fr {
cudaError_t set_max_smem_once(const void *func, int device)
{
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    std::lock_guard<std::mutex> lk(mu);
    for (auto &d : done)
        if (d.first == func && d.second == device) return cudaSuccess;
    int optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess) done.emplace_back(func, device);
    return e;
}

cudaError_t env_time_mark(fr_env *env, int which, cudaStream_t s)
{
    if (!env->k_timing) return cudaSuccess;
    const cudaError_t e = cudaEventRecord(env->k_ev[which], s);
    if (e == cudaSuccess && which == 1) env->k_recorded = 1;
    return e;
}
}  // namespace fr
}

int env_error_count(fr_env *env, uint64_t *count)
{
    FR_NVTX("env_error_count");
    FR_CHECK(env && count, FR_EINVAL, "env_error_count: NULL argument");
    int rc = use_device(env->ctx);
    if (rc) return rc;
    unsigned long long c = 0;
    FR_CUDA(cudaMemcpy(&c, env->v.err, 8, cudaMemcpyDeviceToHost));
    *count = c;
    return FR_OK;
}

// --------------------------------------------------------------- ensemble
int ensemble_create(fr_ctx *ctx, const fr_ensemble_desc *d, fr_ensemble **out)
{
    FR_NVTX("ensemble_create");
    FR_CHECK(ctx && d && out && d->dims && d->params, FR_EINVAL, "ensemble_create: NULL argument");
    *out = nullptr;
    FR_CHECK(d->n_agents >= 1 && d->n_agents <= MAX_AGENTS, FR_EINVAL,
             "ensemble_create: n_agents %d not in 1..8", d->n_agents);
    FR_CHECK(d->n_layers >= 1 && d->n_layers <= MAX_LAYERS, FR_EINVAL,
             "ensemble_create: n_layers %d not in 1..4", d->n_layers);
    for (int l = 0; l <= d->n_layers; ++l)
        FR_CHECK(d->dims[l] >= 1 && d->dims[l] <= 4096, FR_EINVAL, "ensemble_create: dims[%d] = %d", l,
                 d->dims[l]);
    for (int l = 1; l < d->n_layers; ++l)
        FR_CHECK(d->dims[l] <= MAX_HIDDEN, FR_EINVAL, "ensemble_create: hidden width %d > 256",
                 d->dims[l]);
    FR_CHECK(d->precision >= FR_PREC_FP32 && d->precision <= FR_PREC_FP16, FR_EINVAL,
             "ensemble_create: precision %d", d->precision);
    FR_CHECK(d->combine == FR_COMBINE_MEAN || d->combine == FR_COMBINE_VOTE, FR_EINVAL,
             "ensemble_create: combine %d", d->combine);
    uint32_t dueling = 0;
    if (d->heads) {
        for (int j = 0; j < d->n_agents; ++j) {
            FR_CHECK(d->heads[j] == FR_HEAD_Q || d->heads[j] == FR_HEAD_DUELING, FR_EINVAL,
                     "ensemble_create: heads[%d] = %d", j, d->heads[j]);
            if (d->heads[j] == FR_HEAD_DUELING) dueling |= 1u << j;
        }
    }
    FR_CHECK(!dueling || (d->combine == FR_COMBINE_VOTE && d->out_act == 0 && d->dims[d->n_layers] >= 2),
             FR_EINVAL, "ensemble_create: dueling heads need VOTE, identity output and >= 2 outputs");
    const int n_act = d->dims[d->n_layers] - (dueling ? 1 : 0);
    FR_CHECK(d->combine != FR_COMBINE_VOTE || n_act <= 3, FR_EINVAL,
             "ensemble_create: a vote needs at most 3 actions");
    int rc = use_device(ctx);
    if (rc) return rc;
    static std::atomic<uint64_t> serials{0};
    fr_ensemble *e = new (std::nothrow) fr_ensemble();
    FR_CHECK(e, FR_ENOMEM, "ensemble_create: out of host memory");
    e->serial = ++serials;
    e->ctx = ctx;
    e->M = d->n_agents;
    e->L = d->n_layers;
    for (int l = 0; l <= e->L; ++l) e->dims[l] = d->dims[l];
    e->precision = d->precision;
    e->combine = d->combine;
    e->out_act = d->out_act ? 1 : 0;
    e->dueling = dueling;
    e->n_act = n_act;
    for (int j = 0; j < MAX_AGENTS; ++j) e->heads[j] = (dueling >> j) & 1u ? FR_HEAD_DUELING : FR_HEAD_Q;
    int64_t off = 0;
    for (int l = 0; l < e->L; ++l) {
        e->w_off[l] = off;
        off += (int64_t)e->dims[l + 1] * e->dims[l];
        e->b_off[l] = off;
        off += e->dims[l + 1];
    }
    e->P = off;
    for (int j = 0; j < e->M; ++j) e->host_weights[j] = d->weights ? d->weights[j] : 1.0f / (float)e->M;
    const uint64_t pb = (uint64_t)e->M * e->P * 4;
    if ((rc = dev_alloc(ctx, (void **)&e->params, pb)) ||
        (rc = dev_alloc(ctx, (void **)&e->weights, 4ull * MAX_AGENTS))) {
        ensemble_destroy(e);
        return rc;
    }
    e->bytes = pb + 4ull * MAX_AGENTS;
    cudaError_t err = cudaMemcpy(e->params, d->params, pb, cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy(e->weights, e->host_weights, 4ull * MAX_AGENTS, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) {
        ensemble_destroy(e);
        return cuda_fail(err, "ensemble_create upload");
    }
    if (e->precision != FR_PREC_FP32) {
        rc = tc_create(e);
        if (rc) {
            ensemble_destroy(e);
            return rc;
        }
    }
    *out = e;
    return FR_OK;
}

void ensemble_destroy(fr_ensemble *e)
{
    FR_NVTX("ensemble_destroy");
    if (!e) return;
    cudaSetDevice(e->ctx->device);
    f2_release(e);
    tc_destroy(e);
    dev_free(e->ctx, e->params, (uint64_t)e->M * e->P * 4);
    dev_free(e->ctx, e->weights, 4ull * MAX_AGENTS);
    delete e;
}


int ensemble_set_act_scales(fr_ensemble *e, const float *scales)
{
    FR_NVTX("ensemble_set_act_scales");
    FR_CHECK(e && scales, FR_EINVAL, "ensemble_set_act_scales: NULL argument");
    int rc = use_device(e->ctx);
    if (rc) return rc;
    return tc_set_act_scales(e, scales);
}

int ensemble_get_act_scales(const fr_ensemble *e, float *scales)
{
    FR_NVTX("ensemble_get_act_scales");
    FR_CHECK(e && scales, FR_EINVAL, "ensemble_get_act_scales: NULL argument");
    return tc_get_act_scales(e, scales);
}

int ensemble_calibrate_sync(fr_ensemble *e, const float *obs, int32_t n, void *stream)
{
    FR_NVTX("ensemble_calibrate_sync");
    FR_CHECK(e && obs && n >= 1, FR_EINVAL, "ensemble_calibrate_sync: NULL argument or n < 1");
    FR_CHECK(e->precision == FR_PREC_FP8 && e->tc, FR_EINVAL, "ensemble_calibrate_sync: FP8 ensembles only");
    int rc = use_device(e->ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int wmax = 0;
    for (int l = 1; l < e->L; ++l) wmax = std::max(wmax, e->dims[l]);
    const uint64_t hb = 2ull * e->M * n * (uint64_t)wmax * 4;
    void *buf = nullptr;
    unsigned *amax = nullptr;
    FR_CUDA(cudaMallocAsync(&buf, hb + 4ull * MAX_AGENTS * MAX_LAYERS + 16, s));
    amax = (unsigned *)((char *)buf + hb);
    cudaError_t err = cudaMemsetAsync(amax, 0, 4ull * MAX_AGENTS * MAX_LAYERS, s);
    // activation scale = max |input| / 448 over the calibration batch, per
    // agent and layer; layer 0's input is the observation, the same for
    // every agent
    if (err == cudaSuccess) err = launch_absmax(obs, 0, (int64_t)n * e->dims[0], 1, amax, 1, s);
    // hidden layers through the fp32 master weights: ReLU outputs of layer l
    // are layer l + 1's input
    const float *in = obs;
    int64_t in_stride = 0;
    int in_ld = e->dims[0];
    for (int l = 0; l + 1 < e->L && err == cudaSuccess; ++l) {
        const int fin = e->dims[l], fout = e->dims[l + 1];
        float *out = (float *)buf + (int64_t)(l & 1) * e->M * n * wmax;
        const int64_t out_stride = (int64_t)n * fout;
        err = launch_dense_f32(in, in_stride, in_ld, e->params, e->P, e->w_off[l], e->b_off[l], out, out_stride,
                               fout, n, fin, fout, 0, e->M, s);
        if (err == cudaSuccess) err = launch_absmax(out, out_stride, out_stride, e->M, amax + l + 1, MAX_LAYERS, s);
        in = out;
        in_stride = out_stride;
        in_ld = fout;
    }
    unsigned h[MAX_AGENTS * MAX_LAYERS];
    if (err == cudaSuccess) err = cudaMemcpyAsync(h, amax, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(buf, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    FR_CUDA(err);
    float sx[MAX_AGENTS * MAX_LAYERS];
    for (int j = 0; j < e->M; ++j) {
        for (int l = 0; l < e->L; ++l) {
            // layer 0's maximum was recorded once, in slot 0
            float a;
            const unsigned bits = l == 0 ? h[0] : h[j * MAX_LAYERS + l];
            memcpy(&a, &bits, 4);
            sx[j * e->L + l] = a > 0.0f ? a / 448.0f : 1.0f;     // 448: largest finite E4M3
        }
    }
    return tc_set_act_scales(e, sx);
}

int ensemble_q(const fr_ensemble *e, const float *obs, int32_t n, float *q, void *stream)
{
    FR_NVTX("ensemble_q");
    FR_CHECK(e && n >= 0, FR_EINVAL, "ensemble_q: bad argument");
    FR_CHECK(e->combine == FR_COMBINE_VOTE, FR_EINVAL, "ensemble_q: VOTE (Q-network) ensembles only");
    if (n == 0) return FR_OK;
    FR_CHECK(obs && q, FR_EINVAL, "ensemble_q: NULL obs or q");
    int rc = use_device(e->ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int out = e->dims[e->L];
    float *y = nullptr;
    FR_CUDA(cudaMallocAsync((void **)&y, 4ull * e->M * n * out, s));
    rc = forward_any(e, obs, e->dims[0], n, y, s);
    cudaError_t err = cudaSuccess;
    if (rc == FR_OK) err = launch_heads(y, (int64_t)n * out, out, e->M, n, e->n_act, e->dueling, q, s);
    cudaFreeAsync(y, s);
    if (rc) return rc;
    FR_CUDA(err);
    return FR_OK;
}

int ensemble_q_targets(const fr_ensemble *on, const fr_ensemble *tg, const float *next_obs, const float *rew,
                       const uint8_t *done, int32_t n, float gamma, int32_t double_q, float *y, void *stream)
{
    FR_NVTX("ensemble_q_targets");
    FR_CHECK(on && tg && n >= 0, FR_EINVAL, "ensemble_q_targets: bad argument");
    FR_CHECK(on->combine == FR_COMBINE_VOTE && tg->combine == FR_COMBINE_VOTE, FR_EINVAL,
             "ensemble_q_targets: VOTE (Q-network) ensembles only");
    bool same = on->M == tg->M && on->L == tg->L && on->dueling == tg->dueling && on->ctx->device == tg->ctx->device;
    for (int l = 0; l <= on->L && same; ++l) same = on->dims[l] == tg->dims[l];
    FR_CHECK(same, FR_EINVAL, "ensemble_q_targets: online and target differ in shape or heads");
    FR_CHECK(std::isfinite(gamma), FR_EINVAL, "ensemble_q_targets: gamma not finite");
    if (n == 0) return FR_OK;
    FR_CHECK(next_obs && rew && y, FR_EINVAL, "ensemble_q_targets: NULL next_obs, rew or y");
    int rc = use_device(on->ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int out = on->dims[on->L];
    const uint64_t yb = 4ull * on->M * n * out;
    float *ys = nullptr;
    FR_CUDA(cudaMallocAsync((void **)&ys, 2 * yb, s));
    float *yon = ys, *ytg = ys + (uint64_t)on->M * n * out;
    rc = forward_any(tg, next_obs, tg->dims[0], n, ytg, s);
    if (rc == FR_OK && double_q) rc = forward_any(on, next_obs, on->dims[0], n, yon, s);
    cudaError_t err = cudaSuccess;
    if (rc == FR_OK)
        err = launch_q_targets(yon, ytg, (int64_t)n * out, out, on->M, n, on->n_act, on->dueling, rew, done, gamma,
                               double_q ? 1 : 0, y, s);
    cudaFreeAsync(ys, s);
    if (rc) return rc;
    FR_CUDA(err);
    return FR_OK;
}

int ensemble_forward(const fr_ensemble *e, const float *obs, int32_t n, float *y, void *stream)
{
    FR_NVTX("ensemble_forward");
    FR_CHECK(e && n >= 0, FR_EINVAL, "ensemble_forward: bad argument");
    if (n == 0) return FR_OK;
    FR_CHECK(obs && y, FR_EINVAL, "ensemble_forward: NULL obs or y");
    int rc = use_device(e->ctx);
    if (rc) return rc;
    return forward_any(e, obs, e->dims[0], n, y, (cudaStream_t)stream);
}

int ensemble_act(const fr_ensemble *e, const float *obs, int32_t n, void *act, void *stream)
{
    FR_NVTX("ensemble_act");
    FR_CHECK(e && n >= 0, FR_EINVAL, "ensemble_act: bad argument");
    if (n == 0) return FR_OK;
    FR_CHECK(obs && act, FR_EINVAL, "ensemble_act: NULL obs or act");
    int rc = use_device(e->ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int out = e->dims[e->L];
    float *y = nullptr;
    FR_CUDA(cudaMallocAsync((void **)&y, 4ull * e->M * n * out, s));
    rc = forward_any(e, obs, e->dims[0], n, y, s);
    cudaError_t err = cudaSuccess;
    if (!rc) {
        if (e->combine == FR_COMBINE_MEAN)
            err = launch_combine_mean(y, (int64_t)n * out, out, e->weights, e->M, n, out,
                                      (float *)act, out, s);
        else
            err = launch_combine_vote(y, (int64_t)n * out, out, e->M, n, e->n_act, e->dueling, (uint8_t *)act, s);
    }
    cudaFreeAsync(y, s);
    if (rc) return rc;
    FR_CUDA(err);
    return FR_OK;
}

// ---------------------------------------------------------------- rollout
static int plain_rollout(fr_env *env, const fr_ensemble *e, int32_t T, const fr_traj *traj, double *metrics,
                         cudaStream_t s);

int rollout(fr_env *env, const fr_ensemble *e, int32_t T, const fr_traj *traj, double *metrics,
            void *stream)
{
    FR_NVTX("rollout");
    FR_CHECK(env && e && T >= 0, FR_EINVAL, "rollout: bad argument");
    const EnvView &v = env->v;
    const bool stock = v.task == FR_TASK_STOCK;
    FR_CHECK(e->dims[0] == v.D, FR_EINVAL, "rollout: ensemble input %d != observation dim %d",
             e->dims[0], v.D);
    FR_CHECK(stock ? (e->combine == FR_COMBINE_MEAN && e->dims[e->L] == v.K)
                   : (e->combine == FR_COMBINE_VOTE && e->n_act == 3),
             FR_EINVAL, "rollout: ensemble output / combine does not fit the task");
    fr_traj none = {nullptr, 0, nullptr, nullptr, nullptr, nullptr};
    if (!traj) traj = &none;
    const int ld = traj->obs_ld ? traj->obs_ld : v.D;
    FR_CHECK(!traj->obs || ld >= v.D, FR_EINVAL, "rollout: traj obs_ld %d < D %d", ld, v.D);
    int rc = use_device(env->ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (env->path == FR_PATH_AUTO && e->precision != FR_PREC_FP32) {
        // an autotuned path when it still applies, else the default order
        const int tp = env->tune_set ? env->tune_path : -1;
        if ((tp < 0 || tp == 2) && f2_supported(env, e)) rc = f2_rollout(env, e, T, traj, metrics, s);
        else if ((tp < 0 || tp >= 1) && tc_rollout_supported(env, e)) rc = tc_rollout(env, e, T, traj, metrics, s);
        else rc = plain_rollout(env, e, T, traj, metrics, s);
    } else {
        rc = plain_rollout(env, e, T, traj, metrics, s);
    }
    if (rc == FR_OK) env->explore_step += (uint32_t)T;
    return rc;
}

// plain path: one launch per stage per step
static int plain_rollout(fr_env *env, const fr_ensemble *e, int32_t T, const fr_traj *traj, double *metrics,
                         cudaStream_t s)
{
    const EnvView &v = env->v;
    const bool stock = v.task == FR_TASK_STOCK;
    const int ld = traj->obs_ld ? traj->obs_ld : v.D;
    int rc = FR_OK;

    // plain path: one launch per stage per step
    const int N = v.N, out = e->dims[e->L];
    const uint64_t obs_b = (4ull * N * v.D + 255) & ~255ull;
    const uint64_t act_b = ((stock ? 4ull * N * v.K : (uint64_t)N) + 255) & ~255ull;
    const uint64_t y_b = (4ull * e->M * N * out + 255) & ~255ull;
    const bool tiled_ok = !(env->tune_set && !env->tune_tiled);
    const uint64_t tiles_b =
        (e->precision == FR_PREC_FP32 || !tiled_ok) ? 0 : ((tc_tiled_scratch_bytes(e, N) + 255) & ~255ull);
    const uint64_t need = obs_b + act_b + y_b + tiles_b + plain_scratch_bytes(e, N);
    if (env->scratch_bytes < need) {
        FR_CUDA(cudaStreamSynchronize(s));
        dev_free(env->ctx, env->scratch, env->scratch_bytes);
        env->scratch = nullptr;
        env->scratch_bytes = 0;
        rc = dev_alloc(env->ctx, &env->scratch, need);
        if (rc) return rc;
        env->scratch_bytes = need;
    }
    char *sc = (char *)env->scratch;
    float *obs_s = (float *)sc;
    void *act_s = sc + obs_b;
    float *y = (float *)(sc + obs_b + act_b);
    void *tiles = tiles_b ? (void *)(sc + obs_b + act_b + y_b) : nullptr;
    float *hid = (float *)(sc + obs_b + act_b + y_b + tiles_b);
    for (int t = 0; t < T; ++t) {
        const int64_t row = (int64_t)t * N;
        float *obs_t = traj->obs ? traj->obs + row * ld : obs_s;
        const int ldt = traj->obs ? ld : v.D;
        FR_CUDA(launch_env_observe(v, obs_t, ldt, s));
        if (e->precision == FR_PREC_FP32) {
            FR_CUDA(forward_plain(e, obs_t, ldt, N, y, hid, s));
        } else {
            rc = tiles ? tc_forward_tiled(e, obs_t, ldt, N, y, tiles, s) : FR_EINVAL;
            if (rc == FR_EINVAL) rc = tc_forward(e, obs_t, ldt, N, y, s);
            if (rc) return rc;
        }
        void *act_t = traj->act ? (stock ? (void *)((float *)traj->act + row * v.K)
                                         : (void *)((uint8_t *)traj->act + row))
                                : act_s;
        if (stock)
            FR_CUDA(launch_combine_mean(y, (int64_t)N * out, out, e->weights, e->M, N, out,
                                        (float *)act_t, v.K, s));
        else
            FR_CUDA(launch_combine_vote(y, (int64_t)N * out, out, e->M, N, e->n_act, e->dueling, (uint8_t *)act_t, s));
        if (env->explore_kind != FR_EXPLORE_NONE)
            FR_CUDA(launch_explore(v, act_t, explore_of(env, env->explore_step + (uint32_t)t), s));
        FR_CUDA(launch_env_step(v, stock ? FR_ACT_F32_UNIT : FR_ACT_U8_DISCRETE, act_t,
                                traj->rew ? traj->rew + row : nullptr,
                                traj->rew_f32 ? traj->rew_f32 + row : nullptr,
                                traj->done ? traj->done + row : nullptr, nullptr, 0, s));
    }
    if (metrics) FR_CUDA(launch_env_metrics(v, metrics, s));
    return FR_OK;
}

}  // extern "C"
