// fr_fused.cu -- the whole rollout in one persistent kernel.
//
// One thread-block cluster owns a tile of 128 environments for all T steps;
// its CTA of rank j evaluates agent j of the ensemble (Sec. 5.2) on the tile
// with tcgen05 MMAs (weights streamed through, or resident in, a bulk-copy
// ring; accumulators in TMEM).  Every CTA of the cluster keeps the whole
// tile's env state in registers -- one thread per env -- and executes the
// identical trades, so the only data the CTAs exchange per step are the
// agents' outputs:
//   stock : each CTA pushes its tanh actions (fp16, 30 per env) into every
//           CTA's shared memory (DSMEM), double-buffered by step parity;
//           every env thread then forms the anchored weighted mean
//           (Sec. 5.2.1), discretises, trades, and builds the next
//           observation row straight into the BF16 A operand;
//   crypto: each CTA pushes its argmax (one byte per env, four rows per
//           word); every env thread takes the majority vote (Sec. 5.2.2)
//           and trades one lot.
// Stock pushes are followed by remote mbarrier arrivals (release, cluster
// scope); crypto pushes are asynchronous stores that complete transaction
// bytes on the receiving barrier.  Both are waited on with acquire at
// cluster scope.  When a step's weight chunks fit the barrier set, the
// agent's weights stay resident, packed as in its image (crypto: about
// 75 KB per CTA, three CTAs per SM).  No FP64 runs per step: each step's
// post-trade value goes to a value log, and a follow-up kernel replays the
// log in time order through the FP64 Welford / peak / drawdown accumulators.
#include <cuda_fp16.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "fr_env_dev.cuh"
#include "fr_ptx.cuh"
#include "fr_tc.cuh"

namespace fr {

namespace {

constexpr int FU_THREADS = 192;          // producer, MMA, 4 env / epilogue warps
constexpr int FU_MAX_STAGES = 6;
constexpr int SK = 30, SI = 8;           // stock market shape of the fused kernel
constexpr int SD = 1 + 2 * SK + SI * SK; // 301
constexpr int SCH = ((SD + 15) / 16) * 2; // 8-column chunks of the padded K = 304
constexpr int64_t VLOG_NONE = INT64_MIN; // frozen step: nothing happened

struct FusedArgs {
    EnvView v;
    TcPlan plan;
    const uint8_t *img;
    const float *bias;
    float w[MAX_AGENTS];
    int T;
    int stages;
    int resident;          // the agent's whole image stays in shared memory
    uint32_t ring_bytes;   // weight region: stages x TC_CHUNK_MAX, or the image
    float *tr_obs;
    int obs_ld;
    void *tr_act;
    int64_t *tr_rew;
    float *tr_rew_f32;
    uint8_t *tr_done;
    int64_t *vlog;         // [T][N]
    unsigned *err;
    Explore ex;            // exploration of the combined actions
};

__host__ __device__ inline int chunks_per_step(const TcPlan &p)
{
    int n = 0;
    for (int l = 0; l < p.L; ++l) n += p.layer[l].n_chunks;
    return n;
}

__host__ __device__ inline uint32_t xrow_bytes(int task) { return task == FR_TASK_STOCK ? 64u : 1u; }

__host__ __device__ inline uint32_t xbuf_bytes(int task, int M)
{
    return ((2u * (uint32_t)M * 128u * xrow_bytes(task)) + 15u) & ~15u;
}

__host__ __device__ inline uint32_t fused_smem(int task, const TcPlan &p, uint32_t ring_bytes)
{
    return a_part_bytes(p) * (p.split == 3 ? 2u : 1u) + ring_bytes + xbuf_bytes(task, p.M) + 256u + 1024u;
}

// Byte offset of chunk c of layer l in the agent's image; a resident copy
// keeps every chunk at this offset (the image is its chunks end to end).
__host__ __device__ inline uint32_t chunk_off(const TcPlan &p, const TcLayer &ly, int c)
{
    return ly.off + (uint32_t)c * (uint32_t)(ly.N * ly.KC * 2 * p.parts);
}

// ----------------------------------------------------- weight producer
__device__ void fused_producer(const FusedArgs &a, const uint8_t *aimg, uint8_t *ring, uint64_t *full,
                               uint64_t *empty, volatile int *abort)
{
    using namespace ptx;
    const TcPlan &p = a.plan;
    const int S = a.stages;
    const int nps = chunks_per_step(p);
    long i = 0;
    bool ok = true;
    const int steps = a.resident ? 1 : a.T;
    for (int s = 0; s < steps && ok; ++s) {
        for (int l = 0; l < p.L && ok; ++l) {
            const TcLayer &ly = p.layer[l];
            for (int c = 0; c < ly.n_chunks; ++c) {
                const int st = (int)(i % S);
                if (!a.resident &&
                    !mbar_wait(&empty[st], (uint32_t)((i / S) & 1) ^ 1u, abort, a.err, 1u, TC_WAIT_NS)) {
                    ok = false;
                    break;
                }
                const int kc = min(ly.KC, ly.K - c * ly.KC);
                const uint32_t bytes = (uint32_t)(ly.N * kc * 2 * p.parts);
                const uint32_t off = chunk_off(p, ly, c);
                mbar_arrive_expect_tx(&full[st], bytes);
                bulk_g2s(ring + (a.resident ? (size_t)off : (size_t)st * TC_CHUNK_MAX), aimg + off, bytes,
                         &full[st]);
                ++i;
            }
        }
    }
    (void)nps;
    // every copy issued must land before the CTA exits
    for (long j = i - 1; j >= 0 && j >= i - S; --j) {
        volatile int no_abort = 0;
        mbar_wait(&full[j % S], (uint32_t)((j / S) & 1), &no_abort, a.err, 8u, TC_WAIT_NS);
    }
}

// ----------------------------------------------------------- MMA issuer
__device__ void fused_mma(const FusedArgs &a, uint32_t tmem, const uint8_t *A, const uint8_t *ring,
                          uint64_t *full, uint64_t *empty, uint64_t *acc_full, uint64_t *a_ready,
                          volatile int *abort)
{
    using namespace ptx;
    const TcPlan &p = a.plan;
    const int S = a.stages;
    const bool split = p.split == 3;
    const uint32_t a_base = smem_u32(A);
    const uint32_t a_part = a_part_bytes(p);
    long i = 0;
    for (int s = 0; s < a.T; ++s) {
        int ci = 0;   // chunk index within the step (resident stages)
        for (int l = 0; l < p.L; ++l) {
            const TcLayer &ly = p.layer[l];
            if (!mbar_wait(a_ready, (uint32_t)(s * p.L + l) & 1u, abort, a.err, 2u, TC_WAIT_NS)) return;
            tc_fence_after();
            const uint32_t idesc = idesc_16(128, ly.N, p.f16 != 0);
            const uint32_t lbo_b = (uint32_t)(ly.N * 16);
            int kg = 0;
            for (int c = 0; c < ly.n_chunks; ++c, ++ci) {
                int st;
                if (a.resident) {
                    st = ci;
                    if (s == 0 && !mbar_wait(&full[st], 0u, abort, a.err, 4u, TC_WAIT_NS)) return;
                } else {
                    st = (int)(i % S);
                    if (!mbar_wait(&full[st], (uint32_t)((i / S) & 1), abort, a.err, 4u, TC_WAIT_NS)) return;
                }
                tc_fence_after();
                const int kc = min(ly.KC, ly.K - c * ly.KC);
                const uint32_t b_base =
                    smem_u32(ring + (a.resident ? (size_t)chunk_off(p, ly, c) : (size_t)st * TC_CHUNK_MAX));
                const uint32_t b_lo = (uint32_t)(ly.N * kc * 2);
                for (int kk = 0; kk < kc; kk += 16, kg += 16) {
                    const uint32_t ao = a_base + (uint32_t)(kg / 8) * 2048u;
                    const uint32_t bo = b_base + (uint32_t)(kk / 8) * lbo_b;
                    const uint64_t ad = smem_desc(ao, 2048u, 128u);
                    const uint64_t bd = smem_desc(bo, lbo_b, 128u);
                    mma_bf16(tmem, ad, bd, idesc, kg > 0 ? 1u : 0u);
                    if (split) {
                        mma_bf16(tmem, smem_desc(ao + a_part, 2048u, 128u), bd, idesc, 1u);
                        mma_bf16(tmem, ad, smem_desc(bo + b_lo, lbo_b, 128u), idesc, 1u);
                    }
                }
                if (!a.resident) mma_commit(&empty[st]);
                ++i;
            }
            mma_commit(acc_full);
        }
    }
}

// One lane of the warp waits on the barrier (the others hold no shared-
// memory polls against the tensor core's operand reads); the warp then
// continues together.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort, unsigned *err,
                                          unsigned code, bool cluster_scope)
{
    return ptx::warp_wait_all(bar, parity, cluster_scope, abort, err, code, TC_WAIT_NS);
}

// Operand format of the A buffer: BF16, BF16 hi / lo (split), or FP16.
constexpr int FMT_BF16 = 0, FMT_SPLIT = 1, FMT_F16 = 2;
__host__ __device__ inline int operand_fmt(const TcPlan &p) { return p.split == 3 ? FMT_SPLIT : (p.f16 ? FMT_F16 : FMT_BF16); }

// Eight values of row r at 8-column chunk c of the A operand.
__device__ __forceinline__ void put8(const float *v8, uint32_t a_base, uint32_t a_part, int fmt,
                                     uint32_t row_off, int c)
{
    using namespace ptx;
    const uint32_t at = a_base + (uint32_t)c * 2048u + row_off;
    uint32_t w[4];
    if (fmt == FMT_SPLIT) {
        uint32_t wl[4];
        split_pack8(v8, w, wl);
        st_shared_v4(at + a_part, wl[0], wl[1], wl[2], wl[3]);
    } else {
        pack8_16(v8, w, fmt == FMT_F16);
    }
    st_shared_v4(at, w[0], w[1], w[2], w[3]);
}

// Partial fill of a buy order (rare): kept out of line.
__device__ __noinline__ int64_t afford_out_of_line(int64_t c, int64_t p, int fee_bps)
{
    return afford(c, p, fee_bps);
}

// Eight pre-activation values x + b of row r -> ReLU -> the next layer's A
// operand chunk c.  BF16 and FP16 take the ReLU inside the conversion
// (cvt.rn.relu: max(x, 0) rounded, as max then round gives); the split
// format rounds the ReLU'd value into its hi and lo parts.
__device__ __forceinline__ void put8_relu(const float *z8, uint32_t a_base, uint32_t a_part, int fmt,
                                          uint32_t row_off, int c)
{
    using namespace ptx;
    const uint32_t at = a_base + (uint32_t)c * 2048u + row_off;
    uint32_t w[4];
    if (fmt == FMT_SPLIT) {
        float v8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v8[i] = fmaxf(z8[i], 0.0f);
        uint32_t wl[4];
        split_pack8(v8, w, wl);
        st_shared_v4(at + a_part, wl[0], wl[1], wl[2], wl[3]);
    } else if (fmt == FMT_F16) {
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = relu_f16x2_sat(z8[2 * i], z8[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = relu_bf16x2(z8[2 * i], z8[2 * i + 1]);
    }
    st_shared_v4(at, w[0], w[1], w[2], w[3]);
}

// Hidden-layer epilogue for row r: TMEM -> +bias -> ReLU -> the next layer's
// operand format, 32 columns per TMEM wait (two loads in flight), the bias
// read four columns per load (the layer's bias row is 1 KB aligned).
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem_row, const float *bl, int N, uint32_t a_base,
                                                uint32_t a_part, int fmt, uint32_t row_off)
{
    using namespace ptx;
    const float4 *bl4 = (const float4 *)bl;
    auto group8 = [&](const uint32_t *v, int c) {      // columns c .. c + 7
        const float4 b0 = __ldg(bl4 + c / 4), b1 = __ldg(bl4 + c / 4 + 1);
        const float z8[8] = {__uint_as_float(v[0]) + b0.x, __uint_as_float(v[1]) + b0.y,
                             __uint_as_float(v[2]) + b0.z, __uint_as_float(v[3]) + b0.w,
                             __uint_as_float(v[4]) + b1.x, __uint_as_float(v[5]) + b1.y,
                             __uint_as_float(v[6]) + b1.z, __uint_as_float(v[7]) + b1.w};
        put8_relu(z8, a_base, a_part, fmt, row_off, c / 8);
    };
    int c0 = 0;
    for (; c0 + 64 <= N; c0 += 64) {             // two loads in flight per wait
        uint32_t v[32], w[32];
        __syncwarp();
        tmem_ld32(tmem_row + (uint32_t)c0, v);
        tmem_ld32(tmem_row + (uint32_t)c0 + 32u, w);
        tmem_ld_wait();
#pragma unroll
        for (int g = 0; g < 4; ++g) group8(v + g * 8, c0 + g * 8);
#pragma unroll
        for (int g = 0; g < 4; ++g) group8(w + g * 8, c0 + 32 + g * 8);
    }
    for (; c0 + 32 <= N; c0 += 32) {
        uint32_t v[32];
        __syncwarp();
        tmem_ld32(tmem_row + (uint32_t)c0, v);
        tmem_ld_wait();
#pragma unroll
        for (int g = 0; g < 4; ++g) group8(v + g * 8, c0 + g * 8);
    }
    if (c0 < N) {                                   // a 16-column tail
        uint32_t v[16];
        __syncwarp();
        tmem_ld16(tmem_row + (uint32_t)c0, v);
        tmem_ld_wait();
#pragma unroll
        for (int g = 0; g < 2; ++g) group8(v + g * 8, c0 + g * 8);
    }
}

// Stock observation value at compile-time position POS of the state
// [b, p, h, f] (Sec. 3.1) for an env with Ke assets at day d.
template <int POS>
__device__ __forceinline__ float stock_obs_at(int64_t cash, const int64_t *p, const int32_t *h, int Ke,
                                              const float *ind_row)
{
    if constexpr (POS == 0) {
        return obs_scale(cash, 1e-8f);
    } else if constexpr (POS <= SK) {
        constexpr int k = POS - 1;
        return k < Ke ? obs_scale(p[k], 1e-4f) : 0.0f;
    } else if constexpr (POS <= 2 * SK) {
        constexpr int k = POS - 1 - SK;
        return k < Ke ? obs_scale(h[k], 1e-2f) : 0.0f;
    } else if constexpr (POS < SD) {
        constexpr int k = (POS - 1 - 2 * SK) % SK;
        return k < Ke ? __ldg(ind_row + (POS - 1 - 2 * SK)) : 0.0f;
    } else {
        return 0.0f;
    }
}

template <int C>
__device__ __forceinline__ void stock_obs_chunk(int64_t cash, const int64_t *p, const int32_t *h, int Ke,
                                                const float *ind_row, float *v8)
{
    v8[0] = stock_obs_at<C * 8 + 0>(cash, p, h, Ke, ind_row);
    v8[1] = stock_obs_at<C * 8 + 1>(cash, p, h, Ke, ind_row);
    v8[2] = stock_obs_at<C * 8 + 2>(cash, p, h, Ke, ind_row);
    v8[3] = stock_obs_at<C * 8 + 3>(cash, p, h, Ke, ind_row);
    v8[4] = stock_obs_at<C * 8 + 4>(cash, p, h, Ke, ind_row);
    v8[5] = stock_obs_at<C * 8 + 5>(cash, p, h, Ke, ind_row);
    v8[6] = stock_obs_at<C * 8 + 6>(cash, p, h, Ke, ind_row);
    v8[7] = stock_obs_at<C * 8 + 7>(cash, p, h, Ke, ind_row);
}

struct ObsSink {
    uint32_t a_base, a_part, row_off;
    int fmt;              // operand format (FMT_*)
    float *traj;          // fp32 trajectory row or null
};

template <int C>
__device__ __forceinline__ void stock_obs_emit(const ObsSink &o, int64_t cash, const int64_t *p,
                                               const int32_t *h, int Ke, const float *ind_row)
{
    using namespace ptx;
    float v8[8];
    stock_obs_chunk<C>(cash, p, h, Ke, ind_row, v8);
    put8(v8, o.a_base, o.a_part, o.fmt, o.row_off, C);
    if (o.traj) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (C * 8 + u < SD) o.traj[C * 8 + u] = v8[u];
    }
}

template <int C>
struct StockObsRow {
    __device__ __forceinline__ static void run(const ObsSink &o, int64_t cash, const int64_t *p,
                                               const int32_t *h, int Ke, const float *ind_row)
    {
        stock_obs_emit<C>(o, cash, p, h, Ke, ind_row);
        StockObsRow<C + 1>::run(o, cash, p, h, Ke, ind_row);
    }
};
constexpr int SCH_HEAD = 8;   // chunks 0..7 hold cash, prices, holdings (unrolled)
template <>
struct StockObsRow<SCH_HEAD> {
    __device__ __forceinline__ static void run(const ObsSink &, int64_t, const int64_t *, const int32_t *,
                                               int, const float *)
    {
    }
};

// ------------------------------------------------------------ env threads
template <int TASK>
__device__ void fused_env(const FusedArgs &a, uint32_t tmem, uint8_t *A, uint8_t *xbuf, uint64_t *acc_full,
                          uint64_t *a_ready, uint64_t *xready, volatile int *abort, int warp, int lane,
                          int agent, int tile)
{
    using namespace ptx;
    const EnvView &v = a.v;
    const TcPlan &p = a.plan;
    const int M = p.M;
    const int L = p.L;
    const int fmt = operand_fmt(p);
    const uint32_t a_base = smem_u32(A);
    const uint32_t a_part = a_part_bytes(p);
    const int q = warp & 3;                  // TMEM lane quarter
    const int r = q * 32 + lane;             // tile row == TMEM lane
    const int e = tile * 128 + r < v.N ? tile * 128 + r : -1;
    const uint32_t row_off = (uint32_t)(r / 8) * 128u + (uint32_t)(r % 8) * 16u;
    const uint32_t tmem_row = tmem + ((uint32_t)(q * 32) << 16);
    const uint32_t xrow = xrow_bytes(TASK);
    const bool w_obs = agent == 0 && a.tr_obs;
    const bool w_act = agent == 1 % M && a.tr_act;
    const bool w_rew = agent == 2 % M;
    const bool w_log = agent == 0;

    // ---- env state in registers
    int64_t cash = 0;
    int t = 0, start = 0, W = 2, Ke = 0;
    bool done = true;
    int64_t pr[SK];                           // stock: prices at day start + t
    int32_t h[SK];
    int pos = 0;                              // crypto position
    const int16_t *bps = nullptr;
#pragma unroll
    for (int k = 0; k < SK; ++k) {
        pr[k] = 0;
        h[k] = 0;
    }
    if (e >= 0) {
        cash = v.cash[e];
        t = v.t[e];
        done = v.done[e] != 0;
        start = v.start[e];
        W = v.W[e];
        if (TASK == FR_TASK_STOCK) {
            Ke = v.Ke[e];
            bps = v.bps + (int64_t)e * KP;
            const int64_t *crow = v.close + (int64_t)(start + t) * SK;
#pragma unroll
            for (int k = 0; k < SK; ++k) {
                h[k] = v.hold[(int64_t)e * KP + k];
                pr[k] = k < Ke ? perturb(__ldg(crow + k), bps[k]) : 0;
            }
        } else {
            pos = v.hold[e];
        }
    }

    for (int s = 0; s < a.T; ++s) {
        const int d = start + t;
        // ---------------------------------------------- 1. observation row
        if (TASK == FR_TASK_STOCK) {
            ObsSink o{a_base, a_part, row_off, fmt,
                      (w_obs && e >= 0) ? a.tr_obs + ((int64_t)s * v.N + e) * a.obs_ld : nullptr};
            const float *ind_row = e >= 0 ? v.ind + (int64_t)d * SI * SK : v.ind;
            const int ke = e >= 0 ? Ke : 0;
            StockObsRow<0>::run(o, e >= 0 ? cash : 0, pr, h, ke, ind_row);
            // indicator chunks, one loop: position pos reads ind_row[pos - 61]
#pragma unroll 1
            for (int c = SCH_HEAD; c < SCH; ++c) {
                float v8[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int pos = c * 8 + u;
                    const int j = pos - (1 + 2 * SK);
                    v8[u] = (pos < SD && j % SK < ke) ? __ldg(ind_row + j) : 0.0f;
                }
                put8(v8, a_base, a_part, fmt, row_off, c);
                if (o.traj) {
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (c * 8 + u < SD) o.traj[c * 8 + u] = v8[u];
                }
            }
        } else {
            float v8[8];
            float u8[8];
            const bool ok = e >= 0;
            v8[0] = ok ? obs_scale(cash, 1e-8f) : 0.0f;
            v8[1] = ok ? __fdiv_rn(__int2float_rn(pos), __int2float_rn(v.pmax)) : 0.0f;
            const float *f = v.fac + (int64_t)(ok ? d : 0) * FR_CRYPTO_FACTORS;
#pragma unroll
            for (int i = 0; i < 6; ++i) v8[2 + i] = ok ? __ldg(f + i) : 0.0f;
            u8[0] = ok ? __ldg(f + 6) : 0.0f;
            u8[1] = ok ? __ldg(f + 7) : 0.0f;
#pragma unroll
            for (int i = 2; i < 8; ++i) u8[i] = 0.0f;
            put8(v8, a_base, a_part, fmt, row_off, 0);
            put8(u8, a_base, a_part, fmt, row_off, 1);
            if (w_obs && ok) {
                float *o = a.tr_obs + ((int64_t)s * v.N + e) * a.obs_ld;
#pragma unroll
                for (int i = 0; i < 8; ++i) o[i] = v8[i];
                o[8] = u8[0];
                o[9] = u8[1];
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        mbar_arrive(a_ready);

        // ------------------------------------------------ 2. the agent's MLP
        const int b = s & 1;
        // no early exit anywhere in the step loop: a wait that gives up sets
        // the abort flag, later waits return at once and the loop runs to its
        // uniform end, so the warp stays converged at every collective
        for (int l = 0; l < L; ++l) {
            const TcLayer &ly = p.layer[l];
            warp_wait(acc_full, (uint32_t)(s * L + l) & 1u, abort, a.err, 16u, false);
            tc_fence_after();
            const float *bl = a.bias + ((size_t)agent * MAX_LAYERS + l) * 256;
            if (l < L - 1) {
                hidden_epilogue(tmem_row, bl, ly.N, a_base, a_part, fmt, row_off);
                fence_proxy_async_smem();
                tc_fence_before();
                mbar_arrive(a_ready);
                continue;
            }
            // last layer: this agent's output for row r, pushed to every CTA
            const uint32_t xoff = smem_u32(xbuf) + ((uint32_t)(b * M + agent) * 128u + (uint32_t)r) * xrow;
            if (TASK == FR_TASK_STOCK) {
                uint32_t pk[16];
                uint32_t vv[32];
                __syncwarp();
                tmem_ld32(tmem_row, vv);
                tmem_ld_wait();
#pragma unroll
                for (int c = 0; c < 32; c += 2) {
                    const float y0 = c < ly.fout ? tanhf(__uint_as_float(vv[c]) + __ldg(bl + c)) : 0.0f;
                    const float y1 = c + 1 < ly.fout ? tanhf(__uint_as_float(vv[c + 1]) + __ldg(bl + c + 1)) : 0.0f;
                    const __half2 hh = __floats2half2_rn(y0, y1);
                    pk[c / 2] = *(const uint32_t *)&hh;
                }
                for (int m = 0; m < M; ++m) {
                    const uint32_t dst = map_shared_rank(xoff, (uint32_t)m);
                    st_cluster_v4(dst, pk[0], pk[1], pk[2], pk[3]);
                    st_cluster_v4(dst + 16u, pk[4], pk[5], pk[6], pk[7]);
                    st_cluster_v4(dst + 32u, pk[8], pk[9], pk[10], pk[11]);
                    st_cluster_v4(dst + 48u, pk[12], pk[13], pk[14], pk[15]);
                }
            } else {
                uint32_t vv[16];
                __syncwarp();
                tmem_ld16(tmem_row, vv);
                tmem_ld_wait();
                float qv[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) qv[i] = __uint_as_float(vv[i]) + __ldg(bl + i);
                int best = 0;
                for (int i = 1; i < ly.fout && i < 3; ++i)
                    if (qv[i] > qv[best]) best = i;
                // four rows' bytes in one word (lane 4k holds rows 4k..4k+3):
                // this CTA's copy by a plain store, the others' by asynchronous
                // stores that complete their bytes on that CTA's barrier
                uint32_t w4 = (uint32_t)best;
                w4 |= (uint32_t)__shfl_down_sync(FULL_MASK, best, 1) << 8;
                w4 |= (uint32_t)__shfl_down_sync(FULL_MASK, best, 2) << 16;
                w4 |= (uint32_t)__shfl_down_sync(FULL_MASK, best, 3) << 24;
                if ((lane & 3) == 0) {
                    for (int m = 0; m < M; ++m) {
                        if (m == agent)
                            asm volatile("st.shared.u32 [%0], %1;" ::"r"(xoff), "r"(w4) : "memory");
                        else
                            st_async_b32(map_shared_rank(xoff, (uint32_t)m), w4,
                                         map_shared_rank(smem_u32(&xready[b]), (uint32_t)m));
                    }
                }
            }
            if (TASK == FR_TASK_STOCK) {
                __syncwarp();                              // the warp's stores precede lane 0's release
                if (lane == 0) {
                    fence_acq_rel_cluster();               // one release, then relaxed arrivals
                    for (int m = 0; m < M; ++m)
                        mbar_arrive_remote_relaxed(map_shared_rank(smem_u32(&xready[b]), (uint32_t)m));
                }
            } else {
                __syncwarp();                              // the own copy precedes the local arrival
                if (lane == 0) mbar_arrive(&xready[b]);
            }
        }
         // ----------------------------------------- 3. every agent's output in
        warp_wait(&xready[b], (uint32_t)(s >> 1) & 1u, abort, a.err, 32u, true);
        // crypto: arm this buffer's next use (step s + 2) with the other
        // CTAs' bytes; every byte of that use depends on this wait
        if (TASK == FR_TASK_CRYPTO && warp == 2 && lane == 0 && !*abort)
            mbar_arrive_expect_tx(&xready[b], (uint32_t)(M - 1) * 128u);
        if (e < 0) continue;

        // ------------------------------------ 4. combine, trade, reward, log
        const int64_t row = (int64_t)s * v.N + e;
        int64_t rew = 0, vlog = VLOG_NONE;
        bool dn_out = true;
        if (TASK == FR_TASK_STOCK) {
            const uint32_t xr = smem_u32(xbuf) + ((uint32_t)(b * M) * 128u + (uint32_t)r) * 64u;
            float act[32];
            {
                uint32_t w0[16];
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    const uint4 u = ld_shared_v4(xr + 16u * q4);
                    w0[4 * q4 + 0] = u.x; w0[4 * q4 + 1] = u.y; w0[4 * q4 + 2] = u.z; w0[4 * q4 + 3] = u.w;
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float2 f = __half22float2(*(const __half2 *)&w0[i]);
                    act[2 * i] = f.x;
                    act[2 * i + 1] = f.y;
                }
                for (int j = 1; j < M; ++j) {
                    const float wj = a.w[j];
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const uint4 u = ld_shared_v4(xr + (uint32_t)j * 128u * 64u + 16u * q4);
                        const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float2 f = __half22float2(*(const __half2 *)&uu[i]);
                            const int k = 8 * q4 + 2 * i;
                            const float a0x = __half2float(*((const __half *)&w0[4 * q4 + i]));
                            const float a0y = __half2float(*((const __half *)&w0[4 * q4 + i] + 1));
                            act[k] = __fadd_rn(act[k], __fmul_rn(wj, __fsub_rn(f.x, a0x)));
                            act[k + 1] = __fadd_rn(act[k + 1], __fmul_rn(wj, __fsub_rn(f.y, a0y)));
                        }
                    }
                }
            }
            if (a.ex.kind == FR_EXPLORE_GAUSSIAN) {
                // the executed (and recorded) action explores: a_k + sigma z_k
#pragma unroll 1
                for (int k = 0; k < SK; ++k)
                    act[k] = __fadd_rn(act[k], __fmul_rn(a.ex.sigma, explore_normal(a.ex, (uint32_t)e,
                                                                                      a.ex.g0 + (uint32_t)s,
                                                                                      (uint32_t)k)));
            }
            if (w_act) {
                float *ao = (float *)a.tr_act + row * SK;
#pragma unroll
                for (int k = 0; k < SK; ++k) ao[k] = act[k];
            }
            if (!done) {
                const int fee = v.fee_bps;
                int32_t qa[SK];
                int64_t v0 = cash;
#pragma unroll
                for (int k = 0; k < SK; ++k) {
                    bool bad;
                    qa[k] = k < Ke ? discretise(act[k], v.hmax, bad) : 0;
                    v0 += pr[k] * (int64_t)h[k];
                }
#pragma unroll
                for (int k = 0; k < SK; ++k) {                    // sells
                    if (qa[k] < 0) {
                        int64_t n = -(int64_t)qa[k];
                        if (n > h[k]) n = h[k];
                        const int64_t g = n * pr[k];
                        h[k] -= (int32_t)n;
                        cash += g - fee_of(g, fee);
                    }
                }
#pragma unroll
                for (int k = 0; k < SK; ++k) {                    // greedy buys, ascending k
                    if (qa[k] > 0) {
                        const int64_t want = qa[k];
                        const int64_t full = cost_of(want, pr[k], fee);
                        int64_t n = want;
                        int64_t c = full;
                        if (full > cash) {
                            n = afford_out_of_line(cash, pr[k], fee);
                            c = cost_of(n, pr[k], fee);
                        }
                        h[k] += (int32_t)n;
                        cash -= c;
                    }
                }
                t += 1;
                const int64_t *crow = v.close + (int64_t)(start + t) * SK;
                int64_t v1 = cash;
#pragma unroll
                for (int k = 0; k < SK; ++k) {
                    pr[k] = k < Ke ? perturb(__ldg(crow + k), bps[k]) : 0;
                    v1 += pr[k] * (int64_t)h[k];
                }
                rew = v1 - v0;
                done = t == W - 1;
                dn_out = done;
                vlog = done ? -v1 - 1 : v1;
                if (done && v.auto_reset) {
                    cash = v.init_cash;
                    t = 0;
                    done = false;
                    const int64_t *c0 = v.close + (int64_t)start * SK;
#pragma unroll
                    for (int k = 0; k < SK; ++k) {
                        h[k] = 0;
                        pr[k] = k < Ke ? perturb(__ldg(c0 + k), bps[k]) : 0;
                    }
                }
            }
        } else {
            const uint8_t *xr = xbuf + (size_t)(b * M) * 128 + r;
            int cnt[3] = {0, 0, 0};
            for (int j = 0; j < M; ++j) cnt[min((int)xr[(size_t)j * 128], 2)]++;   // clamped after an aborted wait
            int best = 0, bc = cnt[0];
            bool tie = false;
#pragma unroll
            for (int c = 1; c < 3; ++c) {
                if (cnt[c] > bc) { bc = cnt[c]; best = c; tie = false; }
                else if (cnt[c] == bc) tie = true;
            }
            int u = tie ? 1 : best;
            if (a.ex.kind == FR_EXPLORE_EPS_GREEDY) u = explore_greedy(a.ex, (uint32_t)e, a.ex.g0 + (uint32_t)s, u);
            if (w_act) ((uint8_t *)a.tr_act)[row] = (uint8_t)u;
            if (!done) {
                const int64_t m0 = __ldg(v.mid + d);
                const int64_t sp = (int64_t)__ldg(v.spread + d);
                const int64_t v0 = cash + (int64_t)pos * m0;
                const int64_t bid = m0 - sp / 2, ask = bid + sp;
                if (u == 2) {
                    if (pos < v.pmax && cash >= ask) { pos += 1; cash -= ask; }
                } else if (u == 0) {
                    if (pos > 0) { pos -= 1; cash += bid; }
                }
                t += 1;
                const int64_t v1 = cash + (int64_t)pos * __ldg(v.mid + d + 1);
                rew = v1 - v0;
                done = t == W - 1;
                dn_out = done;
                vlog = done ? -v1 - 1 : v1;
                if (done && v.auto_reset) {
                    cash = v.init_cash;
                    pos = 0;
                    t = 0;
                    done = false;
                }
            }
        }
        if (w_rew) {
            if (a.tr_rew) a.tr_rew[row] = rew;
            if (a.tr_rew_f32) a.tr_rew_f32[row] = reward_f32(rew);
            if (a.tr_done) a.tr_done[row] = dn_out ? 1 : 0;
        }
        if (w_log) a.vlog[row] = vlog;
    }

    // crypto: the other CTAs' asynchronous stores of the last two steps have
    // landed before this CTA can exit, also after a wait gave up (bounded)
    if (TASK == FR_TASK_CRYPTO && warp == 2 && lane == 0) {
        volatile int no_abort = 0;
        for (int s = a.T > 2 ? a.T - 2 : 0; s < a.T; ++s)
            mbar_wait_cluster(&xready[s & 1], (uint32_t)(s >> 1) & 1u, &no_abort, a.err, 32u, TC_WAIT_NS);
    }
    // state back to global memory (steps and accumulators: metrics pass)
    if (agent == 0 && e >= 0) {
        v.cash[e] = cash;
        v.done[e] = done ? 1 : 0;
        if (TASK == FR_TASK_STOCK) {
#pragma unroll
            for (int k = 0; k < SK; ++k) v.hold[(int64_t)e * KP + k] = h[k];
        } else {
            v.hold[e] = pos;
        }
    }
}

template <int TASK>
// Crypto tiles are small enough (resident weights ~40 KB, A operand 32 KB,
// 128 TMEM columns) for three CTAs per SM, so a 5-agent ensemble over
// 64 tiles runs in one wave.
__global__ void __launch_bounds__(FU_THREADS, TASK == FR_TASK_CRYPTO ? 3 : 1)
    k_rollout_fused(const __grid_constant__ FusedArgs a)
{
    using namespace ptx;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const TcPlan &p = a.plan;
    const int M = p.M;
    uint8_t *A = base;
    uint8_t *ring = A + a_part_bytes(p) * (p.split == 3 ? 2u : 1u);
    uint8_t *xbuf = ring + a.ring_bytes;
    uint64_t *bars = (uint64_t *)(xbuf + xbuf_bytes(TASK, M));
    uint64_t *full = bars;
    uint64_t *empty = bars + FU_MAX_STAGES;
    uint64_t *acc_full = bars + 2 * FU_MAX_STAGES;
    uint64_t *a_ready = acc_full + 1;
    uint64_t *xready = a_ready + 1;                    // [2]
    uint64_t *drain = xready + 2;                      // the issuer's last commit
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    volatile int *abort = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int agent = (int)cluster_ctarank();
    const int tile = blockIdx.y;

    if (threadIdx.x == 0) {
        for (int s = 0; s < FU_MAX_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(a_ready, 128);
        if (TASK == FR_TASK_STOCK) {
            mbar_init(&xready[0], (uint32_t)(M * 4));    // one arrival per env warp per CTA
            mbar_init(&xready[1], (uint32_t)(M * 4));
        } else {
            // this CTA's 4 env warps plus one arming arrival per use that
            // expects the other CTAs' bytes; the first use of each armed here
            mbar_init(&xready[0], 5u);
            mbar_init(&xready[1], 5u);
            mbar_arrive_expect_tx(&xready[0], (uint32_t)(M - 1) * 128u);
            mbar_arrive_expect_tx(&xready[1], (uint32_t)(M - 1) * 128u);
        }
        mbar_init(drain, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        __syncwarp();
        tmem_alloc(tmem_slot, (uint32_t)p.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    cluster_sync_all();                                // peers' barriers exist before any remote arrive
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) fused_producer(a, a.img + (size_t)agent * p.agent_bytes, ring, full, empty, abort);
    } else if (warp == 1) {
        if (lane == 0) {
            fused_mma(a, tmem, A, ring, full, empty, acc_full, a_ready, abort);
            // every MMA issued has completed before TMEM is released, also
            // when the issuer left early
            mma_commit(drain);
            volatile int no_abort = 0;
            mbar_wait(drain, 0u, &no_abort, a.err, 128u, TC_WAIT_NS);
        }
    } else {
        fused_env<TASK>(a, tmem, A, xbuf, acc_full, a_ready, xready, abort, warp, lane, agent, tile);
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, (uint32_t)p.tmem_cols);
    }
    __syncwarp();
    cluster_sync_all();                                // no peer touches this CTA's smem after exit
}

// Replays the value log through the FP64 episode accumulators in time order
// (one thread per env), advancing the step counters, latching finished
// episodes under auto-reset, and writing the metrics when asked.
__global__ void k_metrics_replay(EnvView v, const int64_t *vlog, int T, double *metrics, const int32_t *t0)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= v.N) return;
    double mu = v.mu[e], m2 = v.m2[e], mdd = v.mdd[e];
    int64_t peak = v.peak[e], vlast = v.vlast[e];
    int n = t0 ? t0[e] : v.t[e];
    double *Lt = v.latched + (int64_t)e * 4;
    for (int s = 0; s < T; ++s) {
        const int64_t x = vlog[(int64_t)s * v.N + e];
        if (x == VLOG_NONE) continue;
        const bool dn = x < 0;
        const int64_t v1 = dn ? -x - 1 : x;
        n += 1;
        const int64_t v0 = vlast;
        acc_push(mu, m2, mdd, peak, vlast, n, v0, v1);
        if (dn && v.auto_reset) {
            acc_final(mu, m2, mdd, vlast, v.init_cash, n, v.ann, Lt);
            Lt[3] = 1.0;
            mu = m2 = mdd = 0.0;
            peak = vlast = v.init_cash;
            n = 0;
        }
    }
    v.mu[e] = mu;
    v.m2[e] = m2;
    v.mdd[e] = mdd;
    v.peak[e] = peak;
    v.vlast[e] = vlast;
    v.t[e] = n;
    if (metrics) {
        double *o = metrics + (int64_t)e * 3;
        if (n == 0 && Lt[3] != 0.0) {
            o[0] = Lt[0];
            o[1] = Lt[1];
            o[2] = Lt[2];
        } else {
            acc_final(mu, m2, mdd, vlast, v.init_cash, n, v.ann, o);
        }
    }
}

// The same replay without auto-reset (one episode per env, no restarts in
// the log), with the work off the serial chain done in parallel.  A block
// takes 16 envs and walks the log in segments of 64 steps, the two phases
// pipelined (phase 1 of segment k + 1 runs while phase 2 runs on segment k):
//  * phase 1, warp-wide: warp w handles envs 2w and 2w + 1, 32 steps per
//    instruction: each valid step's return v1 / v0 - 1 (v0 the previous
//    valid step's value, carried across chunks), the running peak (a prefix
//    max), the drawdown v1 / peak - 1 below the peak and its minimum (min and
//    max are exact, so their order does not matter);
//  * phase 2, one thread per env: only the Welford chain over the stored
//    returns, mean += (r - mean) / n, m2 += (r - mean_old) (r - mean), in step
//    order -- one division per step on the dependent chain instead of three.
// Every value is computed by the same operations as acc_push, so the result
// equals the one-thread-per-env replay bit for bit.
constexpr int RP_ENVS = 16, RP_SEG = 64, RP_PROD = 8, RP_THREADS = 32 * (RP_PROD + 1);

__global__ void __launch_bounds__(RP_THREADS) k_metrics_replay2(EnvView v, const int64_t *vlog, int T, double *metrics,
                                                                 const int32_t *t0)
{
    // two segment buffers: warps 0..7 fill one (phase 1) while warp 8's
    // lanes run the Welford chains over the other (phase 2); named barriers
    // 1 + b (segment in buffer b ready) and 3 + b (buffer b read)
    __shared__ double rho_s[2][RP_ENVS][RP_SEG + 1];
    __shared__ unsigned valid_s[2][RP_ENVS][RP_SEG / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e_base = blockIdx.x * RP_ENVS;
    const int nseg = (T + RP_SEG - 1) / RP_SEG;
    // phase-2 chain state (warp RP_PROD, lanes 0..15, one env each)
    const int ce = e_base + lane;
    const bool chain = warp == RP_PROD && lane < RP_ENVS && ce < v.N;
    double mu = chain ? v.mu[ce] : 0.0, m2 = chain ? v.m2[ce] : 0.0;
    int n = chain ? (t0 ? t0[ce] : v.t[ce]) : 0;
    // phase-1 carries of this warp's two envs
    int64_t vlast_c[2], peak_c[2];
    double mdd_c[2];
    int n_c[2];
    if (warp < RP_PROD) {
        for (int q = 0; q < 2; ++q) {
            const int e = e_base + 2 * warp + q;
            const bool in = e < v.N;
            vlast_c[q] = in ? v.vlast[e] : 1;
            peak_c[q] = in ? v.peak[e] : 1;
            mdd_c[q] = in ? v.mdd[e] : 0.0;
            n_c[q] = in ? (t0 ? t0[e] : v.t[e]) : 0;
        }
        for (int k = 0; k < nseg; ++k) {
            const int b = k & 1, seg = k * RP_SEG, len = min(RP_SEG, T - seg);
            if (k >= 2) ptx::named_bar_sync(3u + (uint32_t)b, RP_THREADS);     // the chains are done with it
            for (int q = 0; q < 2; ++q) {
                const int el = 2 * warp + q, e = e_base + el;
                if (e >= v.N) continue;                                   // warp-uniform
                for (int c = 0; c < len; c += 32) {
                    const int t = seg + c + lane;
                    const int64_t x = c + lane < len ? vlog[(int64_t)t * v.N + e] : VLOG_NONE;
                    const bool valid = x != VLOG_NONE;
                    const int64_t v1 = x < 0 ? -x - 1 : x;
                    const unsigned vm = __ballot_sync(FULL_MASK, valid);
                    if (lane == 0) valid_s[b][el][c / 32] = vm;
                    if (vm == 0u) continue;
                    const unsigned below = vm & ((1u << lane) - 1u);
                    const int pl = below ? 31 - __clz(below) : 0;
                    const int64_t prev = __shfl_sync(FULL_MASK, v1, pl);
                    const int64_t v0 = below ? prev : vlast_c[q];
                    double r = 0.0;
                    if (valid) r = __dsub_rn(__ddiv_rn((double)v1, (double)v0), 1.0);
                    rho_s[b][el][c + lane] = r;
                    int64_t pk = valid ? v1 : INT64_MIN;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int64_t y = __shfl_up_sync(FULL_MASK, pk, o);
                        if (lane >= o && y > pk) pk = y;
                    }
                    if (peak_c[q] > pk) pk = peak_c[q];
                    double dmin = mdd_c[q];
                    if (valid && v1 < pk) {
                        const double dd = __dsub_rn(__ddiv_rn((double)v1, (double)pk), 1.0);
                        if (dd < dmin) dmin = dd;
                    }
#pragma unroll
                    for (int o = 16; o; o >>= 1) dmin = fmin(dmin, __shfl_xor_sync(FULL_MASK, dmin, o));
                    mdd_c[q] = dmin;
                    vlast_c[q] = __shfl_sync(FULL_MASK, v1, 31 - __clz(vm));
                    peak_c[q] = __shfl_sync(FULL_MASK, pk, 31);
                    n_c[q] += __popc(vm);
                }
            }
            ptx::named_bar_arrive(1u + (uint32_t)b, RP_THREADS);               // segment k ready
        }
        for (int q = 0; q < 2; ++q) {
            const int e = e_base + 2 * warp + q;
            if (e < v.N && lane == 0) {
                v.mdd[e] = mdd_c[q];
                v.peak[e] = peak_c[q];
                v.vlast[e] = vlast_c[q];
                if (!t0) v.t[e] = n_c[q];
            }
        }
    } else {
        for (int k = 0; k < nseg; ++k) {
            const int b = k & 1, len = min(RP_SEG, T - k * RP_SEG);
            ptx::named_bar_sync(1u + (uint32_t)b, RP_THREADS);
            if (chain) {
                for (int c = 0; c < len; ++c) {
                    if (!((valid_s[b][lane][c >> 5] >> (c & 31)) & 1u)) continue;
                    const double r = rho_s[b][lane][c];
                    n += 1;
                    const double delta = __dsub_rn(r, mu);
                    mu = __dadd_rn(mu, __ddiv_rn(delta, (double)n));
                    m2 = __dadd_rn(m2, __dmul_rn(delta, __dsub_rn(r, mu)));
                }
            }
            // the producers wait on this only for the segment two ahead
            if (k + 2 < nseg) ptx::named_bar_arrive(3u + (uint32_t)b, RP_THREADS);
        }
        if (chain) {
            v.mu[ce] = mu;
            v.m2[ce] = m2;
        }
    }
    __syncthreads();
    if (metrics && chain) {
        double *o = metrics + (int64_t)ce * 3;
        const double *Lt = v.latched + (int64_t)ce * 4;
        if (n == 0 && Lt[3] != 0.0) {
            o[0] = Lt[0];
            o[1] = Lt[1];
            o[2] = Lt[2];
        } else {
            acc_final(mu, m2, v.mdd[ce], v.vlast[ce], v.init_cash, n, v.ann, o);
        }
    }
}

// CTAs of the fused kernel one SM holds with `smem` bytes of dynamic shared
// memory: the SM's shared memory (1 KB reserved per CTA), the kernel's
// launch bounds (three crypto CTAs, one stock CTA) and its 512 TMEM columns.
int fused_per_sm(int task, const TcPlan &p, uint32_t smem, int device)
{
    int cap = 0;
    if (cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess) return 1;
    const int by_smem = cap / (int)(smem + 1024u);
    const int by_bounds = task == FR_TASK_CRYPTO ? 3 : 1;
    return std::max(1, std::min(std::min(by_smem, by_bounds), 512 / p.tmem_cols));
}

// The weight layout: resident (one barrier per chunk, the image packed end
// to end) when a step's chunks fit the barrier set and the image fits,
// unless a 2-stage streaming ring lets more CTAs share an SM (a tile runs
// all its steps on one CTA per agent, so CTAs per SM decide how many waves
// the grid takes); else the largest ring that fits.  Measured on the
// 8,192-env crypto ensemble: BF16X3 resident (1 CTA per SM) 46.9 ms,
// 2-stage ring (2 per SM) 36.2 ms; BF16 resident (3 per SM) 16.3 ms,
// 2-stage ring (3 per SM) 16.9 ms.
struct PickKey {
    int task, device, M, L, split, nps, tmem_cols;
    uint32_t agent_bytes, a_part;
    bool operator<(const PickKey &o) const
    {
        return std::tie(task, device, M, L, split, nps, tmem_cols, agent_bytes, a_part) <
               std::tie(o.task, o.device, o.M, o.L, o.split, o.nps, o.tmem_cols, o.agent_bytes, o.a_part);
    }
};
struct PickVal {
    int stages, resident;
    uint32_t ring_bytes;
};

int pick_stages(int task, const TcPlan &p, int optin, int device, int *resident, uint32_t *ring_bytes)
{
    // cached per kernel shape: the device queries run on a first call,
    // never inside a later stream capture
    static std::mutex mu;
    static std::map<PickKey, PickVal> cache;
    const int nps = chunks_per_step(p);
    const PickKey key{task, device, p.M, p.L, p.split, nps, p.tmem_cols, p.agent_bytes, a_part_bytes(p)};
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *resident = it->second.resident;
            *ring_bytes = it->second.ring_bytes;
            return it->second.stages;
        }
    }
    int best = 0;
    const uint32_t ring2 = 2u * TC_CHUNK_MAX;
    if (nps <= FU_MAX_STAGES && fused_smem(task, p, p.agent_bytes) <= (uint32_t)optin) {
        best = nps;
        *resident = 1;
        *ring_bytes = p.agent_bytes;
        if (fused_smem(task, p, ring2) <= (uint32_t)optin &&
            fused_per_sm(task, p, fused_smem(task, p, ring2), device) >
                fused_per_sm(task, p, fused_smem(task, p, p.agent_bytes), device)) {
            best = 2;
            *resident = 0;
            *ring_bytes = ring2;
        }
    } else {
        for (int st = FU_MAX_STAGES; st >= 2; --st) {
            if (fused_smem(task, p, (uint32_t)st * TC_CHUNK_MAX) <= (uint32_t)optin) {
                best = st;
                *resident = 0;
                *ring_bytes = (uint32_t)st * TC_CHUNK_MAX;
                break;
            }
        }
    }
    if (best > 0) {
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = PickVal{best, *resident, *ring_bytes};
    }
    return best;
}

}  // namespace

bool tc_rollout_supported(const fr_env *env, const fr_ensemble *e)
{
    if (!e->tc || e->M > 8 || e->tc->plan.esz != 2 || e->dueling) return false;   // BF16, plain heads
    const EnvView &v = env->v;
    const TcPlan &p = e->tc->plan;
    if (v.task == FR_TASK_STOCK) {
        if (v.K != SK || v.I != SI || e->combine != FR_COMBINE_MEAN || e->dims[0] != SD ||
            e->dims[e->L] != SK || e->out_act != 1 || v.buy_order != FR_BUY_ASCENDING)
            return false;
    } else {
        if (e->combine != FR_COMBINE_VOTE || e->dims[0] != FR_CRYPTO_OBS_DIM || e->dims[e->L] != 3 ||
            p.KA > 512)
            return false;
    }
    int optin = 0, resident = 0;
    uint32_t ring_bytes = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, env->ctx->device) !=
        cudaSuccess)
        return false;
    return pick_stages(v.task, p, optin, env->ctx->device, &resident, &ring_bytes) > 0;
}

// The first fused kernel's largest ring for this pair (0: the kernel does not
// apply) and the chunks of one step (the ring holds the weights resident when
// it has at least that many stages).
int tc_rollout_max_stages(const fr_env *env, const fr_ensemble *e, int *chunks_per_step_out)
{
    if (!tc_rollout_supported(env, e)) return 0;
    int optin = 0, resident = 0;
    uint32_t ring_bytes = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, env->ctx->device) != cudaSuccess)
        return 0;
    *chunks_per_step_out = chunks_per_step(e->tc->plan);
    return pick_stages(env->v.task, e->tc->plan, optin, env->ctx->device, &resident, &ring_bytes);
}

int tc_rollout(fr_env *env, const fr_ensemble *e, int T, const fr_traj *traj, double *metrics,
               cudaStream_t s)
{
    const EnvView &v = env->v;
    const TcPlan &p = e->tc->plan;
    int optin = 0, resident = 0;
    uint32_t ring_bytes = 0;
    FR_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, env->ctx->device));
    int stages = pick_stages(v.task, p, optin, env->ctx->device, &resident, &ring_bytes);
    FR_CHECK(stages > 0, FR_EINVAL, "fused rollout: plan does not fit in shared memory");
    if (env->tune_set && env->tune_stages >= 2 && env->tune_stages < stages) {
        // an autotuned ring: fewer stages, the weights streamed
        stages = env->tune_stages;
        resident = 0;
        ring_bytes = (uint32_t)stages * TC_CHUNK_MAX;
    }
    if (T == 0) {
        if (metrics) FR_CUDA(launch_env_metrics(v, metrics, s));
        return FR_OK;
    }
    // value log [T][N] in the env's scratch (grown outside any timed region)
    const uint64_t need = (uint64_t)T * v.N * 8;
    if (env->scratch_bytes < need) {
        FR_CUDA(cudaStreamSynchronize(s));
        dev_free(env->ctx, env->scratch, env->scratch_bytes);
        env->scratch = nullptr;
        env->scratch_bytes = 0;
        int rc = dev_alloc(env->ctx, &env->scratch, need);
        if (rc) return rc;
        env->scratch_bytes = need;
    }
    FusedArgs a;
    memset(&a, 0, sizeof(a));
    a.v = v;
    a.plan = p;
    a.img = e->tc->img;
    a.bias = e->tc->bias;
    for (int j = 0; j < MAX_AGENTS; ++j) a.w[j] = e->host_weights[j];
    a.T = T;
    a.stages = stages;
    a.resident = resident;
    a.ring_bytes = ring_bytes;
    a.tr_obs = traj->obs;
    a.obs_ld = traj->obs_ld ? traj->obs_ld : v.D;
    a.tr_act = traj->act;
    a.tr_rew = traj->rew;
    a.tr_rew_f32 = traj->rew_f32;
    a.tr_done = traj->done;
    a.vlog = (int64_t *)env->scratch;
    a.err = e->tc->err;
    a.ex = explore_of(env, env->explore_step);

    const uint32_t smem = fused_smem(v.task, p, ring_bytes);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p.M, ceil_div(v.N, 128), 1);
    cfg.blockDim = dim3(FU_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)p.M;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    FR_CUDA(env_time_mark(env, 0, s));
    if (v.task == FR_TASK_STOCK) {
        FR_CUDA(set_max_smem_once((const void *)k_rollout_fused<FR_TASK_STOCK>, env->ctx->device));
        FR_CUDA(cudaLaunchKernelEx(&cfg, k_rollout_fused<FR_TASK_STOCK>, a));
    } else {
        FR_CUDA(set_max_smem_once((const void *)k_rollout_fused<FR_TASK_CRYPTO>, env->ctx->device));
        FR_CUDA(cudaLaunchKernelEx(&cfg, k_rollout_fused<FR_TASK_CRYPTO>, a));
    }
    FR_CUDA(env_time_mark(env, 1, s));
    FR_CUDA(launch_metrics_replay(v, a.vlog, T, metrics, s));
    return FR_OK;
}

cudaError_t launch_metrics_replay(const EnvView &v, const int64_t *vlog, int T, double *metrics,
                                  cudaStream_t s, const int32_t *t0)
{
    if (!v.auto_reset) {
        k_metrics_replay2<<<ceil_div(v.N, RP_ENVS), RP_THREADS, 0, s>>>(v, vlog, T, metrics, t0);
        return cudaGetLastError();
    }
    // auto-reset: one thread per env, spread over every SM: the replay is
    // bound by the FP64 units, and 2,048 envs in blocks of 256 would use 8 SMs
    const int per_block = std::min(256, std::max(16, (int)ceil_div(v.N, 152) + 15) / 16 * 16);
    k_metrics_replay<<<ceil_div(v.N, per_block), per_block, 0, s>>>(v, vlog, T, metrics, t0);
    return cudaGetLastError();
}

}  // namespace fr
