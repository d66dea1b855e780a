// fr_actor.cu -- the ensemble's actor MLPs at large batch (BF16 operands).
//
// Two launches:
//   * k_obs_tiles rewrites the fp32 observations once as BF16 in the
//     tensor-core operand layout, tile by tile (128 rows, K-major, 8-column
//     chunks of 2 KB), so that a CTA fetches its whole A operand with bulk
//     copies and no conversion work;
//   * k_tc_actor: one CTA per 128-row tile runs every agent of the ensemble
//     on that one A operand.  The agents' weight chunks (the same pre-packed
//     images as the single-agent kernel) stream through a multi-stage ring
//     of 1-D bulk copies; one thread issues tcgen05.mma (M = 128, N = layer
//     width, FP32 accumulator in TMEM); eight epilogue warps, two per TMEM
//     lane quarter, each take half of the layer's columns: bias (kept in
//     shared memory), ReLU and the next layer's BF16 A operand in shared
//     memory, or the agent's output.
// Limits, measured: an SM streams L2-resident data at 36 B/clk (bulk
// copies) to 43 B/clk (16-byte cp.async), and a 128-row tile consumes ~50
// B/clk of weights at full tensor rate.  Per-phase clock counters showed the
// single MMA-issuing thread, not the copies, setting the pace: a barrier
// wait and the loop around two MMAs cost ~500 cycles of issue against 256
// cycles of tensor work.  So the ring streams whole K = 16 steps in 32 KB
// stages (4 MMAs per wait for a 256-wide layer), the descriptors advance by
// constant offsets, and the epilogue keeps four TMEM loads in flight.  The
// MMAs of a layer still wait for the previous layer's epilogue.  Neither
// one weight copy delivered to all CTAs of a 4-CTA cluster nor cp.async
// producers made this kernel faster.
// The products, their order and every rounding are those of the
// single-agent kernel, so both give identical results.
#include <cuda_bf16.h>

#include <algorithm>

#include "fr_common.cuh"
#include "fr_env_dev.cuh"
#include "fr_ptx.cuh"
#include "fr_tc.cuh"

namespace fr {

namespace {

constexpr int TA_THREADS = 320;          // producer, MMA issuer, 8 epilogue warps
constexpr int TA_MAX_STAGES = 6;

struct TaLayout {
    uint32_t obs_a, h_a, ring, bias, dq, bars, total;
    int stages;
    uint32_t stage_bytes;
};

// operand bytes: 2 KB per core-matrix column of 8 (BF16) or 16 (E4M3) elements
__host__ __device__ inline uint32_t obs_tile_bytes(const TcPlan &p) { return (uint32_t)(p.layer[0].K / p.ck) * 2048u; }

__host__ __device__ inline uint32_t hidden_a_bytes(const TcPlan &p)
{
    int k = 16;
    for (int l = 1; l < p.L; ++l) k = p.layer[l].K > k ? p.layer[l].K : k;
    return (uint32_t)(k / p.ck) * 2048u;
}

__host__ __device__ inline TaLayout ta_layout(const TcPlan &p, int stages, uint32_t stage_bytes)
{
    TaLayout L;
    L.stages = stages;
    L.stage_bytes = stage_bytes;
    L.obs_a = 0;
    L.h_a = obs_tile_bytes(p);
    L.ring = L.h_a + hidden_a_bytes(p);
    L.bias = L.ring + (uint32_t)stages * stage_bytes;           // [M][L][256] fp32
    L.dq = L.bias + (uint32_t)(p.M * p.L) * 1024u;              // FP8: [M][L][256] sx * sw
    L.bars = L.dq + (p.esz == 1 ? (uint32_t)(p.M * p.L) * 1024u : 0u);
    L.total = L.bars + 256u;
    return L;
}

// fp32 obs [n][ld] (first fin columns) -> BF16 tiles [tiles][K/8][128][8]
// (the BF16 operand of the large-batch kernels), HBM-bound: a block stages
// 32 observation rows in shared memory with coalesced loads (consecutive
// threads, consecutive floats), then each thread writes 16-byte core-matrix
// rows; within a core column row r sits at byte 16 r, so a warp's 32 rows
// are 512 contiguous bytes.  Reads from the stage are conflict-free for odd
// row lengths (lanes r and r' hit banks 301 r and 301 r' mod 32).
constexpr int OT_ROWS = 32;
constexpr int OT_THREADS = 256;

__global__ void __launch_bounds__(OT_THREADS) k_obs_tiles2(const float *__restrict__ obs, int ld, int n, int fin,
                                                             int nchunks, int f16, uint4 *out)
{
    extern __shared__ float st[];                       // [OT_ROWS][fin]
    const int64_t r0 = (int64_t)blockIdx.x * OT_ROWS;
    const int rows = (int)max((int64_t)0, min((int64_t)OT_ROWS, (int64_t)n - r0));
    if (ld == fin && (((uintptr_t)obs) & 15u) == 0) {
        // packed rows: the block's rows are one span starting 16-byte aligned
        // (32 rows x fin floats is a multiple of 4 floats); float4 loads, four
        // in flight per thread, the span's tail and the rows past n scalar
        const int tot = OT_ROWS * fin, have = rows * fin, have4 = have / 4;
        const float4 *src4 = (const float4 *)(obs + r0 * ld);
        float4 *st4 = (float4 *)st;
        int i = threadIdx.x;
        for (; i + 3 * OT_THREADS < have4; i += 4 * OT_THREADS) {
            const float4 a = __ldg(src4 + i), b = __ldg(src4 + i + OT_THREADS), c = __ldg(src4 + i + 2 * OT_THREADS),
                         d = __ldg(src4 + i + 3 * OT_THREADS);
            st4[i] = a;
            st4[i + OT_THREADS] = b;
            st4[i + 2 * OT_THREADS] = c;
            st4[i + 3 * OT_THREADS] = d;
        }
        for (; i < have4; i += OT_THREADS) st4[i] = __ldg(src4 + i);
        for (int k = 4 * have4 + threadIdx.x; k < tot; k += OT_THREADS) st[k] = k < have ? __ldg(obs + r0 * ld + k) : 0.0f;
    } else {
        for (int i = threadIdx.x; i < OT_ROWS * fin; i += OT_THREADS) {
            const int r = i / fin, k = i - r * fin;
            st[i] = r < rows ? __ldg(obs + (r0 + r) * ld + k) : 0.0f;
        }
    }
    __syncthreads();
    const int64_t tile = r0 / 128;
    const int rt = (int)(r0 % 128);                     // first row's index within its tile
    for (int i = threadIdx.x; i < OT_ROWS * nchunks; i += OT_THREADS) {
        const int c = i / OT_ROWS, r = i % OT_ROWS;
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = c * 8 + u;
            v[u] = k < fin ? st[r * fin + k] : 0.0f;
        }
        uint32_t w[4];
        pack8_16(v, w, f16 != 0);
        out[(tile * nchunks + c) * 128 + rt + r] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// fp32 obs [n][ld] -> E4M3 tiles [tiles][K/16][128][16] of obs * inv (the
// agents' common layer-0 activation scale), the single-agent kernel's codes
__global__ void k_obs_tiles_e4m3(const float *__restrict__ obs, int ld, int n, int fin, int nchunks, float inv,
                                 uint4 *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tiles = (n + 127) / 128;
    if (i >= tiles * nchunks * 128) return;
    const int row = (int)(i % 128);
    const int c = (int)((i / 128) % nchunks);
    const int64_t tile = i / (128 * (int64_t)nchunks);
    const int64_t g = tile * 128 + row;
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int k = c * 16 + u;
        v[u] = (g < n && k < fin) ? __ldg(obs + g * ld + k) : 0.0f;
    }
    uint32_t w[4];
    e4m3_pack16(v, inv, w);
    out[i] = make_uint4(w[0], w[1], w[2], w[3]);
}

template <bool FP8>
__global__ void __launch_bounds__(TA_THREADS, 1)
k_tc_actor(const __grid_constant__ TcPlan plan, const uint8_t *__restrict__ img, const float *__restrict__ bias,
           const uint8_t *__restrict__ obs_tiles, int n, float *__restrict__ y, unsigned *err, int stages,
           uint32_t stage_bytes, const float *__restrict__ dq, const float *__restrict__ inv_sx)
{
    using namespace ptx;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const TaLayout L = ta_layout(plan, stages, stage_bytes);
    const uint32_t obs_a = smem_u32(base + L.obs_a), h_a = smem_u32(base + L.h_a);
    uint8_t *ring = base + L.ring;
    uint64_t *bars = (uint64_t *)(base + L.bars);
    uint64_t *full = bars;                                   // [stages]
    uint64_t *empty = bars + TA_MAX_STAGES;                  // [stages]
    uint64_t *obs_full = bars + 2 * TA_MAX_STAGES;
    uint64_t *acc_full = obs_full + 1;
    uint64_t *a_ready = obs_full + 2;
    uint64_t *drain = obs_full + 3;
    uint32_t *tmem_slot = (uint32_t *)(obs_full + 4);
    volatile int *abort = (volatile int *)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x;
    const int S = stages;
    float *bias_s = (float *)(base + L.bias);
    float *dq_s = (float *)(base + L.dq);                   // FP8 only
    constexpr bool fp8 = FP8;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(obs_full, 1);
        mbar_init(acc_full, 1);
        mbar_init(a_ready, 8);                               // one arrival per epilogue warp
        mbar_init(drain, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        __syncwarp();
        tmem_alloc(tmem_slot, (uint32_t)plan.tmem_cols);
        tmem_relinquish();
    }
    for (int i = threadIdx.x; i < plan.M * plan.L * 256; i += TA_THREADS) {
        const int j = i / (plan.L * 256), l = (i / 256) % plan.L, c = i % 256;
        bias_s[i] = bias[((size_t)j * MAX_LAYERS + l) * 256 + c];
        if (fp8) dq_s[i] = dq[((size_t)j * MAX_LAYERS + l) * 256 + c];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------- operands into the CTA
        if (lane == 0) {
            const uint32_t ob = obs_tile_bytes(plan);
            const uint8_t *src = obs_tiles + (size_t)tile * ob;
            mbar_arrive_expect_tx(obs_full, ob);
            for (uint32_t o = 0; o < ob; o += TC_CHUNK_MAX)
                bulk_g2s(base + L.obs_a + o, src + o, min(TC_CHUNK_MAX, ob - o), obs_full);
            // a layer's image is its K-major core-matrix columns end to end
            // (N x 16 bytes each, two per K = 16 step), so the ring streams it
            // in stages of whole K = 16 steps regardless of the image's chunks
            int i = 0, s = 0;
            uint32_t ph = 0;
            bool ok = true;
            for (int j = 0; j < plan.M && ok; ++j) {
                const uint8_t *aimg = img + (size_t)j * plan.agent_bytes;
                for (int l = 0; l < plan.L && ok; ++l) {
                    const TcLayer &ly = plan.layer[l];
                    const int steps = ly.K / plan.kmma, step_b = ly.N * 32, sps = (int)stage_bytes / step_b;
                    for (int k16 = 0; k16 < steps; k16 += sps, ++i) {
                        if (!mbar_wait(&empty[s], ph ^ 1u, abort, err, 1u, TC_WAIT_NS)) {
                            ok = false;
                            break;
                        }
                        const uint32_t bytes = (uint32_t)(min(sps, steps - k16) * step_b);
                        mbar_arrive_expect_tx(&full[s], bytes);
                        bulk_g2s(ring + (size_t)s * stage_bytes, aimg + ly.off + (size_t)k16 * step_b, bytes, &full[s]);
                        if (++s == S) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                }
            }
            // every copy issued lands before the CTA may exit
            volatile int no_abort = 0;
            mbar_wait(obs_full, 0u, &no_abort, err, 8u, TC_WAIT_NS);
            for (int k = i - 1; k >= 0 && k >= i - S; --k)
                mbar_wait(&full[k % S], (uint32_t)(k / S) & 1u, &no_abort, err, 8u, TC_WAIT_NS);   // stages issued
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issue
        // One thread issues every MMA, so its loop is latency-bound: the ring
        // stage and phase advance incrementally, and each layer's operand
        // descriptors are built once and advanced by constant byte offsets
        // (2 core-matrix columns of A = 4,096 B and of B = 2 N 16 B per K = 16;
        // the start-address field holds bytes / 16).
        if (lane == 0) {
            int s = 0, step = 0;
            uint32_t ph = 0;
            bool ok = mbar_wait(obs_full, 0u, abort, err, 2u, TC_WAIT_NS);
            const uint32_t ring_u = smem_u32(ring);
            for (int j = 0; j < plan.M && ok; ++j) {
                for (int l = 0; l < plan.L && ok; ++l, ++step) {
                    const TcLayer &ly = plan.layer[l];
                    // the previous layer's epilogue has read TMEM and written this A
                    if (step > 0 && !mbar_wait(a_ready, (uint32_t)(step - 1) & 1u, abort, err, 2u, TC_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t idesc = fp8 ? idesc_e4m3(128, ly.N) : idesc_bf16(128, ly.N);
                    const uint32_t lbo_b = (uint32_t)(ly.N * 16);
                    const uint64_t b_step = (uint64_t)((2u * lbo_b) >> 4);
                    uint64_t ad = smem_desc(l == 0 ? obs_a : h_a, 2048u, 128u);
                    const uint64_t bd_ring = smem_desc(ring_u, lbo_b, 128u);
                    uint32_t acc = 0u;
                    const int steps = ly.K / plan.kmma, sps = (int)stage_bytes / (ly.N * 32);
                    for (int k16 = 0; k16 < steps; k16 += sps) {
                        if (!mbar_wait(&full[s], ph, abort, err, 4u, TC_WAIT_NS)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const int n_mma = min(sps, steps - k16);
                        uint64_t bd = bd_ring + (uint64_t)(((uint32_t)s * stage_bytes) >> 4);
                        for (int u = 0; u < n_mma; ++u) {
                            if (fp8)
                                mma_e4m3(tmem, ad, bd, idesc, acc);
                            else
                                mma_bf16(tmem, ad, bd, idesc, acc);
                            acc = 1u;
                            ad += 256u;
                            bd += b_step;
                        }
                        mma_commit(&empty[s]);
                        if (++s == S) {
                            s = 0;
                            ph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    mma_commit(acc_full);
                }
            }
            // every MMA issued completes before TMEM is released
            mma_commit(drain);
            volatile int no_abort = 0;
            mbar_wait(drain, 0u, &no_abort, err, 128u, TC_WAIT_NS);
        }
    } else {
        // ------------------------------------------------------- epilogue
        const int q = warp & 3;                       // TMEM lane quarter of this warp
        const int half = (warp - 2) >> 2;             // which half of the columns
        const int r = q * 32 + lane;
        const int grow = tile * 128 + r;
        const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
        const uint32_t row_off = (uint32_t)(r / 8) * 128u + (uint32_t)(r % 8) * 16u;
        int step = 0;
        // no early exit: a wait that gives up sets the abort flag, the later
        // ones return at once, and the loop runs to its uniform end
        for (int j = 0; j < plan.M; ++j) {
            for (int l = 0; l < plan.L; ++l, ++step) {
                const TcLayer &ly = plan.layer[l];
                const bool last = l == plan.L - 1;
                warp_wait_all(acc_full, (uint32_t)step & 1u, false, abort, err, 16u, TC_WAIT_NS);
                tc_fence_after();
                const float *bl = bias_s + (j * plan.L + l) * 256;
                const float *dql = dq_s + (j * plan.L + l) * 256;                   // FP8 only
                const float inv_next = fp8 && !last ? __ldg(inv_sx + (size_t)j * MAX_LAYERS + l + 1) : 1.0f;
                // columns of this warp: two 16-aligned halves of N (a narrow
                // layer all to half 0); every group of 16 stays inside N
                const int split = ly.N >= 64 ? ((ly.N / 2 + 15) & ~15) : ly.N;
                const int c_lo = half == 0 ? 0 : split;
                const int c_hi = half == 0 ? split : ly.N;
                // up to four 16-column TMEM loads in flight per wait; the bias
                // is read as float4 (the 16-column groups are 16-aligned)
                for (int c4 = c_lo; c4 < c_hi; c4 += 64) {
                    const int g = min(4, (c_hi - c4) / 16);          // warp-uniform
                    uint32_t v[4][16];
                    __syncwarp();
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (u < g) tmem_ld16(trow + (uint32_t)(c4 + 16 * u), v[u]);
                    tmem_ld_wait();
#pragma unroll
                    for (int u4 = 0; u4 < 4; ++u4) {
                        if (u4 >= g) break;
                        const int c0 = c4 + 16 * u4;
                        float x[16];
                        const float4 *b4 = (const float4 *)(bl + c0);
                        if constexpr (FP8) {
                            // dequantise: fma(acc, sx * sw[n], b[n]); then ReLU and the next
                            // layer's E4M3 codes of x / sx' (one 16-column core column)
                            const float4 *d4 = (const float4 *)(dql + c0);
#pragma unroll
                            for (int q4 = 0; q4 < 4; ++q4) {
                                const float4 bb = b4[q4], dd = d4[q4];
                                x[4 * q4 + 0] = __fmaf_rn(__uint_as_float(v[u4][4 * q4 + 0]), dd.x, bb.x);
                                x[4 * q4 + 1] = __fmaf_rn(__uint_as_float(v[u4][4 * q4 + 1]), dd.y, bb.y);
                                x[4 * q4 + 2] = __fmaf_rn(__uint_as_float(v[u4][4 * q4 + 2]), dd.z, bb.z);
                                x[4 * q4 + 3] = __fmaf_rn(__uint_as_float(v[u4][4 * q4 + 3]), dd.w, bb.w);
                            }
                            if (!last) {
#pragma unroll
                                for (int u = 0; u < 16; ++u) x[u] = fmaxf(x[u], 0.0f);
                                uint32_t w[4];
                                e4m3_pack16(x, inv_next, w);
                                st_shared_v4(h_a + (uint32_t)(c0 / 16) * 2048u + row_off, w[0], w[1], w[2], w[3]);
                                continue;
                            }
                        } else {
#pragma unroll
                            for (int q4 = 0; q4 < 4; ++q4) {
                                const float4 bb = b4[q4];
                                x[4 * q4 + 0] = __uint_as_float(v[u4][4 * q4 + 0]) + bb.x;
                                x[4 * q4 + 1] = __uint_as_float(v[u4][4 * q4 + 1]) + bb.y;
                                x[4 * q4 + 2] = __uint_as_float(v[u4][4 * q4 + 2]) + bb.z;
                                x[4 * q4 + 3] = __uint_as_float(v[u4][4 * q4 + 3]) + bb.w;
                            }
                        }
                        if (!last) {
                            uint32_t w[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                const __nv_bfloat162 b =
                                    __floats2bfloat162_rn(fmaxf(x[2 * u], 0.0f), fmaxf(x[2 * u + 1], 0.0f));
                                w[u] = *(const uint32_t *)&b;
                            }
                            const uint32_t at = h_a + (uint32_t)(c0 / 8) * 2048u + row_off;
                            st_shared_v4(at, w[0], w[1], w[2], w[3]);
                            st_shared_v4(at + 2048u, w[4], w[5], w[6], w[7]);
                        } else if (grow < n) {
                            float *yr = y + ((size_t)j * n + grow) * ly.fout;
#pragma unroll
                            for (int u = 0; u < 16; ++u) {
                                const int col = c0 + u;
                                if (col < ly.fout) yr[col] = plan.out_act ? tanhf(x[u]) : x[u];
                            }
                        }
                    }
                }
                if (fp8 && !last && (ly.N & 31) && c_lo < c_hi && c_hi == ly.N) {
                    // the next layer's K is rounded up to 32: zero the 16 columns past N
                    st_shared_v4(h_a + (uint32_t)(ly.N / 16) * 2048u + row_off, 0u, 0u, 0u, 0u);
                }
                fence_proxy_async_smem();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(a_ready);
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, (uint32_t)plan.tmem_cols);
    }
}

// ------------------------------------------------------------------------
// k_tc_actor2: the BF16 large-batch forward, pipelined over half layers,
// with the hidden activations in tensor memory.  Persistent: CTA b takes
// tiles b, b + grid, ...; each tile's M agents are M "chains" of L layers.
//
// Each layer's outputs are computed in at most two "groups" of <= 128
// columns (a 256-wide layer in two halves), group after group for the whole
// batch.  Tensor memory (512 columns) holds two 128-column accumulator
// regions, used by groups alternately, and two 128-column BF16 operand
// buffers H0 / H1, used by hidden layers alternately (hidden layer lambda of
// the batch writes H[lambda & 1]; the next layer reads its A operand from
// there).  While the epilogue turns group g's accumulator into its half of
// the next layer's operand, the tensor cores run group g + 1; the next
// layer's first group starts on the K steps whose operand half is ready.
//
// Warps: 0 producer (observation tiles and the weight ring, one bulk copy
// per stage from the grouped weight image), 1 MMA issuer, 2.. epilogue
// (warp w reads TMEM lane quarter w % 4 and every TB_SUBS-th 16-column block
// of a group).  Producer and MMA warps run warp-uniform loops and one
// elected lane issues.  Per output element the products, their order and
// every rounding are those of k_tc_forward: identical results.
constexpr int TB_EPI_WARPS = 16;                   // four per TMEM lane quarter
constexpr int TB_SUBS = TB_EPI_WARPS / 4;          // warps sharing a lane quarter
constexpr int TB_MAXB = (8 + TB_SUBS - 1) / TB_SUBS;  // 16-column blocks per warp and group
constexpr int TB_THREADS = 64 + 32 * TB_EPI_WARPS;
constexpr int TB_MAX_STAGES = 12;

// Launch shape: observation buffers (1: the next tile loads once the last
// agent's first layer has read the buffer; 2: during the whole tile) and
// the weight ring.
struct TbShape {
    int nobs, stages;
    uint32_t stage_bytes;
};

struct TbLayout {
    uint32_t ring, bias, bars, total;
};

__host__ __device__ inline TbLayout tb_layout(const TcPlan &p, const TbShape &sh)
{
    TbLayout L;
    L.ring = (uint32_t)sh.nobs * obs_tile_bytes(p);
    L.bias = L.ring + (uint32_t)sh.stages * sh.stage_bytes;
    L.bars = L.bias + (uint32_t)(p.M * p.L) * 1024u;
    L.total = L.bars + 512u;
    return L;
}

// Output groups of a layer: one of N columns up to 128, else two halves
// (the first rounded up to 16).
__host__ __device__ inline int tb_halves(int N) { return N > 128 ? 2 : 1; }
__host__ __device__ inline int tb_h0(int N) { return N > 128 ? ((N / 2 + 15) & ~15) : N; }

// The plan runs on k_tc_actor2: BF16 (not split), every layer at most 256
// wide (so a hidden layer's BF16 output fits one 128-column buffer).
bool tb_plan_ok(const TcPlan &p)
{
    if (p.split != 1 || p.esz != 2) return false;
    for (int l = 0; l < p.L; ++l) {
        if (p.layer[l].N > 256) return false;
        if (l > 0 && p.layer[l].K > 256) return false;
    }
    return true;
}

// Launch shape for a plan: one observation buffer and two 64 KB stages
// (measured fastest: each stage handoff costs the MMA warp a barrier round
// trip, so few large stages beat many small ones), else the largest ring
// of >= 2 stages that fits.
TbShape tb_shape(const TcPlan &p, int optin)
{
    for (uint32_t sb : {65536u, 32768u, 16384u}) {
        TbShape sh{1, 2, sb};
        if (tb_layout(p, sh).total + 1024u <= (uint32_t)optin) return sh;
    }
    return TbShape{1, 0, 0u};
}

__global__ void __launch_bounds__(TB_THREADS, 1)
k_tc_actor2(const __grid_constant__ TcPlan plan, const TbShape sh, const uint8_t *__restrict__ img,
            const float *__restrict__ bias, const uint8_t *__restrict__ obs_tiles, int n, int tiles,
            float *__restrict__ y, unsigned *err)
{
    using namespace ptx;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const TbLayout Lo = tb_layout(plan, sh);
    const int S = sh.stages, NOBS = sh.nobs;
    const uint32_t SB = sh.stage_bytes;
    uint8_t *ring = base + Lo.ring;
    float *bias_s = (float *)(base + Lo.bias);
    uint64_t *bars = (uint64_t *)(base + Lo.bars);
    uint64_t *full = bars;                       // [S] weight stage landed
    uint64_t *empty = full + TB_MAX_STAGES;      // [S] weight stage read
    uint64_t *obs_full = empty + TB_MAX_STAGES;  // [NOBS]
    uint64_t *obs_empty = obs_full + 2;          // [NOBS]
    uint64_t *acc_full = obs_empty + 2;          // [2] a group's MMAs into region r are done
    uint64_t *acc_free = acc_full + 2;           // [2] the epilogue has read region r
    uint64_t *h_ready = acc_free + 2;            // [2] operand half h of the next layer written
    uint64_t *drain = h_ready + 2;
    uint32_t *tmem_slot = (uint32_t *)(drain + 1);
    volatile int *abort = (volatile int *)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ob = obs_tile_bytes(plan);
    const int M = plan.M, NL = plan.L;

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&obs_full[b], 1);
            mbar_init(&obs_empty[b], 1);
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_free[b], TB_EPI_WARPS);
            mbar_init(&h_ready[b], TB_EPI_WARPS);
        }
        mbar_init(drain, 1);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        __syncwarp();
        tmem_alloc(tmem_slot, 512u);
        tmem_relinquish();
    }
    for (int i = threadIdx.x; i < M * NL * 256; i += TB_THREADS) {
        const int j = i / (NL * 256), l = (i / 256) % NL, c = i % 256;
        bias_s[i] = bias[((size_t)j * MAX_LAYERS + l) * 256 + c];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int my_tiles = blockIdx.x < tiles ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == 0) {
        // ------------------------------------ observation tiles and weights
        // Tile k goes to buffer k % NOBS once tile k - NOBS's last first
        // layer has read it; it is only waited for when every first-layer
        // stage of that tile has been issued (so no wait is on MMAs whose
        // weights are still to come).
        int i = 0, s = 0;
        uint32_t ph = 0;
        bool ok = true;
        int next_obs = 0;
        for (int k = 0; k < my_tiles && ok; ++k) {
            for (int j = 0; j < M && ok; ++j) {
                const uint8_t *aimg = img + (size_t)j * plan.agent_bytes;      // the grouped image
                for (int l = 0; l < NL && ok; ++l) {
                    const TcLayer &ly = plan.layer[l];
                    const int nh = tb_halves(ly.N), h0 = tb_h0(ly.N), steps = ly.K / 16;
                    for (int h = 0; h < nh && ok; ++h) {
                        const int n0 = h ? h0 : 0, ng = h ? ly.N - h0 : h0;
                        const uint32_t col_b = (uint32_t)ng * 16u, kstep_b = 2u * col_b;
                        const int sps = (int)(SB / kstep_b);
                        for (int k16 = 0; k16 < steps; k16 += sps, ++i) {
                            while (next_obs < my_tiles &&
                                   (next_obs <= k + NOBS - 1 || (NOBS == 1 && next_obs == k + 1 && j == M - 1 && l >= 1))) {
                                const int kn = next_obs, b = kn % NOBS;
                                if (kn >= NOBS && !warp_wait_all(&obs_empty[b], (uint32_t)((kn - NOBS) / NOBS) & 1u,
                                                                 false, abort, err, 1u, TC_WAIT_NS)) {
                                    ok = false;
                                    break;
                                }
                                const uint8_t *src = obs_tiles + (size_t)(blockIdx.x + (size_t)kn * gridDim.x) * ob;
                                uint8_t *dst = base + (uint32_t)b * ob;
                                if (elect_one()) {
                                    mbar_arrive_expect_tx(&obs_full[b], ob);
                                    for (uint32_t o = 0; o < ob; o += TC_CHUNK_MAX)
                                        bulk_g2s(dst + o, src + o, min(TC_CHUNK_MAX, ob - o), &obs_full[b]);
                                }
                                __syncwarp();
                                ++next_obs;
                            }
                            if (!ok) break;
                            if (!warp_wait_all(&empty[s], ph ^ 1u, false, abort, err, 1u, TC_WAIT_NS)) {
                                ok = false;
                                break;
                            }
                            const int nk = min(sps, steps - k16);
                            if (elect_one()) {
                                mbar_arrive_expect_tx(&full[s], (uint32_t)nk * kstep_b);
                                // group h of the layer: rows [n0, n0 + ng), its core
                                // columns (ng x 16 bytes each) end to end
                                const uint8_t *src = aimg + ly.off + (size_t)n0 * ly.K * 2 + (size_t)k16 * kstep_b;
                                bulk_g2s(ring + (size_t)s * SB, src, (uint32_t)nk * kstep_b, &full[s]);
                            }
                            __syncwarp();
                            if (++s == S) {
                                s = 0;
                                ph ^= 1u;
                            }
                        }
                    }
                }
            }
        }
        // every copy issued lands before the CTA may exit
        volatile int no_abort = 0;
        for (int k = i - 1; k >= 0 && k >= i - S; --k)
            warp_wait_all(&full[k % S], (uint32_t)(k / S) & 1u, false, &no_abort, err, 8u, TC_WAIT_NS);
        for (int k = next_obs - 1; k >= 0 && k >= next_obs - NOBS; --k)
            warp_wait_all(&obs_full[k % NOBS], (uint32_t)(k / NOBS) & 1u, false, &no_abort, err, 8u, TC_WAIT_NS);
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issue
        int s = 0, g = 0, lam = 0;
        uint32_t ph = 0, hp0 = 0, hp1 = 0;
        bool ok = true;
        const uint32_t ring_u = smem_u32(ring);
        for (int k = 0; k < my_tiles && ok; ++k) {
            const int b = k % NOBS;
            if (!warp_wait_all(&obs_full[b], (uint32_t)(k / NOBS) & 1u, false, abort, err, 2u, TC_WAIT_NS)) break;
            const uint32_t obs_u = smem_u32(base + (uint32_t)b * ob);
            for (int j = 0; j < M && ok; ++j) {
                for (int l = 0; l < NL && ok; ++l) {
                    const TcLayer &ly = plan.layer[l];
                    const int nh = tb_halves(ly.N), h0 = tb_h0(ly.N), steps = ly.K / 16;
                    // the previous layer's operand halves: K steps [0, ksplit) need half 0
                    const int ksplit = l > 0 ? (tb_halves(plan.layer[l - 1].N) == 2 ? tb_h0(plan.layer[l - 1].N) / 16
                                                                                      : steps)
                                             : steps;
                    const uint32_t hbuf = tmem + 256u + 128u * (uint32_t)((lam - 1) & 1);
                    for (int h = 0; h < nh && ok; ++h, ++g) {
                        const int r = g & 1, n0 = h ? h0 : 0, ng = h ? ly.N - h0 : h0;
                        const uint32_t D = tmem + 128u * (uint32_t)r;
                        // region r was last read by group g - 2's epilogue
                        if (g >= 2 &&
                            !warp_wait_all(&acc_free[r], (uint32_t)((g >> 1) - 1) & 1u, false, abort, err, 2u, TC_WAIT_NS)) {
                            ok = false;
                            break;
                        }
                        const uint32_t idesc = idesc_16(128, ng, plan.f16 != 0);
                        const uint32_t col_b = (uint32_t)ng * 16u;
                        const uint64_t b_step = (uint64_t)((2u * col_b) >> 4);
                        const uint64_t bd_ring = smem_desc(ring_u, col_b, 128u);
                        const int sps = (int)(SB / (2u * col_b));
                        for (int k16 = 0; k16 < steps && ok; k16 += sps) {
                            if (!warp_wait_all(&full[s], ph, false, abort, err, 4u, TC_WAIT_NS)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const int nk = min(sps, steps - k16);
                            const uint64_t bd = bd_ring + (uint64_t)(((uint32_t)s * SB) >> 4);
                            // issue in at most two runs: an operand half may have to be waited for
                            for (int u0 = 0; u0 < nk;) {
                                const int kk = k16 + u0;
                                if (l > 0 && h == 0 && (kk == 0 || kk == ksplit)) {
                                    const bool second = kk != 0;
                                    if (!warp_wait_all(&h_ready[second ? 1 : 0], second ? hp1 : hp0, false, abort, err,
                                                       2u, TC_WAIT_NS)) {
                                        ok = false;
                                        break;
                                    }
                                    if (second)
                                        hp1 ^= 1u;
                                    else
                                        hp0 ^= 1u;
                                    tc_fence_after();
                                }
                                int u1 = nk;
                                if (l > 0 && h == 0 && kk < ksplit && k16 + nk > ksplit) u1 = ksplit - k16;
                                if (elect_one()) {
                                    for (int u = u0; u < u1; ++u) {
                                        const uint32_t kq = (uint32_t)(k16 + u);
                                        if (l == 0)
                                            mma_bf16(D, smem_desc(obs_u, 2048u, 128u) + 256u * kq, bd + b_step * (uint32_t)u,
                                                     idesc, kq ? 1u : 0u);
                                        else
                                            mma_bf16_ta(D, hbuf + 8u * kq, bd + b_step * (uint32_t)u, idesc, kq ? 1u : 0u);
                                    }
                                }
                                __syncwarp();
                                u0 = u1;
                            }
                            if (!ok) break;
                            if (elect_one()) mma_commit(&empty[s]);
                            __syncwarp();
                            if (++s == S) {
                                s = 0;
                                ph ^= 1u;
                            }
                        }
                        if (!ok) break;
                        if (elect_one()) {
                            if (l == 0 && h == nh - 1 && j == M - 1) mma_commit(&obs_empty[b]);   // tile's last obs read
                            mma_commit(&acc_full[r]);
                        }
                        __syncwarp();
                        (void)n0;
                    }
                    if (l < NL - 1) ++lam;
                }
            }
        }
        // every MMA issued completes before TMEM is released
        if (elect_one()) mma_commit(drain);
        __syncwarp();
        volatile int no_abort = 0;
        warp_wait_all(drain, 0u, false, &no_abort, err, 128u, TC_WAIT_NS);
    } else {
        // ------------------------------------------------------- epilogue
        const int q = warp & 3;                       // TMEM lane quarter (warp id mod 4)
        const int sub = (warp - 2) >> 2;              // 16-column blocks sub, sub + TB_SUBS, ...
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        int g = 0, lam = 0;
        // no early exit: a wait that gives up sets the abort flag, the later
        // ones return at once, and the loops run to their uniform end
        for (int k = 0; k < my_tiles; ++k) {
            const int row = (int)(blockIdx.x + (size_t)k * gridDim.x) * 128 + q * 32 + lane;
            for (int j = 0; j < M; ++j) {
                for (int l = 0; l < NL; ++l) {
                    const TcLayer &ly = plan.layer[l];
                    const bool last = l == NL - 1;
                    const int nh = tb_halves(ly.N), h0 = tb_h0(ly.N);
                    const uint32_t hbuf = tmem + 256u + 128u * (uint32_t)(lam & 1) + lane_off;
                    for (int h = 0; h < nh; ++h, ++g) {
                        const int r = g & 1, n0 = h ? h0 : 0, ng = h ? ly.N - h0 : h0;
                        const uint32_t D = tmem + 128u * (uint32_t)r + lane_off;
                        warp_wait_all(&acc_full[r], (uint32_t)(g >> 1) & 1u, false, abort, err, 16u, TC_WAIT_NS);
                        tc_fence_after();
                        const int G = ng / 16;
                        const int cnt = G > sub ? (G - sub + TB_SUBS - 1) / TB_SUBS : 0;   // warp-uniform
                        uint32_t v[TB_MAXB][16];
                        __syncwarp();
#pragma unroll
                        for (int u = 0; u < TB_MAXB; ++u)
                            if (u < cnt) tmem_ld16(D + (uint32_t)(16 * (sub + TB_SUBS * u)), v[u]);
                        tmem_ld_wait();
                        // the accumulator is in registers: region r is free for group g + 2
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&acc_free[r]);
                        const float *bl = bias_s + (j * NL + l) * 256 + n0;
#pragma unroll
                        for (int u = 0; u < TB_MAXB; ++u) {
                            if (u >= cnt) break;
                            const int c0 = 16 * (sub + TB_SUBS * u);
                            const float4 *b4 = (const float4 *)(bl + c0);
                            float x[16];
#pragma unroll
                            for (int q4 = 0; q4 < 4; ++q4) {
                                const float4 bb = b4[q4];
                                x[4 * q4 + 0] = __uint_as_float(v[u][4 * q4 + 0]) + bb.x;
                                x[4 * q4 + 1] = __uint_as_float(v[u][4 * q4 + 1]) + bb.y;
                                x[4 * q4 + 2] = __uint_as_float(v[u][4 * q4 + 2]) + bb.z;
                                x[4 * q4 + 3] = __uint_as_float(v[u][4 * q4 + 3]) + bb.w;
                            }
                            if (!last) {
                                uint32_t w[8];
#pragma unroll
                                if (plan.f16) {
#pragma unroll
                                    for (int e = 0; e < 8; ++e) w[e] = relu_f16x2_sat(x[2 * e], x[2 * e + 1]);
                                } else {
#pragma unroll
                                    for (int e = 0; e < 8; ++e) w[e] = relu_bf16x2(x[2 * e], x[2 * e + 1]);
                                }
                                tmem_st8(hbuf + (uint32_t)((n0 + c0) / 2), w);
                            } else if (row < n) {
                                float *yr = y + ((size_t)j * n + row) * ly.fout + n0;
#pragma unroll
                                for (int e = 0; e < 16; ++e) {
                                    const int col = n0 + c0 + e;
                                    if (col < ly.fout) yr[c0 + e] = plan.out_act ? tanhf(x[e]) : x[e];
                                }
                            }
                        }
                        if (!last) {
                            tmem_st_wait();
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&h_ready[h]);
                        }
                    }
                    if (!last) ++lam;
                }
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, 512u);
    }
}

// Ring shape: the largest stage (32 or 16 KB, at least one K = 16 step of
// the widest layer) with 2..TA_MAX_STAGES stages that fits; bigger stages
// give the single MMA-issuing thread more MMAs per barrier wait.
int ta_stages(const TcPlan &p, int optin, uint32_t *stage_bytes)
{
    if (p.split != 1) return 0;
    int nmax = 16;
    for (int l = 0; l < p.L; ++l) nmax = p.layer[l].N > nmax ? p.layer[l].N : nmax;
    for (uint32_t sb : {32768u, 16384u}) {
        if (sb < (uint32_t)nmax * 32u) continue;
        for (int s = TA_MAX_STAGES; s >= 2; --s) {
            if (ta_layout(p, s, sb).total + 1024u <= (uint32_t)optin) {
                *stage_bytes = sb;
                return s;
            }
        }
    }
    return 0;
}

}  // namespace

// 0 when this path does not apply: no BF16 plan, or fewer 128-row tiles than
// SMs (one CTA per tile would leave SMs idle; the single-agent kernel's
// tiles x agents CTAs then fill the GPU better)
uint64_t tc_tiled_scratch_bytes(const fr_ensemble *e, int n)
{
    if (!e->tc || e->tc->plan.split != 1) return 0;                          // BF16 or FP8, not split
    // FP8: one observation tile serves every agent, so they must share the
    // layer-0 activation scale (calibration always gives them the same)
    if (e->tc->plan.esz == 1 && !(e->tc->scaled && e->tc->shared_l0)) return 0;
    const int tiles = (int)ceil_div(n, 128);
    if (tiles < e->ctx->sm_count) return 0;
    return (uint64_t)tiles * obs_tile_bytes(e->tc->plan);
}

// The large-batch BF16 forward; FR_EINVAL when the plan does not fit (the
// caller then uses tc_forward).
int tc_forward_tiled(const fr_ensemble *e, const float *obs, int ld, int n, float *y, void *scratch, cudaStream_t s)
{
    const TcImage *t = e->tc;
    FR_CHECK(t && t->plan.split == 1 && scratch, FR_EINVAL, "tc_forward_tiled: needs a BF16 or FP8 plan and scratch");
    const bool fp8 = t->plan.esz == 1;
    FR_CHECK(!fp8 || (t->scaled && t->shared_l0), FR_EINVAL, "tc_forward_tiled: FP8 needs one layer-0 scale");
    const TcPlan &p = t->plan;
    int optin = 0;
    FR_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, e->ctx->device));
    // k_tc_actor2 for BF16 plans it takes, else k_tc_actor
    const TbShape sh = !fp8 && tb_plan_ok(p) && t->img2 ? tb_shape(p, optin) : TbShape{1, 0, 0u};
    uint32_t stage_bytes = 0;
    // k_tc_actor takes BF16 and FP8 operands only
    const int stages = sh.stages >= 2 || p.f16 ? 0 : ta_stages(p, optin, &stage_bytes);
    FR_CHECK(sh.stages >= 2 || stages >= 2, FR_EINVAL, "tc_forward_tiled: the plan does not fit in shared memory");
    const int tiles = (int)ceil_div(n, 128);
    const int nch = p.layer[0].K / p.ck;
    const int64_t threads = (int64_t)tiles * nch * 128;
    if (fp8)
        k_obs_tiles_e4m3<<<ceil_div(threads, 256), 256, 0, s>>>(obs, ld, n, p.layer[0].fin, nch, 1.0f / t->sx[0][0],
                                                                (uint4 *)scratch);
    else {
        // rows past n in the last tile stay zero: the 32-row blocks cover
        // whole tiles, the ones past n write zeros
        const size_t st_bytes = (size_t)OT_ROWS * p.layer[0].fin * sizeof(float);
        static_assert(128 % OT_ROWS == 0, "blocks tile the 128-row tiles");
        if (st_bytes > 48 * 1024) FR_CUDA(cudaFuncSetAttribute(k_obs_tiles2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                               (int)st_bytes));
        k_obs_tiles2<<<tiles * (128 / OT_ROWS), OT_THREADS, st_bytes, s>>>(obs, ld, n, p.layer[0].fin, nch, p.f16,
                                                                           (uint4 *)scratch);
    }
    FR_CUDA(cudaGetLastError());
    if (sh.stages >= 2) {
        const uint32_t smem2 = tb_layout(p, sh).total + 1024u;
        FR_CUDA(set_max_smem_once((const void *)k_tc_actor2, e->ctx->device));
        const int grid = std::min(tiles, e->ctx->sm_count);
        k_tc_actor2<<<grid, TB_THREADS, smem2, s>>>(p, sh, t->img2, t->bias, (const uint8_t *)scratch, n, tiles, y,
                                                    t->err);
        FR_CUDA(cudaGetLastError());
        return FR_OK;
    }
    const uint32_t smem = ta_layout(p, stages, stage_bytes).total + 1024u;
    if (fp8) {
        FR_CUDA(set_max_smem_once((const void *)k_tc_actor<true>, e->ctx->device));
        k_tc_actor<true><<<tiles, TA_THREADS, smem, s>>>(p, t->img, t->bias, (const uint8_t *)scratch, n, y, t->err,
                                                         stages, stage_bytes, t->dq, t->inv_sx);
    } else {
        FR_CUDA(set_max_smem_once((const void *)k_tc_actor<false>, e->ctx->device));
        k_tc_actor<false><<<tiles, TA_THREADS, smem, s>>>(p, t->img, t->bias, (const uint8_t *)scratch, n, y, t->err,
                                                          stages, stage_bytes, t->dq, t->inv_sx);
    }
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

}  // namespace fr
