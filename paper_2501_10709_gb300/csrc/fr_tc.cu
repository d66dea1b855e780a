// fr_tc.cu -- the ensemble's actor MLPs on the 5th-generation tensor cores.
//
// One CTA computes one agent's network (Sec. 6.1: dense layers, ReLU hidden
// activations) for a tile of 128 observation rows:
//   * the weights are pre-packed on the host into BF16 "chunks" laid out
//     exactly as the tcgen05 K-major no-swizzle canonical form, and a
//     producer warp streams them from global memory (L2-resident) into a
//     two-stage shared-memory ring with 1-D bulk copies (TMA);
//   * one thread issues tcgen05.mma (M = 128, N = layer width, K = 16 per
//     instruction) with the FP32 accumulator in tensor memory (TMEM);
//   * four epilogue warps read the accumulator back with tcgen05.ld, add the
//     bias, apply ReLU, and write the next layer's A operand (BF16) straight
//     into shared memory; the last layer applies tanh or identity.
// With FP8 E4M3 operands the MMA is kind::f8f6f4 (K = 32 per instruction),
// the epilogue dequantises with the per-channel factor sx * sw before the
// bias and quantises the next layer's input with the agent's activation scale.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fr_common.cuh"
#include "fr_ptx.cuh"
#include "fr_tc.cuh"

namespace fr {

namespace {

inline int round16(int x) { return (x + 15) & ~15; }

inline uint16_t f32_to_bf16_rne(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0xffffu) ? 0x40u : 0u));
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
}

// FP16 bits of f, round to nearest even, saturating at +-65504 (NaN stays NaN).
inline uint16_t f32_to_f16_sat(float f)
{
    if (!(std::fabs(f) <= 65504.0f)) f = std::isnan(f) ? f : (f > 0.0f ? 65504.0f : -65504.0f);
    const __half h = __float2half_rn(f);
    uint16_t u;
    memcpy(&u, &h, 2);
    return u;
}

inline float bf16_to_f32(uint16_t b)
{
    const uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// byte offset of element (n, kk) inside a chunk of a layer with N rows, for
// ck elements (of esz bytes) per core-matrix row
inline uint32_t chunk_off(int N, int n, int kk, int ck, int esz)
{
    return (uint32_t)((kk / ck) * (N * 16) + (n / 8) * 128 + (n % 8) * 16 + (kk % ck) * esz);
}

bool make_plan(const fr_ensemble *e, TcPlan &p)
{
    p.split = e->precision == FR_PREC_BF16X3 ? 3 : 1;
    p.f16 = e->precision == FR_PREC_FP16 ? 1 : 0;
    p.parts = p.split == 3 ? 2 : 1;
    const bool fp8 = e->precision == FR_PREC_FP8;
    p.esz = fp8 ? 1 : 2;
    p.kmma = fp8 ? 32 : 16;
    p.ck = fp8 ? 16 : 8;
    p.M = e->M;
    p.L = e->L;
    p.out_act = e->out_act;
    p.KA = 0;
    int nmax = 0;
    uint32_t off = 0;
    for (int l = 0; l < e->L; ++l) {
        TcLayer &ly = p.layer[l];
        ly.fin = e->dims[l];
        ly.fout = e->dims[l + 1];
        ly.K = (ly.fin + p.kmma - 1) / p.kmma * p.kmma;
        ly.N = round16(ly.fout);
        if (ly.N > 256 || ly.K > 512) return false;
        int kc = (int)(TC_CHUNK_MAX / (uint32_t)(ly.N * p.esz * p.parts));
        kc = kc / p.kmma * p.kmma;
        ly.KC = kc < ly.K ? kc : ly.K;
        ly.n_chunks = (ly.K + ly.KC - 1) / ly.KC;
        ly.off = off;
        off += (uint32_t)ly.N * ly.K * p.esz * p.parts;
        p.KA = ly.K > p.KA ? ly.K : p.KA;
        nmax = ly.N > nmax ? ly.N : nmax;
    }
    p.agent_bytes = (off + 1023u) & ~1023u;
    int c = 32;
    while (c < nmax) c <<= 1;
    p.tmem_cols = c;
    return true;
}

// Ring stage of the single-agent kernel.  Without split operands a layer's
// image is its K-major core-matrix columns end to end, streamed in stages of
// whole MMA steps (N x 32 bytes each: two core columns); 32 KB stages give the
// MMA-issuing thread up to four MMAs per barrier wait on a 256-wide layer.
// Split (hi / lo) images keep one chunk per stage.
inline __host__ __device__ uint32_t tc_stage_bytes(const TcPlan &p) { return p.split == 3 ? TC_CHUNK_MAX : 32768u; }

uint32_t tc_smem_bytes(const TcPlan &p)
{
    return a_part_bytes(p) * (p.split == 3 ? 2u : 1u) + TC_STAGES * tc_stage_bytes(p) + 256u + 1024u;
}

// Geometry of weight-stream unit u of layer ly: its bytes, its offset in the
// layer's image, its MMAs and (split images) the lo part's offset within it.
struct TcUnit {
    uint32_t bytes, src, lo;
    int n_mma;
};
__device__ __forceinline__ int tc_units(const TcPlan &p, const TcLayer &ly)
{
    if (p.split == 3) return ly.n_chunks;
    const int steps = ly.K / p.kmma, sps = (int)(tc_stage_bytes(p) / (uint32_t)(ly.N * 32));
    return (steps + sps - 1) / sps;
}
__device__ __forceinline__ TcUnit tc_unit(const TcPlan &p, const TcLayer &ly, int u)
{
    TcUnit t;
    if (p.split == 3) {
        const int kc = min(ly.KC, ly.K - u * ly.KC);
        t.bytes = (uint32_t)(ly.N * kc * 2 * 2);
        t.src = (uint32_t)(u * ly.N * ly.KC * 2 * 2);
        t.lo = (uint32_t)(ly.N * kc * 2);
        t.n_mma = kc / 16;
    } else {
        const int steps = ly.K / p.kmma, step_b = ly.N * 32, sps = (int)(tc_stage_bytes(p) / (uint32_t)step_b);
        const int k0 = u * sps;
        t.n_mma = min(sps, steps - k0);
        t.bytes = (uint32_t)(t.n_mma * step_b);
        t.src = (uint32_t)(k0 * step_b);
        t.lo = 0;
    }
    return t;
}

// ------------------------------------------------------------------ kernel
__global__ void __launch_bounds__(TC_THREADS) k_tc_forward(TcPlan plan, const uint8_t *__restrict__ img,
                                                            const float *__restrict__ bias,
                                                            const float *__restrict__ dq,
                                                            const float *__restrict__ inv_sx,
                                                            const float *__restrict__ obs, int ld, int n,
                                                            float *__restrict__ y, unsigned *err)
{
    using namespace ptx;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *A = base;
    const uint32_t a_part = a_part_bytes(plan);                  // bytes of one A part
    const bool split = plan.split == 3;
    const bool fp8 = plan.esz == 1;
    uint8_t *ring = A + a_part * (split ? 2u : 1u);
    const uint32_t stage_b = tc_stage_bytes(plan);
    uint64_t *bars = (uint64_t *)(ring + TC_STAGES * stage_b);
    uint64_t *full = bars;
    uint64_t *empty = bars + TC_STAGES;
    uint64_t *acc_full = bars + 2 * TC_STAGES;
    uint64_t *a_ready = acc_full + 1;
    uint32_t *tmem_slot = (uint32_t *)(a_ready + 1);
    volatile int *abort = (volatile int *)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = blockIdx.x * 128;
    const int agent = blockIdx.y;
    const uint8_t *aimg = img + (size_t)agent * plan.agent_bytes;

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(a_ready, 128);
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        __syncwarp();
        tmem_alloc(tmem_slot, (uint32_t)plan.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ weight producer
        if (lane == 0) {
            int i = 0;
            bool ok = true;
            for (int l = 0; l < plan.L && ok; ++l) {
                const TcLayer &ly = plan.layer[l];
                const int nu = tc_units(plan, ly);
                for (int c = 0; c < nu; ++c) {
                    const int s = i % TC_STAGES;
                    const uint32_t ph = (uint32_t)(i / TC_STAGES) & 1u;
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort, err, 1u, TC_WAIT_NS)) { ok = false; break; }
                    const TcUnit un = tc_unit(plan, ly, c);
                    mbar_arrive_expect_tx(&full[s], un.bytes);
                    bulk_g2s(ring + s * stage_b, aimg + ly.off + un.src, un.bytes, &full[s]);
                    ++i;
                }
            }
            // every copy issued must land before the CTA may exit
            for (int j = i - 1; j >= 0 && j >= i - TC_STAGES; --j) {
                volatile int no_abort = 0;
                mbar_wait(&full[j % TC_STAGES], (uint32_t)(j / TC_STAGES) & 1u, &no_abort, err, 8u,
                          TC_WAIT_NS);
            }
        }
    } else if (warp == 1) {
        // -------------------------------------------------- MMA issuer
        // one thread issues every MMA: the descriptors are built once per
        // stage and advanced by constant offsets (two core-matrix columns per
        // MMA: 4,096 B of A and 2 N 16 B of B, in 16-byte units), and the
        // stage and phase advance incrementally
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0;
            const uint32_t a_base = smem_u32(A);
            const uint32_t ring_u = smem_u32(ring);
            const uint64_t a_lo = (uint64_t)(a_part >> 4);
            for (int l = 0; l < plan.L; ++l) {
                const TcLayer &ly = plan.layer[l];
                if (!mbar_wait(a_ready, (uint32_t)l & 1u, abort, err, 2u, TC_WAIT_NS)) break;
                tc_fence_after();
                const uint32_t idesc = fp8 ? idesc_e4m3(128, ly.N) : idesc_16(128, ly.N, plan.f16 != 0);
                const uint32_t lbo_b = (uint32_t)(ly.N * 16);
                const uint64_t b_step = (uint64_t)((2u * lbo_b) >> 4);
                const int nu = tc_units(plan, ly);
                uint64_t ad = smem_desc(a_base, 2048u, 128u);
                uint32_t accum = 0u;
                bool ok = true;
                for (int c = 0; c < nu; ++c) {
                    if (!mbar_wait(&full[s], ph, abort, err, 4u, TC_WAIT_NS)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const TcUnit un = tc_unit(plan, ly, c);
                    uint64_t bd = smem_desc(ring_u + (uint32_t)s * stage_b, lbo_b, 128u);
                    const uint64_t b_lo = (uint64_t)(un.lo >> 4);
                    for (int u = 0; u < un.n_mma; ++u) {
                        if (fp8) {
                            mma_e4m3(tmem, ad, bd, idesc, accum);
                        } else {
                            mma_bf16(tmem, ad, bd, idesc, accum);
                        }
                        if (split) {
                            mma_bf16(tmem, ad + a_lo, bd, idesc, 1u);
                            mma_bf16(tmem, ad, bd + b_lo, idesc, 1u);
                        }
                        accum = 1u;
                        ad += 256u;
                        bd += b_step;
                    }
                    mma_commit(&empty[s]);
                    if (++s == TC_STAGES) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(acc_full);
            }
        }
    } else {
        // ------------------------------------------------------ epilogue
        const int q = warp & 3;                 // TMEM lane quarter of this warp
        const int r = q * 32 + lane;            // row of the tile owned by this thread
        const int grow = row0 + r;
        const uint32_t a_base = smem_u32(A);
        // observation tile -> BF16 (or E4M3) A operand, one row at a time per warp
        const TcLayer &l0 = plan.layer[0];
        const float *qa = inv_sx + (size_t)agent * MAX_LAYERS;        // FP8 only
        for (int rr = 0; rr < 32 && fp8; ++rr) {
            const int row = q * 32 + rr;
            const int g = row0 + row;
            const float inv = qa[0];
            for (int c = lane; c < l0.K / 16; c += 32) {
                float v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int k = c * 16 + i;
                    v[i] = (g < n && k < l0.fin) ? __ldg(obs + (int64_t)g * ld + k) : 0.0f;
                }
                uint32_t w[4];
                e4m3_pack16(v, inv, w);
                const uint32_t at = a_base + (uint32_t)c * 2048u + (uint32_t)(row / 8) * 128u + (uint32_t)(row % 8) * 16u;
                st_shared_v4(at, w[0], w[1], w[2], w[3]);
            }
        }
        for (int rr = 0; rr < 32 && !fp8; ++rr) {
            const int row = q * 32 + rr;
            const int g = row0 + row;
            for (int c = lane; c < l0.K / 8; c += 32) {
                float v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int k = c * 8 + i;
                    v[i] = (g < n && k < l0.fin) ? __ldg(obs + (int64_t)g * ld + k) : 0.0f;
                }
                uint32_t w[4], wl[4];
                if (split)
                    split_pack8(v, w, wl);
                else
                    pack8_16(v, w, plan.f16 != 0);
                const uint32_t at = a_base + (uint32_t)c * 2048u + (uint32_t)(row / 8) * 128u + (uint32_t)(row % 8) * 16u;
                st_shared_v4(at, w[0], w[1], w[2], w[3]);
                if (split) st_shared_v4(at + a_part, wl[0], wl[1], wl[2], wl[3]);
            }
        }
        fence_proxy_async_smem();
        mbar_arrive(a_ready);
        const uint32_t row_off = (uint32_t)(r / 8) * 128u + (uint32_t)(r % 8) * 16u;
        for (int l = 0; l < plan.L; ++l) {
            const TcLayer &ly = plan.layer[l];
            const bool last = l == plan.L - 1;
            if (!mbar_wait(acc_full, (uint32_t)l & 1u, abort, err, 16u, TC_WAIT_NS)) break;
            tc_fence_after();
            const float *bl = bias + ((size_t)agent * MAX_LAYERS + l) * 256;
            const float *dl = dq + ((size_t)agent * MAX_LAYERS + l) * 256;          // FP8 only
            for (int c0 = 0; c0 < ly.N; c0 += 16) {
                uint32_t v[16];
                __syncwarp();
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                tmem_ld_wait();
                float x[16];
                if (fp8) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        x[i] = __fmaf_rn(__uint_as_float(v[i]), __ldg(dl + c0 + i), __ldg(bl + c0 + i));
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i) x[i] = __uint_as_float(v[i]) + __ldg(bl + c0 + i);
                }
                if (!last && fp8) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) x[i] = fmaxf(x[i], 0.0f);
                    uint32_t w[4];
                    e4m3_pack16(x, qa[l + 1], w);
                    st_shared_v4(a_base + (uint32_t)(c0 / 16) * 2048u + row_off, w[0], w[1], w[2], w[3]);
                } else if (!last) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) x[i] = fmaxf(x[i], 0.0f);
                    uint32_t w[8], wl[8];
                    if (split) {
                        split_pack8(x, w, wl);
                        split_pack8(x + 8, w + 4, wl + 4);
                    } else {
                        pack8_16(x, w, plan.f16 != 0);
                        pack8_16(x + 8, w + 4, plan.f16 != 0);
                    }
                    const uint32_t at = a_base + (uint32_t)(c0 / 8) * 2048u + row_off;
                    st_shared_v4(at, w[0], w[1], w[2], w[3]);
                    st_shared_v4(at + 2048u, w[4], w[5], w[6], w[7]);
                    if (split) {
                        st_shared_v4(at + a_part, wl[0], wl[1], wl[2], wl[3]);
                        st_shared_v4(at + a_part + 2048u, wl[4], wl[5], wl[6], wl[7]);
                    }
                } else if (grow < n) {
                    float *yr = y + ((size_t)agent * n + grow) * ly.fout;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int col = c0 + i;
                        if (col < ly.fout) yr[col] = plan.out_act ? tanhf(x[i]) : x[i];
                    }
                }
            }
            if (!last && fp8 && (ly.N & 31)) {
                // the next layer's K is rounded up to 32: zero the 16 columns past N
                st_shared_v4(a_base + (uint32_t)(ly.N / 16) * 2048u + row_off, 0u, 0u, 0u, 0u);
            }
            if (!last) {
                fence_proxy_async_smem();
                tc_fence_before();
                mbar_arrive(a_ready);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, (uint32_t)plan.tmem_cols);
    }
}

}  // namespace

// ------------------------------------------------------------- host side
int tc_create(fr_ensemble *e)
{
    if (e->precision != FR_PREC_BF16 && e->precision != FR_PREC_BF16X3 && e->precision != FR_PREC_FP8 &&
        e->precision != FR_PREC_FP16) {
        set_error("ensemble_create: precision %d has no tensor-core path in this build", e->precision);
        return FR_EINVAL;
    }
    TcImage *t = new TcImage();
    if (!make_plan(e, t->plan)) {
        delete t;
        set_error("ensemble_create: layer sizes exceed the tensor-core kernel (N <= 256, K <= 512)");
        return FR_EINVAL;
    }
    const TcPlan &p = t->plan;
    // pack the fp32 master weights into BF16 chunks on the host
    std::vector<float> host((size_t)e->M * e->P);
    cudaError_t err = cudaMemcpy(host.data(), e->params, host.size() * 4, cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) {
        delete t;
        return cuda_fail(err, "tc_create weights");
    }
    std::vector<uint8_t> img((size_t)e->M * p.agent_bytes, 0);
    std::vector<float> bias((size_t)e->M * MAX_LAYERS * 256, 0.0f);
    const bool fp8 = p.esz == 1;
    const bool grouped = p.split == 1 && !fp8;           // BF16 or FP16
    std::vector<uint8_t> img2(grouped ? img.size() : 0, 0);
    for (int j = 0; j < e->M; ++j) {
        const float *P = host.data() + (size_t)j * e->P;
        uint8_t *aimg = img.data() + (size_t)j * p.agent_bytes;
        for (int l = 0; l < e->L; ++l) {
            const TcLayer &ly = p.layer[l];
            const float *W = P + e->w_off[l];
            const float *B = P + e->b_off[l];
            for (int n = 0; n < ly.fout; ++n) {
                bias[((size_t)j * MAX_LAYERS + l) * 256 + n] = B[n];
                // FP8: per-output-channel scale max_k |W[n][k]| / 448 (1 for a zero row)
                float amax = 0.0f;
                for (int k = 0; k < ly.fin; ++k) amax = std::max(amax, std::fabs(W[(size_t)n * ly.fin + k]));
                const float sw = amax > 0.0f ? amax / E4M3_MAX : 1.0f;
                const float inv = 1.0f / sw;
                t->sw[j][l][n] = sw;
                for (int k = 0; k < ly.fin; ++k) {
                    const int c = k / ly.KC, kk = k % ly.KC;
                    const int kc = std::min(ly.KC, ly.K - c * ly.KC);
                    const size_t off = ly.off + (size_t)c * ly.N * ly.KC * p.esz * p.parts +
                                       chunk_off(ly.N, n, kk, p.ck, p.esz);
                    const float wv = W[(size_t)n * ly.fin + k];
                    if (fp8) {
                        aimg[off] = (uint8_t)__nv_cvt_float_to_fp8(wv * inv, __NV_SATFINITE, __NV_E4M3);
                        continue;
                    }
                    const uint16_t b = p.f16 ? f32_to_f16_sat(wv) : f32_to_bf16_rne(wv);
                    memcpy(aimg + off, &b, 2);
                    if (grouped) {
                        // rows [0, h0) then [h0, N), each group [K/8][rows][8]
                        const int h0 = ly.N > 128 ? ((ly.N / 2 + 15) & ~15) : ly.N;
                        const int hh = n >= h0, n0 = hh ? h0 : 0, ng = hh ? ly.N - h0 : h0, nn = n - n0;
                        const size_t off2 = ly.off + (size_t)(hh ? h0 : 0) * ly.K * 2 + (size_t)(k / 8) * ng * 16 +
                                            (size_t)(nn / 8) * 128 + (size_t)(nn % 8) * 16 + (size_t)(k % 8) * 2;
                        memcpy(img2.data() + (size_t)j * p.agent_bytes + off2, &b, 2);
                    }
                    if (p.split == 3) {
                        const uint16_t bl = f32_to_bf16_rne(wv - bf16_to_f32(b));
                        memcpy(aimg + off + (size_t)ly.N * kc * 2, &bl, 2);
                    }
                }
            }
        }
    }
    const uint64_t ib = img.size(), bb = bias.size() * 4;
    const uint64_t qb = fp8 ? bb + (uint64_t)e->M * MAX_LAYERS * 4 : 0;   // dq + inv_sx
    int rc;
    if ((rc = dev_alloc(e->ctx, (void **)&t->img, ib)) || (rc = dev_alloc(e->ctx, (void **)&t->bias, bb)) ||
        (rc = dev_alloc(e->ctx, (void **)&t->err, 256)) ||
        (fp8 && (rc = dev_alloc(e->ctx, (void **)&t->dq, qb))) ||
        (grouped && (rc = dev_alloc(e->ctx, (void **)&t->img2, ib)))) {
        dev_free(e->ctx, t->img, ib);
        dev_free(e->ctx, t->img2, grouped ? ib : 0);
        dev_free(e->ctx, t->bias, bb);
        dev_free(e->ctx, t->err, 256);
        delete t;
        return rc;
    }
    if (fp8) t->inv_sx = t->dq + (size_t)e->M * MAX_LAYERS * 256;
    t->bytes = ib + bb + 256 + qb + (grouped ? ib : 0);
    err = cudaMemcpy(t->img, img.data(), ib, cudaMemcpyHostToDevice);
    if (err == cudaSuccess && grouped) err = cudaMemcpy(t->img2, img2.data(), ib, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(t->bias, bias.data(), bb, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemset(t->err, 0, 256);
    int optin = 0;
    if (err == cudaSuccess)
        err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, e->ctx->device);
    if (err == cudaSuccess && tc_smem_bytes(p) > (uint32_t)optin) {
        e->tc = t;
        set_error("ensemble_create: tensor-core plan needs %u bytes of shared memory > %d",
                  tc_smem_bytes(p), optin);
        return FR_EINVAL;
    }
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_tc_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    e->tc = t;
    if (err != cudaSuccess) return cuda_fail(err, "tc_create upload");
    return FR_OK;
}

void tc_destroy(fr_ensemble *e)
{
    if (!e || !e->tc) return;
    TcImage *t = e->tc;
    dev_free(e->ctx, t->img, (uint64_t)e->M * t->plan.agent_bytes);
    if (t->img2) dev_free(e->ctx, t->img2, (uint64_t)e->M * t->plan.agent_bytes);
    dev_free(e->ctx, t->bias, (uint64_t)e->M * MAX_LAYERS * 256 * 4);
    dev_free(e->ctx, t->err, 256);
    if (t->dq) dev_free(e->ctx, t->dq, (uint64_t)e->M * MAX_LAYERS * (256 + 1) * 4);
    delete t;
    e->tc = nullptr;
}

// Set the FP8 activation scales sx[j][l] (host [M][L]): recompute the
// dequantisation factors and inverse scales on the host and upload them.
int tc_set_act_scales(fr_ensemble *e, const float *scales)
{
    TcImage *t = e->tc;
    FR_CHECK(t && t->plan.esz == 1, FR_EINVAL, "activation scales apply to FP8 ensembles only");
    for (int i = 0; i < e->M * e->L; ++i)
        FR_CHECK(std::isfinite(scales[i]) && scales[i] > 0.0f, FR_EINVAL,
                 "activation scale %d (%g) must be finite and > 0", i, (double)scales[i]);
    std::vector<float> dq((size_t)e->M * MAX_LAYERS * 256, 0.0f), inv((size_t)e->M * MAX_LAYERS, 0.0f);
    for (int j = 0; j < e->M; ++j) {
        for (int l = 0; l < e->L; ++l) {
            const float sx = scales[j * e->L + l];
            t->sx[j][l] = sx;
            inv[(size_t)j * MAX_LAYERS + l] = 1.0f / sx;
            for (int n = 0; n < t->plan.layer[l].fout; ++n)
                dq[((size_t)j * MAX_LAYERS + l) * 256 + n] = sx * t->sw[j][l][n];
        }
    }
    FR_CUDA(cudaMemcpy(t->dq, dq.data(), dq.size() * 4, cudaMemcpyHostToDevice));
    FR_CUDA(cudaMemcpy(t->inv_sx, inv.data(), inv.size() * 4, cudaMemcpyHostToDevice));
    t->scaled = true;
    t->scale_version += 1;
    t->shared_l0 = true;
    for (int j = 1; j < e->M; ++j) t->shared_l0 = t->shared_l0 && t->sx[j][0] == t->sx[0][0];
    return FR_OK;
}

int tc_get_act_scales(const fr_ensemble *e, float *scales)
{
    const TcImage *t = e->tc;
    FR_CHECK(t && t->plan.esz == 1, FR_EINVAL, "activation scales apply to FP8 ensembles only");
    FR_CHECK(t->scaled, FR_ENOTREADY, "FP8 ensemble has no activation scales yet");
    for (int j = 0; j < e->M; ++j)
        for (int l = 0; l < e->L; ++l) scales[j * e->L + l] = t->sx[j][l];
    return FR_OK;
}

int tc_forward(const fr_ensemble *e, const float *obs, int ld, int n, float *y, cudaStream_t s)
{
    const TcImage *t = e->tc;
    FR_CHECK(t, FR_EINVAL, "tensor-core image missing");
    FR_CHECK(t->plan.esz != 1 || t->scaled, FR_ENOTREADY,
             "FP8 ensemble needs activation scales (ensemble_set_act_scales or ensemble_calibrate_sync)");
    dim3 grid(ceil_div(n, 128), e->M);
    k_tc_forward<<<grid, TC_THREADS, tc_smem_bytes(t->plan), s>>>(t->plan, t->img, t->bias, t->dq, t->inv_sx,
                                                                  obs, ld, n, y, t->err);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

int tc_device_errors(const fr_ensemble *e, unsigned *flags)
{
    *flags = 0;
    if (!e->tc) return FR_OK;
    FR_CUDA(cudaMemcpy(flags, e->tc->err, 4, cudaMemcpyDeviceToHost));
    return FR_OK;
}

}  // namespace fr

extern "C" int ensemble_device_errors(const fr_ensemble *e, uint32_t *flags)
{
    FR_NVTX("ensemble_device_errors");
    FR_CHECK(e && flags, FR_EINVAL, "ensemble_device_errors: NULL argument");
    FR_CUDA(cudaSetDevice(e->ctx->device));
    unsigned f = 0;
    int rc = fr::tc_device_errors(e, &f);
    *flags = f;
    return rc;
}
