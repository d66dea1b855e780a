// fr_tc.cuh -- tensor-core weight images shared by the actor kernel
// (fr_tc.cu) and the fused rollout kernel (fr_fused.cu).
//
// Each agent's weights are packed on the host into BF16 (or FP8 E4M3)
// "chunks": a chunk holds K columns [c*KC, c*KC + kc) of one layer for all N
// output rows, laid out in the tcgen05 K-major, no-swizzle canonical form
// (8-row x 16-byte core matrices, i.e. 8 BF16 or 16 E4M3 elements along K;
// adjacent core matrices along K are N*16 bytes apart, adjacent 8-row groups
// 128 bytes apart).  With split precision the chunk holds the BF16 "hi" part
// followed by the BF16 rounding of the remainder ("lo").
//
// FP8 (E4M3, round to nearest even, saturating at +-448): row n of layer l is
// stored as codes of W[n][k] * (1 / sw[n]) with the per-output-channel scale
// sw[n] = max_k |W[n][k]| / 448 (1 when the row is zero); the layer's input x
// is quantised as codes of x * (1 / sx[l]) with a static per-agent, per-layer
// activation scale; the accumulator is dequantised as
// fma(acc, sx[l] * sw[n], b[n]).  All of these are float32 operations.
#pragma once

#include <cuda_bf16.h>

#include "fr_common.cuh"
#include "fr_ptx.cuh"

namespace fr {

constexpr int TC_STAGES = 2;                  // ring stages of the forward kernel
constexpr uint32_t TC_CHUNK_MAX = 16384;      // bytes per ring stage
constexpr int TC_THREADS = 192;               // producer, MMA, 4 epilogue warps
constexpr uint64_t TC_WAIT_NS = 2000000000ull;
constexpr float E4M3_MAX = 448.0f;            // largest finite E4M3 value

struct TcLayer {
    int fin, fout;        // true sizes
    int K, N;             // padded: N to 16, K to kmma (16 BF16, 32 E4M3)
    int KC;               // K columns per streamed chunk
    int n_chunks;
    uint32_t off;         // byte offset of the layer's chunks in an agent image
};

struct TcPlan {
    int M, L, out_act;
    int split;            // 1: BF16 (or FP16) operands; 3: hi/lo split, three products
    int f16;              // 1: FP16 operands instead of BF16 (split 1 only)
    int parts;            // operand parts stored per chunk: 1 (hi) or 2 (hi, lo)
    int esz;              // operand element bytes: 2 (BF16) or 1 (E4M3)
    int kmma;             // K per tcgen05.mma: 16 (kind::f16) or 32 (kind::f8f6f4)
    int ck;               // elements per 16-byte core-matrix row: 8 or 16
    int KA;               // K extent of the shared A buffer (max layer K)
    int tmem_cols;        // power of two >= max N
    uint32_t agent_bytes;
    TcLayer layer[MAX_LAYERS];
};

struct TcImage {
    TcPlan plan;
    uint8_t *img;         // device [M][agent_bytes] BF16 chunks
    // BF16 without split: the same weights with each layer's output rows in
    // at most two groups (k_tc_actor2's halves), each group's K-major core
    // columns end to end, so a run of K steps of one group is contiguous
    uint8_t *img2 = nullptr;
    float *bias;          // device [M][MAX_LAYERS][256] fp32, zero padded
    unsigned *err;        // device error flags
    uint64_t bytes;
    // FP8 only: dequantisation factors sx[l] * sw[n] [M][MAX_LAYERS][256] and
    // the inverse activation scales 1 / sx[l] [M][MAX_LAYERS] (device); the
    // scales themselves (host) and whether activation scales were set
    float *dq = nullptr;
    float *inv_sx = nullptr;
    float sw[MAX_AGENTS][MAX_LAYERS][256];
    float sx[MAX_AGENTS][MAX_LAYERS];
    bool scaled = false;
    bool shared_l0 = false;   // every agent has the same layer-0 scale
    uint32_t scale_version = 0;   // bumped whenever the activation scales change
};


// A operand bytes (one part) of a plan
inline __host__ __device__ uint32_t a_part_bytes(const TcPlan &p) { return (uint32_t)(p.KA / p.ck) * 2048u; }

// Two floats -> E4M3 codes (round to nearest even, saturating), `lo` in the
// low byte.
__device__ __forceinline__ uint32_t e4m3x2(float lo, float hi)
{
    uint16_t r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
    return (uint32_t)r;
}

// Sixteen floats times `inv` -> sixteen E4M3 codes in K order (4 words).
__device__ __forceinline__ void e4m3_pack16(const float *v, float inv, uint32_t *w)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        w[i] = e4m3x2(__fmul_rn(v[4 * i], inv), __fmul_rn(v[4 * i + 1], inv)) |
               (e4m3x2(__fmul_rn(v[4 * i + 2], inv), __fmul_rn(v[4 * i + 3], inv)) << 16);
    }
}

// Two floats -> one word of two 16-bit operands (BF16 round to nearest even,
// or FP16 round to nearest even saturating at +-65504), a in the low half.
__device__ __forceinline__ uint32_t pack2_16(float a, float b, bool f16)
{
    if (f16) return ptx::f16x2_sat(a, b);
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *(const uint32_t *)&h;
}

// Eight floats -> four words of 16-bit operands, K order.
__device__ __forceinline__ void pack8_16(const float *v, uint32_t *w, bool f16)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = pack2_16(v[2 * i], v[2 * i + 1], f16);
}

// Eight floats -> BF16 hi parts (round to nearest) and the BF16 rounding of
// what hi leaves over (x - hi), packed two per word in K order.
__device__ __forceinline__ void split_pack8(const float *v, uint32_t *hi, uint32_t *lo)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
        hi[i] = *(const uint32_t *)&h;
        lo[i] = *(const uint32_t *)&l;
    }
}


}  // namespace fr
