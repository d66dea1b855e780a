// fr_tc.cuh -- tensor-core weight images shared by the actor kernel
// (fr_tc.cu) and the fused rollout kernel (fr_fused.cu).
//
// Each agent's weights are packed on the host into BF16 "chunks": a chunk
// holds K columns [c*KC, c*KC + kc) of one layer for all N output rows, laid
// out in the tcgen05 K-major, no-swizzle canonical form (8-row x 16-byte core
// matrices; adjacent core matrices along K are N*16 bytes apart, adjacent
// 8-row groups 128 bytes apart).  With split precision the chunk holds the
// BF16 "hi" part followed by the BF16 rounding of the remainder ("lo").
#pragma once

#include <cuda_bf16.h>

#include "fr_common.cuh"

namespace fr {

constexpr int TC_STAGES = 2;                  // ring stages of the forward kernel
constexpr uint32_t TC_CHUNK_MAX = 16384;      // bytes per ring stage
constexpr int TC_THREADS = 192;               // producer, MMA, 4 epilogue warps
constexpr uint64_t TC_WAIT_NS = 2000000000ull;

struct TcLayer {
    int fin, fout;        // true sizes
    int K, N;             // padded to multiples of 16
    int KC;               // K columns per streamed chunk
    int n_chunks;
    uint32_t off;         // byte offset of the layer's chunks in an agent image
};

struct TcPlan {
    int M, L, out_act;
    int split;            // 1: BF16 operands; 3: hi/lo split, three products
    int parts;            // operand parts stored per chunk: 1 (hi) or 2 (hi, lo)
    int KA;               // K extent of the shared A buffer (max layer K)
    int tmem_cols;        // power of two >= max N
    uint32_t agent_bytes;
    TcLayer layer[MAX_LAYERS];
};

struct TcImage {
    TcPlan plan;
    uint8_t *img;         // device [M][agent_bytes] BF16 chunks
    float *bias;          // device [M][MAX_LAYERS][256] fp32, zero padded
    unsigned *err;        // device error flags
    uint64_t bytes;
};


// A operand bytes (one part) of a plan
inline __host__ __device__ uint32_t a_part_bytes(const TcPlan &p) { return (uint32_t)(p.KA / 8) * 2048u; }

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
