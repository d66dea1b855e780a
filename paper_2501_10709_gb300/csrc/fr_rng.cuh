// fr_rng.cuh -- counter-based randomness: the exploring rollouts' draws and
// the per-env price perturbations.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC 2011): ten rounds, each mapping counter words
// (c0, c1, c2, c3) under key (k0, k1) to
//   (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// the key advanced by the Weyl constants between rounds.  A draw is a pure
// function of (seed, env, global step, component), so a rollout explores
// identically whatever the launch shape or the order of execution.
#pragma once

#include <stdint.h>

namespace fr {

__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                       uint32_t k0, uint32_t k1, uint32_t *out)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014, with Stafford's mix13 finaliser): advance by the
// golden gamma, then three xor-shift / multiply rounds.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// The per-env price perturbation of Sec. 5.1 (+-1% at R = 100): basis points
// of env i, asset k, uniform on [-R, R] as z mod (2R + 1) - R with
// z = splitmix64(seed ^ splitmix64(i << 8 | k)).
__host__ __device__ __forceinline__ int16_t perturb_bps(uint64_t seed, uint32_t i, uint32_t k, int R)
{
    const uint64_t z = splitmix64(seed ^ splitmix64(((uint64_t)i << 8) | (uint64_t)k));
    return (int16_t)((int64_t)(z % (uint64_t)(2 * R + 1)) - R);
}

// Exploration parameters as the kernels take them.
struct Explore {
    int kind;                 // FR_EXPLORE_*
    float sigma;              // Gaussian: a_k + sigma z
    uint32_t thr;             // greedy: replace when (x >> 8) < thr = floor(eps 2^24)
    uint32_t k0, k1;          // seed
    uint32_t g0;              // global step of the rollout's first step
};

// Standard normal draw of env e, global step g, component k: Box-Muller in
// float32 from u = ((x >> 8) + 1/2) 2^-24 of Philox(e, g, k, 0).
__device__ __forceinline__ float explore_normal(const Explore &x, uint32_t e, uint32_t g, uint32_t k)
{
    uint32_t w[4];
    philox4x32_10(e, g, k, 0u, x.k0, x.k1, w);
    const float u0 = __fadd_rn(__fmul_rn((float)(w[0] >> 8), 5.9604644775390625e-8f), 2.98023223876953125e-8f);
    const float u1 = __fadd_rn(__fmul_rn((float)(w[1] >> 8), 5.9604644775390625e-8f), 2.98023223876953125e-8f);
    return sqrtf(-2.0f * logf(u0)) * cospif(2.0f * u1);
}

// The greedy replacement of a discrete action of env e at global step g.
__device__ __forceinline__ int explore_greedy(const Explore &x, uint32_t e, uint32_t g, int action)
{
    uint32_t w[4];
    philox4x32_10(e, g, 0u, 1u, x.k0, x.k1, w);
    if ((w[2] >> 8) < x.thr) return (int)(((uint64_t)(w[3] >> 8) * 3u) >> 24);
    return action;
}

}  // namespace fr
