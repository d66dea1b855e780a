// fr_replay.cu -- the device-resident replay buffer between the simulation
// phase (producer) and the learning phase (consumer) of Sec. 3.2, fed by the
// T x N x D sample tensors a rollout keeps in GPU memory (Sec. 4.3.2).
//
// The buffer is a FIFO ring of C transitions (s, a, r, s', done) in
// structure-of-arrays form: obs[C][Dp], next[C][Dp] (Dp = D rounded up to 4),
// act float [C][Kp] (stock) or uint8 [C] (crypto), rew float [C] (the
// learner's reward copy), done uint8 [C].  The count of transitions ever
// pushed lives on the device, so pushes and samples are asynchronous and
// capturable.
//
// Push: the rows of a trajectory in (t, env) order; row (t, e) is a real
// step unless the env was already done before it (done[t-1][e], or not live
// at the start of the rollout), which frozen envs show without auto-reset.
// Valid rows are appended in that order: a count kernel (one block per 1024
// rows), a one-block scan that also advances the device counter, and a
// scatter kernel that ranks its rows again and copies them, one warp per
// row so that every copy is coalesced.  s' of row (t, e) is obs[t+1][e], or
// the caller's observation after the rollout for t = T - 1.
//
// Sample: B uniform draws over the current contents (Philox4x32-10 of
// (b, counter, 3) under the seed; index = (x0 * size) >> 32, 0 = oldest),
// gathered one warp per row.
#include <new>

#include "fr_common.cuh"

namespace fr {
namespace {

constexpr int RP_ROWS = 1024;         // rows per count / scatter block

__device__ __forceinline__ bool rp_valid(int64_t r, int N, const uint8_t *done, const uint8_t *live0,
                                         int auto_reset)
{
    if (auto_reset) return true;
    const int64_t t = r / N, e = r % N;
    if (t == 0) return live0 ? live0[e] != 0 : true;
    return done[r - N] == 0;
}

__global__ void __launch_bounds__(RP_ROWS) k_rp_count(int64_t rows, int N, const uint8_t *done,
                                                      const uint8_t *live0, int auto_reset, int64_t *counts)
{
    const int64_t r = (int64_t)blockIdx.x * RP_ROWS + threadIdx.x;
    const int v = r < rows && rp_valid(r, N, done, live0, auto_reset);
    const int c = __syncthreads_count(v);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// Exclusive scan of the block counts (in place), then state[1] = the count
// before this push and state[0] += this push's valid rows.
__global__ void __launch_bounds__(1024) k_rp_scan(int64_t *counts, int nb, int64_t *state)
{
    __shared__ int64_t part[32];
    __shared__ int64_t carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const int64_t x = i < nb ? counts[i] : 0;
        int64_t s = x;                               // inclusive warp scan
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane == 31) part[warp] = s;
        __syncthreads();
        if (warp == 0) {
            int64_t p = part[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, p, o);
                if (lane >= o) p += y;
            }
            part[lane] = p;                          // inclusive over warps
        }
        __syncthreads();
        const int64_t carry = carry_s;
        const int64_t excl = carry + (warp ? part[warp - 1] : 0) + s - x;
        if (i < nb) counts[i] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + part[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        state[1] = state[0];
        state[0] += carry_s;
    }
}

struct RpBuf {
    float *obs, *next, *rew;
    void *act;
    uint8_t *done;
    int64_t C;
    int D, Dp, K, Kp, act_u8;
};

// Copy two rows of D floats (either pair may be absent: NULL source or
// destination) by one warp, with up to ten loads per row and lane in flight
// before the stores (a plain strided loop keeps one per row in flight).
__device__ __forceinline__ void rp_copy2(float *dst, const float *src, float *ndst, const float *nsrc, int D,
                                         int lane)
{
    for (int k0 = 0; k0 < D; k0 += 320) {
        float x[10], y[10];
#pragma unroll
        for (int u = 0; u < 10; ++u) {
            const int k = k0 + lane + 32 * u;
            x[u] = (src && k < D) ? __ldg(src + k) : 0.0f;
            y[u] = (nsrc && k < D) ? __ldg(nsrc + k) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 10; ++u) {
            const int k = k0 + lane + 32 * u;
            if (k < D) {
                if (dst) dst[k] = x[u];
                if (ndst) ndst[k] = y[u];
            }
        }
    }
}

__global__ void __launch_bounds__(RP_ROWS) k_rp_scatter(RpBuf b, int64_t rows, int N, int ld, const float *obs,
                                                        const void *act, const float *rew, const uint8_t *done,
                                                        const float *last_obs, const uint8_t *live0,
                                                        int auto_reset, const int64_t *offsets,
                                                        const int64_t *state)
{
    __shared__ int64_t slot_s[RP_ROWS];
    __shared__ int wcount[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * RP_ROWS;
    const int64_t r = r0 + threadIdx.x;
    const bool v = r < rows && rp_valid(r, N, done, live0, auto_reset);
    const unsigned m = __ballot_sync(0xffffffffu, v);
    if (lane == 0) wcount[warp] = __popc(m);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wcount[w];
    const int rank = before + __popc(m & ((1u << lane) - 1u));
    slot_s[threadIdx.x] = v ? (state[1] + offsets[blockIdx.x] + rank) % b.C : -1;
    __syncthreads();
    // copy: warp w handles rows w, w + 32, ... of the block
    for (int i = warp; i < RP_ROWS; i += 32) {
        const int64_t slot = slot_s[i];
        if (slot < 0) continue;
        const int64_t row = r0 + i;
        const int64_t e = row % N;
        const float *src = obs + row * ld;
        const float *nsrc = row + N < rows ? obs + (row + N) * ld : last_obs + e * ld;   // t < T - 1: obs[t+1][e]
        rp_copy2(b.obs + slot * b.Dp, src, b.next + slot * b.Dp, nsrc, b.D, lane);
        if (b.act_u8) {
            if (lane == 0) ((uint8_t *)b.act)[slot] = ((const uint8_t *)act)[row];
        } else {
            for (int k = lane; k < b.K; k += 32)
                ((float *)b.act)[slot * b.Kp + k] = __ldg((const float *)act + row * b.K + k);
        }
        if (lane == 0) {
            b.rew[slot] = rew[row];
            b.done[slot] = done[row];
        }
    }
}

__global__ void __launch_bounds__(256) k_rp_sample(RpBuf b, int B, uint32_t k0, uint32_t k1, uint32_t c0,
                                                   uint32_t c1, const int64_t *state, float *obs, void *act,
                                                   float *rew, float *next, uint8_t *done, int64_t *index,
                                                   unsigned *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= B) return;
    const int64_t total = state[0];
    const int64_t size = total < b.C ? total : b.C;
    uint32_t w[4];
    philox4x32_10((uint32_t)i, c0, c1, 3u, k0, k1, w);
    const int64_t idx = size > 0 ? (int64_t)(((uint64_t)w[0] * (uint64_t)size) >> 32) : -1;
    if (idx < 0) {
        if (lane == 0) {
            atomicOr(err, 1u);
            if (index) index[i] = -1;
        }
        return;
    }
    const int64_t slot = (total - size + idx) % b.C;
    rp_copy2(obs ? obs + i * b.D : nullptr, obs ? b.obs + slot * b.Dp : nullptr, next ? next + i * b.D : nullptr,
             next ? b.next + slot * b.Dp : nullptr, b.D, lane);
    if (act) {
        if (b.act_u8) {
            if (lane == 0) ((uint8_t *)act)[i] = ((const uint8_t *)b.act)[slot];
        } else {
            for (int k = lane; k < b.K; k += 32) ((float *)act)[i * b.K + k] = ((const float *)b.act)[slot * b.Kp + k];
        }
    }
    if (lane == 0) {
        if (rew) rew[i] = b.rew[slot];
        if (done) done[i] = b.done[slot];
        if (index) index[i] = idx;
    }
}

}  // namespace
}  // namespace fr

using namespace fr;

struct fr_replay {
    fr_ctx *ctx;
    int task;
    RpBuf b;
    int64_t *state;          // device [3]: transitions ever pushed, count before the last push, error flags
    unsigned *err;           // low word of state[2]: bit 0 = a sample drew from an empty buffer
    void *block;
    uint64_t bytes;
};

extern "C" {

int replay_create(fr_ctx *ctx, const fr_env *env, int64_t capacity, fr_replay **out)
{
    FR_NVTX("replay_create");
    FR_CHECK(ctx && env && out, FR_EINVAL, "replay_create: NULL argument");
    *out = nullptr;
    FR_CHECK(capacity >= 1 && capacity <= 0x7fffffffLL, FR_EINVAL, "replay_create: capacity %lld not in 1..2^31-1",
             (long long)capacity);
    FR_CUDA(cudaSetDevice(ctx->device));
    fr_replay *rb = new (std::nothrow) fr_replay();
    FR_CHECK(rb, FR_ENOMEM, "replay_create: out of host memory");
    rb->ctx = ctx;
    rb->task = env->v.task;
    RpBuf &b = rb->b;
    b.C = capacity;
    b.D = env->v.D;
    b.Dp = (b.D + 3) & ~3;
    b.act_u8 = env->v.task == FR_TASK_CRYPTO;
    b.K = b.act_u8 ? 1 : env->v.K;
    b.Kp = (b.K + 3) & ~3;
    // every segment padded to 256 bytes, so each array (the int64 counters
    // after the byte-sized done flags included) starts aligned for any capacity
    const uint64_t C = (uint64_t)capacity;
    auto pad = [](uint64_t x) { return (x + 255) & ~255ull; };
    const uint64_t ob = pad(C * b.Dp * 4), ab = pad(b.act_u8 ? C : C * b.Kp * 4), rbb = pad(C * 4), db = pad(C);
    rb->bytes = 2 * ob + ab + rbb + db + 256;
    int rc = dev_alloc(ctx, &rb->block, rb->bytes);
    if (rc) {
        delete rb;
        return rc;
    }
    char *p = (char *)rb->block;
    b.obs = (float *)p;
    b.next = (float *)(p + ob);
    b.act = p + 2 * ob;
    b.rew = (float *)(p + 2 * ob + ab);
    b.done = (uint8_t *)(p + 2 * ob + ab + rbb);
    rb->state = (int64_t *)(p + 2 * ob + ab + rbb + db);
    rb->err = (unsigned *)(rb->state + 2);
    if (((uintptr_t)b.next | (uintptr_t)b.act | (uintptr_t)b.rew | (uintptr_t)b.done | (uintptr_t)rb->state) & 255u) {
        dev_free(ctx, rb->block, rb->bytes);
        delete rb;
        set_error("replay_create: internal layout misaligned");
        return FR_EINVAL;
    }
    cudaError_t e = cudaMemset(rb->state, 0, 256);
    if (e != cudaSuccess) {
        dev_free(ctx, rb->block, rb->bytes);
        delete rb;
        return cuda_fail(e, "replay_create");
    }
    *out = rb;
    return FR_OK;
}

void replay_destroy(fr_replay *rb)
{
    FR_NVTX("replay_destroy");
    if (!rb) return;
    cudaSetDevice(rb->ctx->device);
    dev_free(rb->ctx, rb->block, rb->bytes);
    delete rb;
}

int replay_push(fr_replay *rb, const fr_env *env, const fr_traj *tr, int32_t T, const float *last_obs,
                const uint8_t *live0, void *stream)
{
    FR_NVTX("replay_push");
    FR_CHECK(rb && env && tr && last_obs, FR_EINVAL, "replay_push: NULL argument");
    FR_CHECK(env->v.task == rb->task && env->v.D == rb->b.D && (rb->b.act_u8 || env->v.K == rb->b.K), FR_EINVAL,
             "replay_push: env shape does not match the buffer");
    FR_CHECK(tr->obs && tr->act && tr->rew_f32 && tr->done, FR_EINVAL,
             "replay_push: the trajectory needs obs, act, rew_f32 and done");
    FR_CHECK(T >= 0, FR_EINVAL, "replay_push: T < 0");
    const int ld = tr->obs_ld ? tr->obs_ld : env->v.D;
    FR_CHECK(ld >= env->v.D, FR_EINVAL, "replay_push: obs_ld %d < D", ld);
    if (T == 0) return FR_OK;
    FR_CUDA(cudaSetDevice(rb->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int N = env->v.N;
    const int64_t rows = (int64_t)T * N;
    const int64_t nb = (rows + RP_ROWS - 1) / RP_ROWS;
    FR_CHECK(nb <= 0x7fffffffLL, FR_EINVAL, "replay_push: trajectory too large");
    int64_t *counts = nullptr;
    FR_CUDA(cudaMallocAsync((void **)&counts, (size_t)nb * 8, s));
    const int ar = env->v.auto_reset;
    k_rp_count<<<(unsigned)nb, RP_ROWS, 0, s>>>(rows, N, tr->done, live0, ar, counts);
    k_rp_scan<<<1, 1024, 0, s>>>(counts, (int)nb, rb->state);
    k_rp_scatter<<<(unsigned)nb, RP_ROWS, 0, s>>>(rb->b, rows, N, ld, tr->obs, tr->act, tr->rew_f32, tr->done,
                                                  last_obs, live0, ar, counts, rb->state);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(counts, s);
    FR_CUDA(e);
    return FR_OK;
}

int replay_sample(fr_replay *rb, int32_t B, uint64_t seed, uint64_t counter, float *obs, void *act, float *rew,
                  float *next_obs, uint8_t *done, int64_t *index, void *stream)
{
    FR_NVTX("replay_sample");
    FR_CHECK(rb && B >= 0, FR_EINVAL, "replay_sample: bad argument");
    if (B == 0) return FR_OK;
    FR_CUDA(cudaSetDevice(rb->ctx->device));
    const int64_t threads = (int64_t)B * 32;
    k_rp_sample<<<ceil_div(threads, 256), 256, 0, (cudaStream_t)stream>>>(
        rb->b, B, (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)counter, (uint32_t)(counter >> 32), rb->state,
        obs, act, rew, next_obs, done, index, rb->err);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}

int replay_size_sync(fr_replay *rb, int64_t *size, int64_t *pushed, uint32_t *errors, void *stream)
{
    FR_NVTX("replay_size_sync");
    FR_CHECK(rb, FR_EINVAL, "replay_size_sync: NULL buffer");
    FR_CUDA(cudaSetDevice(rb->ctx->device));
    int64_t h[4] = {0, 0, 0, 0};
    cudaStream_t s = (cudaStream_t)stream;
    FR_CUDA(cudaMemcpyAsync(h, rb->state, 32, cudaMemcpyDeviceToHost, s));
    FR_CUDA(cudaStreamSynchronize(s));
    if (pushed) *pushed = h[0];
    if (size) *size = h[0] < rb->b.C ? h[0] : rb->b.C;
    if (errors) *errors = (uint32_t)(h[2] & 0xffffffffu);
    return FR_OK;
}

}  // extern "C"
