// fr_env_kernels.cu -- the reset / step / reward operations of every SubEnv
// (Sec. 4.2.2), one launch over the whole VecEnv.  Stock envs are stepped by
// one warp per env (lane = asset, warp-shuffle int64 reductions for the
// total-asset value); crypto envs by one thread per env.
#include "fr_env_dev.cuh"

namespace fr {

namespace {

constexpr int kBlock = 256;

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

template <int KIND>
__global__ void __launch_bounds__(kBlock) k_stock_step(EnvView v, const void *act, int64_t *rew,
                                                        float *rew_f32, uint8_t *done_out,
                                                        float *obs, int ld)
{
    const int e = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= v.N) return;                     // uniform per warp
    int32_t q = 0;
    if (lane < v.Ke[e]) {
        if (KIND == FR_ACT_I32_SHARES) {
            q = ((const int32_t *)act)[(int64_t)e * v.K + lane];
        } else {
            bool bad;
            q = discretise(((const float *)act)[(int64_t)e * v.K + lane], v.hmax, bad);
            if (bad) atomicAdd(v.err, 1ull);
        }
    }
    bool done;
    const int64_t r = stock_step_warp(v, e, lane, q, done);
    if (lane == 0) {
        if (rew) rew[e] = r;
        if (rew_f32) rew_f32[e] = reward_f32(r);
        if (done_out) done_out[e] = done ? 1 : 0;
    }
    if (obs) {
        __syncwarp();
        stock_obs_warp(v, e, lane, obs + (int64_t)e * ld);
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

cudaError_t launch_env_step(const EnvView &v, int kind, const void *act, int64_t *rew,
                            float *rew_f32, uint8_t *done, float *obs, int ld, cudaStream_t s)
{
    if (v.task == FR_TASK_STOCK) {
        const unsigned grid = ceil_div((int64_t)v.N * 32, kBlock);
        if (kind == FR_ACT_I32_SHARES)
            k_stock_step<FR_ACT_I32_SHARES><<<grid, kBlock, 0, s>>>(v, act, rew, rew_f32, done, obs, ld);
        else
            k_stock_step<FR_ACT_F32_UNIT><<<grid, kBlock, 0, s>>>(v, act, rew, rew_f32, done, obs, ld);
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
