// fr_tune.cu -- the autotuner of the batched rollouts: for one env batch and
// ensemble it times the launch configurations the library has for that pair
// and keeps the fastest.  The candidates are
//   * the resident-weight fused stock kernel, with and without tile packing
//     (packing only when the windows differ and auto-reset is off);
//   * the first fused kernel with its weight ring at the most stages that fit
//     (weights resident when a step's chunks fit), at the smallest resident
//     ring and at two stages (weights streamed every step);
//   * the unfused path, with and without the large-batch actor kernel.
// Each candidate runs a short rollout on the env's own state, once to warm
// up and twice timed with CUDA events, the state restored from a host
// snapshot before every run and at the end.  The choice is kept in the env
// and in a process-wide cache keyed by the pair's shape (task, envs,
// assets, uniform or uneven windows, auto-reset, networks, precision, heads,
// SM count), so a later env of the same shape takes it without timing.
// Packing, ring depth and the actor kernel never change results; the three
// paths compute the same function at the same precision class, and each is
// checked against the oracle at the stated tolerance.
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "fr_common.cuh"

using namespace fr;

namespace {

struct TuneCfg {
    int path, packed, stages, tiled;
};

std::mutex g_tune_mu;
std::map<std::vector<int64_t>, TuneCfg> g_tune;

std::vector<int64_t> tune_key(const fr_env *env, const fr_ensemble *e, bool uneven)
{
    const EnvView &v = env->v;
    std::vector<int64_t> k = {v.task,      v.N,          v.K,           v.I,        v.D,
                              uneven,      v.auto_reset, e->M,          e->L,       e->precision,
                              e->combine,  e->out_act,   e->dueling,    env->ctx->sm_count, env->ctx->device,
                              v.buy_order};
    for (int l = 0; l <= e->L; ++l) k.push_back(e->dims[l]);
    return k;
}

void apply(fr_env *env, const TuneCfg &c)
{
    env->tune_set = 1;
    env->tune_path = c.path;
    env->tune_stages = c.stages;
    env->tune_tiled = c.tiled;
    env->pack_off = c.packed ? 0 : 1;
}

void report(fr_tune_report *out, int i, const TuneCfg &c, float ms)
{
    out->path[i] = c.path;
    out->packed[i] = c.packed;
    out->stages[i] = c.stages;
    out->tiled[i] = c.tiled;
    out->ms[i] = ms;
}

}  // namespace

extern "C" {

int env_autotune(fr_env *env, const fr_ensemble *e, int32_t T_probe, int32_t flags, fr_tune_report *out,
                 void *stream)
{
    FR_NVTX("env_autotune");
    FR_CHECK(env && e && out, FR_EINVAL, "env_autotune: NULL argument");
    FR_CHECK(T_probe >= 1 && T_probe <= 4096, FR_EINVAL, "env_autotune: T_probe %d not in 1..4096", T_probe);
    FR_CHECK(env->ctx == e->ctx || env->ctx->device == e->ctx->device, FR_EINVAL,
             "env_autotune: env and ensemble on different devices");
    memset(out, 0, sizeof(*out));
    FR_CUDA(cudaSetDevice(env->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int N = env->v.N;
    std::vector<int32_t> W(N);
    FR_CUDA(cudaMemcpy(W.data(), env->v.W, 4ull * N, cudaMemcpyDeviceToHost));
    bool uneven = false;
    for (int i = 1; i < N && !uneven; ++i) uneven = W[i] != W[0];
    const std::vector<int64_t> key = tune_key(env, e, uneven);
    if (!(flags & FR_TUNE_FORCE)) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            apply(env, it->second);
            out->n = 1;
            out->cached = 1;
            report(out, 0, it->second, 0.0f);
            return FR_OK;
        }
    }
    // candidates for this pair
    std::vector<TuneCfg> cand;
    const bool tensor = e->precision != FR_PREC_FP32;
    if (tensor && env->path == FR_PATH_AUTO) {
        if (f2_supported(env, e)) {
            cand.push_back({2, 1, 0, 1});
            if (uneven && !env->v.auto_reset) cand.push_back({2, 0, 0, 1});
        }
        int nps = 0;
        const int smax = tc_rollout_max_stages(env, e, &nps);
        if (smax >= 2) {
            std::vector<int> st = {smax};
            if (nps >= 2 && nps < smax) st.push_back(nps);
            if (smax > 2 && nps != 2) st.push_back(2);
            for (int x : st) cand.push_back({1, 1, x, 1});
        }
    }
    cand.push_back({0, 1, 0, 1});
    if (tensor && tc_tiled_scratch_bytes(e, N) > 0) cand.push_back({0, 1, 0, 0});
    if ((int)cand.size() > FR_TUNE_MAX) cand.resize(FR_TUNE_MAX);

    // the env's state and knobs, restored whatever happens
    size_t len = 0;
    int rc = env_snapshot(env, nullptr, 0, &len);
    if (rc) return rc;
    std::vector<uint8_t> snap(len);
    if ((rc = env_snapshot(env, snap.data(), len, &len))) return rc;
    const int o_set = env->tune_set, o_path = env->tune_path, o_st = env->tune_stages, o_tiled = env->tune_tiled,
              o_pack = env->pack_off;
    const uint32_t o_step = env->explore_step;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t ce = cudaEventCreate(&ev[0]);
    if (ce == cudaSuccess) ce = cudaEventCreate(&ev[1]);
    int best = -1;
    float best_ms = 0.0f;
    for (size_t c = 0; c < cand.size() && rc == FR_OK && ce == cudaSuccess; ++c) {
        apply(env, cand[c]);
        float sum = 0.0f;
        for (int r = 0; r < 3 && rc == FR_OK && ce == cudaSuccess; ++r) {
            if ((rc = env_restore(env, snap.data(), len))) break;
            env->explore_step = o_step;
            ce = cudaEventRecord(ev[0], s);
            if (ce == cudaSuccess) rc = rollout(env, e, T_probe, nullptr, nullptr, s);
            if (rc == FR_OK && ce == cudaSuccess) ce = cudaEventRecord(ev[1], s);
            if (rc == FR_OK && ce == cudaSuccess) ce = cudaEventSynchronize(ev[1]);
            float ms = 0.0f;
            if (rc == FR_OK && ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (r > 0) sum += ms;                              // the first run warms up
        }
        if (rc != FR_OK || ce != cudaSuccess) break;
        const float ms = sum / 2.0f;
        report(out, (int)c, cand[c], ms);
        out->n = (int)c + 1;
        if (best < 0 || ms < best_ms) {
            best = (int)c;
            best_ms = ms;
        }
    }
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    const int rrc = env_restore(env, snap.data(), len);
    env->explore_step = o_step;
    if (rc == FR_OK && ce != cudaSuccess) rc = cuda_fail(ce, "env_autotune");
    if (rc == FR_OK) rc = rrc;
    if (rc != FR_OK || best < 0) {
        env->tune_set = o_set;
        env->tune_path = o_path;
        env->tune_stages = o_st;
        env->tune_tiled = o_tiled;
        env->pack_off = o_pack;
        return rc ? rc : FR_EINVAL;
    }
    apply(env, cand[best]);
    out->chosen = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = cand[best];
    return FR_OK;
}

int env_tune_set(fr_env *env, int32_t path, int32_t packed, int32_t stages, int32_t tiled)
{
    FR_NVTX("env_tune_set");
    FR_CHECK(env, FR_EINVAL, "env_tune_set: NULL env");
    FR_CHECK(path >= 0 && path <= 2 && (stages == 0 || stages >= 2), FR_EINVAL,
             "env_tune_set: path %d or stages %d out of range", path, stages);
    apply(env, TuneCfg{path, packed ? 1 : 0, stages, tiled ? 1 : 0});
    return FR_OK;
}

int env_tune_clear(fr_env *env)
{
    FR_NVTX("env_tune_clear");
    FR_CHECK(env, FR_EINVAL, "env_tune_clear: NULL env");
    env->tune_set = 0;
    env->pack_off = 0;
    return FR_OK;
}

}  // extern "C"
