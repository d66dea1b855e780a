// fr_validate.cu -- Sharpe-softmax ensemble weights from a validation
// window (Sec. 5.2.1): every agent trades the validation envs alone, its
// Sharpe ratio is the mean over those envs of the episode Sharpe (the same
// FP64 statistic as env_metrics), agents below the threshold are discarded,
// and the remaining weights are a softmax of the Sharpe ratios.  The
// ensemble's combine weights are then set to them.
#include <math.h>

#include <vector>

#include "fr_common.cuh"

using namespace fr;

namespace {

// Softmax of the kept agents' Sharpe ratios (max subtracted first; sums in
// agent order); the rest get 0.  When no agent reaches the threshold the best
// one (lowest index on ties) is kept alone.
void sharpe_softmax(int M, const double *S, double threshold, double *w)
{
    std::vector<int> keep;
    for (int j = 0; j < M; ++j)
        if (S[j] >= threshold) keep.push_back(j);
    if (keep.empty()) {
        int best = 0;
        for (int j = 1; j < M; ++j)
            if (S[j] > S[best]) best = j;
        keep.push_back(best);
    }
    double m = S[keep[0]];
    for (int j : keep) m = S[j] > m ? S[j] : m;
    double sum = 0.0;
    for (int j = 0; j < M; ++j) w[j] = 0.0;
    for (int j : keep) {
        w[j] = exp(S[j] - m);
        sum += w[j];
    }
    for (int j : keep) w[j] = w[j] / sum;
}

}  // namespace

extern "C" {

int ensemble_set_weights(fr_ensemble *e, const float *w)
{
    FR_NVTX("ensemble_set_weights");
    FR_CHECK(e && w, FR_EINVAL, "ensemble_set_weights: NULL argument");
    FR_CHECK(e->combine == FR_COMBINE_MEAN, FR_EINVAL, "ensemble_set_weights: weights apply to MEAN only");
    for (int j = 0; j < e->M; ++j)
        FR_CHECK(isfinite(w[j]), FR_EINVAL, "ensemble_set_weights: weight %d is not finite", j);
    FR_CUDA(cudaSetDevice(e->ctx->device));
    for (int j = 0; j < e->M; ++j) e->host_weights[j] = w[j];
    FR_CUDA(cudaMemcpy(e->weights, e->host_weights, 4ull * MAX_AGENTS, cudaMemcpyHostToDevice));
    return FR_OK;
}

int ensemble_validate(fr_ensemble *e, fr_env *env, int32_t T, double threshold, double *sharpe,
                      float *weights, void *stream)
{
    FR_NVTX("ensemble_validate");
    FR_CHECK(e && env && T >= 1, FR_EINVAL, "ensemble_validate: bad argument");
    FR_CHECK(e->combine == FR_COMBINE_MEAN, FR_EINVAL, "ensemble_validate: weights apply to MEAN ensembles");
    FR_CHECK(isfinite(threshold) || threshold == -INFINITY, FR_EINVAL, "ensemble_validate: threshold");
    FR_CUDA(cudaSetDevice(e->ctx->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int N = env->v.N;
    // the validation envs' state, restored before every agent and at the end
    size_t need = 0;
    int rc = env_snapshot(env, nullptr, 0, &need);
    if (rc) return rc;
    std::vector<uint8_t> snap(need);
    rc = env_snapshot(env, snap.data(), need, &need);
    if (rc) return rc;
    std::vector<float> P((size_t)e->M * e->P);
    FR_CUDA(cudaMemcpy(P.data(), e->params, P.size() * 4, cudaMemcpyDeviceToHost));
    double *met = nullptr;
    FR_CUDA(cudaMalloc(&met, 24ull * N));
    std::vector<double> hm((size_t)N * 3), S(e->M);
    for (int j = 0; j < e->M && rc == FR_OK; ++j) {
        fr_ensemble_desc d{};
        d.n_agents = 1;
        d.n_layers = e->L;
        d.dims = e->dims;
        d.params = P.data() + (size_t)j * e->P;
        d.weights = nullptr;
        d.precision = e->precision;
        d.combine = e->combine;
        d.out_act = e->out_act;
        d.heads = &e->heads[j];
        fr_ensemble *one = nullptr;
        if ((rc = ensemble_create(e->ctx, &d, &one))) break;
        if (e->precision == FR_PREC_FP8) {
            // the agent keeps its own activation scales
            float sx[MAX_AGENTS * MAX_LAYERS];
            if (!(rc = tc_get_act_scales(e, sx))) rc = tc_set_act_scales(one, sx + (size_t)j * e->L);
            if (rc) {
                ensemble_destroy(one);
                break;
            }
        }
        if (!(rc = env_restore(env, snap.data(), snap.size())) &&
            !(rc = rollout(env, one, T, nullptr, met, s))) {
            const cudaError_t ce = cudaMemcpyAsync(hm.data(), met, 24ull * N, cudaMemcpyDeviceToHost, s);
            rc = ce == cudaSuccess ? (cudaStreamSynchronize(s) == cudaSuccess ? FR_OK : FR_ECUDA) : FR_ECUDA;
            if (rc) set_error("ensemble_validate: metrics copy failed");
        }
        ensemble_destroy(one);
        if (rc) break;
        double sum = 0.0;
        for (int i = 0; i < N; ++i) sum += hm[3 * (size_t)i + 1];
        S[j] = sum / N;
    }
    cudaFree(met);
    const int rc2 = env_restore(env, snap.data(), snap.size());
    if (rc) return rc;
    if (rc2) return rc2;
    std::vector<double> w(e->M);
    sharpe_softmax(e->M, S.data(), threshold, w.data());
    std::vector<float> wf(e->M);
    for (int j = 0; j < e->M; ++j) {
        wf[j] = (float)w[j];
        if (sharpe) sharpe[j] = S[j];
        if (weights) weights[j] = wf[j];
    }
    return ensemble_set_weights(e, wf.data());
}

}  // extern "C"
