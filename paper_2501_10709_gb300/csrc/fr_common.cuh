// fr_common.cuh -- internal structures shared by the library's translation
// units: the device view of an environment batch, the ensemble's device
// images, error plumbing and launch helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/finrl_gb300.h"
#include "fr_rng.cuh"

namespace fr {

// ----------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

#define FR_CUDA(call)                                              \
    do {                                                           \
        cudaError_t e__ = (call);                                  \
        if (e__ != cudaSuccess) return ::fr::cuda_fail(e__, #call); \
    } while (0)

#define FR_CHECK(cond, code, ...)            \
    do {                                     \
        if (!(cond)) {                       \
            ::fr::set_error(__VA_ARGS__);    \
            return (code);                   \
        }                                    \
    } while (0)

// NVTX range, in the library's own domain "finrl_gb300", on the calling host
// thread for the duration of an ABI call: a profiler shows which call issued
// which launches (e.g. ncu --nvtx --nvtx-include "finrl_gb300@rollout/").
// Without an attached tool each push / pop is one test of a null pointer.
struct NvtxScope {
    explicit NvtxScope(const char *name)
    {
        nvtxEventAttributes_t a = {};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(domain(), &a);
    }
    ~NvtxScope() { nvtxDomainRangePop(domain()); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
    static nvtxDomainHandle_t domain()
    {
        static const nvtxDomainHandle_t d = nvtxDomainCreateA("finrl_gb300");
        return d;
    }
};
#define FR_NVTX(name) ::fr::NvtxScope fr_nvtx_scope_(name)

// --------------------------------------------------------- device layouts
constexpr int KP = 32;          // padded asset slots per env (one per lane)
constexpr int BPS_ONE = 10000;  // basis points per unit

// Device view of an env batch, passed by value to kernels.  Per-env state
// is structure-of-arrays; holdings and perturbations are [N][32] so one
// env's row is a single 128-byte (resp. 64-byte) line.
struct EnvView {
    int task, N, K, I, D;
    int hmax, fee_bps, pmax, auto_reset;
    int buy_order;              // FR_BUY_ASCENDING / FR_BUY_LARGEST_FIRST (stock)
    int narrow;                 // stock: prices, orders and step sums fit 32 bits (env_create proves it)
    int64_t init_cash;
    double ann;                 // Sharpe annualisation factor A
    // market
    int n_days;
    int64_t S;
    const int64_t *close;       // [n_days][K]
    const float *ind;           // [n_days][I][K]
    const int64_t *mid;         // [S]
    const uint8_t *spread;      // [S]
    const float *fac;           // [S][8]
    // per-env constants
    const int32_t *Ke;          // [N]
    const int32_t *start;       // [N]
    const int32_t *W;           // [N]
    const int16_t *bps;         // [N][32]
    // state
    int64_t *cash;              // [N]
    int32_t *hold;              // stock [N][32] shares; crypto [N] lots
    int32_t *t;                 // [N] steps taken this episode
    uint8_t *done;              // [N]
    // FP64 episode accumulators
    double *mu, *m2, *mdd;      // [N]
    int64_t *peak, *vlast;      // [N]
    double *latched;            // [N][4]: metrics of the last auto-reset episode + valid flag
    unsigned long long *err;    // [1] non-finite / invalid actions seen
};

}  // namespace fr

// ---------------------------------------------------------- opaque handles
struct fr_ctx {
    int device;
    int sm_count;
    uint64_t budget;
    uint64_t used;
    int cc_major, cc_minor;
};

struct fr_market {
    fr_ctx *ctx;
    int task;
    int n_days, K, I;
    int64_t S;
    int64_t close_max;          // largest close (stock), for the range proofs of the step kernel
    int64_t *close;
    float *ind;
    int64_t *mid;
    uint8_t *spread;
    float *fac;
    uint64_t bytes;
};

struct fr_ensemble;

struct fr_env {
    fr_ctx *ctx;
    const fr_market *mkt;
    fr::EnvView v;
    void *block;                // single allocation holding all per-env arrays
    uint64_t bytes;
    // scratch for the plain rollout path (grown on demand)
    void *scratch;
    uint64_t scratch_bytes;
    int path;                   // FR_PATH_*
    // asset-count slots of the fused stock kernel's indicator table
    int32_t *slot_of_env;       // device [N] (+ slot_ke [32] after it)
    int32_t *slot_ke;
    int n_slots;
    // the fused stock kernel's indicator rows and table Z, kept across
    // rollouts while the ensemble (by serial) and the slot set are unchanged
    void *zbuf;
    uint64_t zbuf_bytes;
    uint64_t z_serial;          // serial of the ensemble Z was built for; 0 = stale
    int z_cache_off;            // rebuild Z on every rollout
    // tile packing of the fused stock kernel (envs sorted by window into
    // 128-env tiles; each tile runs until its longest window is over)
    int pack_state;             // 0 unknown, 1 not packed (uniform windows), 2 packed
    int32_t *pack_perm;         // device [tiles*128] env at each tile position, -1 empty
    int32_t *pack_tile_w;       // device [tiles] longest window of each tile
    float pack_efficiency;      // sum(W_e - 1) / sum over tiles of 128 * (max W - 1)
    int pack_off;               // packing switched off by the caller
    // exploration of rollouts (kind, sigma, threshold, seed) and the global
    // step counter of its draws
    int explore_kind;
    float explore_sigma;
    uint32_t explore_thr;
    uint64_t explore_seed;
    uint32_t explore_step;
    // launch configuration chosen by env_autotune (tune_set = 0: the default
    // choice): path 2 the resident-weight fused kernel, 1 the first fused
    // kernel, 0 unfused; the first fused kernel's ring stages (0 = the most
    // that fit); whether the unfused path may use the large-batch actor kernel
    int tune_set;
    int tune_path;
    int tune_stages;
    int tune_tiled;
    // optional events around the main rollout kernel
    cudaEvent_t k_ev[2];
    int k_timing;               // record on the next rollouts
    int k_recorded;             // a pair has been recorded
    int last_ctas, last_tile;   // launch shape of the last fused stock rollout (0: none yet)
    // split fused stock rollouts: the pieces' stream (highest priority) and
    // its ordering events (created at first use)
    cudaStream_t split_stream;
    cudaEvent_t split_ev[5];    // one per piece, and the rollout's start
    int split_prio;
    int split_off;              // 1: never split (env_set_rollout_split)
};

namespace fr {
// The env's exploration settings for a rollout whose first step is global
// step g0.
inline Explore explore_of(const fr_env *env, uint32_t g0)
{
    Explore x;
    x.kind = env->explore_kind;
    x.sigma = env->explore_sigma;
    x.thr = env->explore_thr;
    x.k0 = (uint32_t)env->explore_seed;
    x.k1 = (uint32_t)(env->explore_seed >> 32);
    x.g0 = g0;
    return x;
}

// Record the timing event `which` (0 before, 1 after the main kernel) on s
// when timing is on.
cudaError_t env_time_mark(fr_env *env, int which, cudaStream_t s);
}  // namespace fr

namespace fr {

// Account `bytes` against the context budget; FR_ENOMEM when it would not fit.
int ctx_reserve(fr_ctx *ctx, uint64_t bytes);
void ctx_release(fr_ctx *ctx, uint64_t bytes);
// cudaMalloc with budget accounting.
int dev_alloc(fr_ctx *ctx, void **p, uint64_t bytes);
// true when an armed host fault injection (fr_fault_inject) fails this event
bool fault_hit(int kind);
void dev_free(fr_ctx *ctx, void *p, uint64_t bytes);

inline unsigned ceil_div(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Raise a kernel's dynamic shared-memory limit to the device's opt-in
// maximum, once per kernel and device (so that rollouts after the first make
// no such call and can be captured into a CUDA graph).  fr_api.cu.
cudaError_t set_max_smem_once(const void *func, int device);

// ------------------------------------------------------- kernel launchers
// env kernels (fr_env_kernels.cu)
cudaError_t launch_env_reset(const EnvView &v, cudaStream_t s);
// exploration of a step's combined actions in place (stock float [N][K],
// crypto uint8 [N]); x.g0 is this step's global step
cudaError_t launch_explore(const EnvView &v, void *act, const Explore &x, cudaStream_t s);
cudaError_t launch_env_step(const EnvView &v, int kind, const void *act,
                            int64_t *rew, float *rew_f32, uint8_t *done,
                            float *obs, int ld_obs, cudaStream_t s);
cudaError_t launch_env_observe(const EnvView &v, float *obs, int ld, cudaStream_t s);
cudaError_t launch_env_metrics(const EnvView &v, double *out, cudaStream_t s);
// the 8 indicators of a market from device close / high / low (fr_prep.cu)
cudaError_t launch_indicators(const int64_t *close, const int64_t *high, const int64_t *low, int T, int K,
                              float *ind, cudaStream_t s);
cudaError_t launch_env_get_state(const EnvView &v, int64_t *cash, int32_t *hold,
                                 int32_t *steps, uint8_t *done, cudaStream_t s);

}  // namespace fr

// ------------------------------------------------------------- ensembles
namespace fr {
constexpr int MAX_AGENTS = 8;
constexpr int MAX_LAYERS = 4;
constexpr int MAX_HIDDEN = 256;
struct TcImage;   // tensor-core weight images (fr_tc.cu)
}  // namespace fr

struct fr_ensemble {
    fr_ctx *ctx;
    int M, L;
    int dims[fr::MAX_LAYERS + 1];
    int precision, combine, out_act;
    int64_t P;                           // fp32 parameters per agent
    int64_t w_off[fr::MAX_LAYERS], b_off[fr::MAX_LAYERS];
    float *params;                       // device [M][P] fp32 master copy
    float *weights;                      // device [M] combine weights
    float host_weights[fr::MAX_AGENTS];
    int heads[fr::MAX_AGENTS];           // FR_HEAD_* per agent
    uint32_t dueling;                    // bit j: agent j has a dueling head
    int n_act;                           // actions (dims[L] - 1 with a dueling agent)
    fr::TcImage *tc;                     // tensor-core images or NULL
    uint64_t serial;                     // unique per created ensemble (cache key)
    uint64_t bytes;
};

namespace fr {
// Q-values of one agent's output row y: a plain head reads y_a; a dueling
// head gives (y_0 + y_{1+a}) - m with m = (y_1 + ... + y_n) / n summed in
// index order, every float32 operation rounded once.
struct HeadQ {
    const float *y;
    bool dueling;
    int nact;
    float m;
    __device__ __forceinline__ HeadQ(const float *y_, bool d, int n) : y(y_), dueling(d), nact(n), m(0.0f)
    {
        if (dueling) {
            float s = 0.0f;
            for (int b = 0; b < nact; ++b) s = __fadd_rn(s, y[1 + b]);
            m = __fdiv_rn(s, (float)nact);
        }
    }
    __device__ __forceinline__ float q(int a) const
    {
        return dueling ? __fsub_rn(__fadd_rn(y[0], y[1 + a]), m) : y[a];
    }
    // argmax, lowest index on ties
    __device__ __forceinline__ int argmax() const
    {
        int best = 0;
        float bq = q(0);
        for (int a = 1; a < nact; ++a) {
            const float qa = q(a);
            if (qa > bq) {
                bq = qa;
                best = a;
            }
        }
        return best;
    }
};

// plain fp32 kernels (fr_plain.cu)
cudaError_t launch_dense_f32(const float *X, int64_t x_stride, int ldx, const float *P,
                             int64_t p_stride, int64_t w_off, int64_t b_off, float *Y,
                             int64_t y_stride, int ldy, int n, int fin, int fout, int act, int M,
                             cudaStream_t s);
// max |x| of M matrices of `count` floats (stride apart) into out[j * out_stride]
// as float bits (atomic max; out zeroed by the caller)
cudaError_t launch_absmax(const float *x, int64_t stride, int64_t count, int M, unsigned *out, int out_stride,
                          cudaStream_t s);
cudaError_t launch_combine_mean(const float *Y, int64_t y_stride, int ldy, const float *w, int M,
                                int n, int K, float *out, int ldo, cudaStream_t s);
// Q-values after the heads, q [M][n][nact]; DQN-family learning targets [M][n]
cudaError_t launch_heads(const float *Y, int64_t y_stride, int ldy, int M, int n, int nact, uint32_t dueling,
                         float *q, cudaStream_t s);
cudaError_t launch_q_targets(const float *Yon, const float *Ytg, int64_t y_stride, int ldy, int M, int n, int nact,
                             uint32_t dueling, const float *rew, const uint8_t *done, float gamma, int double_q,
                             float *y, cudaStream_t s);
// majority vote of the agents' argmax actions; agents with bit j of
// `dueling` set take Q from a dueling head (fr_plain.cu)
cudaError_t launch_combine_vote(const float *Y, int64_t y_stride, int ldy, int M, int n, int nact,
                                uint32_t dueling, uint8_t *out, cudaStream_t s);

// Bytes of scratch the plain forward needs for n rows (two hidden buffers).
inline uint64_t plain_scratch_bytes(const fr_ensemble *e, int n)
{
    int w = 0;
    for (int l = 1; l < e->L; ++l) w = e->dims[l] > w ? e->dims[l] : w;
    return 2ull * (uint64_t)e->M * (uint64_t)n * (uint64_t)w * sizeof(float);
}
// Per-agent outputs y[M][n][dims[L]] from obs[n][ld] through the fp32 path.
cudaError_t forward_plain(const fr_ensemble *e, const float *obs, int ld, int n, float *y,
                          float *scratch, cudaStream_t s);

// tensor-core path (fr_tc.cu)
int tc_create(fr_ensemble *e);
void tc_destroy(fr_ensemble *e);
// Per-agent outputs through the tcgen05 kernels; obs rows of stride ld.
int tc_forward(const fr_ensemble *e, const float *obs, int ld, int n, float *y, cudaStream_t s);
// FP8 activation scales sx[j][l] (host [M][L]) of an FP8 ensemble (fr_tc.cu)
int tc_set_act_scales(fr_ensemble *e, const float *scales);
int tc_get_act_scales(const fr_ensemble *e, float *scales);
// Large-batch BF16 forward over tiled observations (fr_actor.cu): scratch of
// tc_tiled_scratch_bytes (0 = this ensemble has no such path).
uint64_t tc_tiled_scratch_bytes(const fr_ensemble *e, int n);
int tc_forward_tiled(const fr_ensemble *e, const float *obs, int ld, int n, float *y, void *scratch,
                     cudaStream_t s);
// Whether the fused persistent rollout supports this env / ensemble pair.
bool tc_rollout_supported(const fr_env *env, const fr_ensemble *e);
// FP64 episode accumulators from a rollout's value log (fr_fused.cu)
// t0 (NULL: the env's step counters) gives each env's step count before the
// logged steps.  With t0 the caller has already advanced the counters: the
// replay without auto-reset leaves them alone, the one with auto-reset
// writes them (its count restarts with every episode, as the kernel's).
cudaError_t launch_metrics_replay(const EnvView &v, const int64_t *vlog, int T, double *metrics,
                                  cudaStream_t s, const int32_t *t0 = nullptr);
// fused stock rollout with resident weights (fr_fused2.cu)
bool f2_supported(const fr_env *env, const fr_ensemble *e);
int f2_rollout(fr_env *env, const fr_ensemble *e, int T, const fr_traj *traj, double *metrics,
               cudaStream_t s);
void f2_release(const fr_ensemble *e);
int tc_rollout_max_stages(const fr_env *env, const fr_ensemble *e, int *chunks_per_step_out);
int tc_rollout(fr_env *env, const fr_ensemble *e, int T, const fr_traj *traj, double *metrics,
               cudaStream_t s);
}  // namespace fr
