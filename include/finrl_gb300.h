/*
 * finrl_gb300.h -- C ABI of the GB300 sampling library for the stock- and
 * crypto-trading environments of "Revisiting Ensemble Methods for Stock
 * Trading and Crypto Trading Tasks at ACM ICAIF FinRL Contests 2023/2024"
 * (arXiv 2501.10709).
 *
 * The library steps thousands of parallel trading environments (the paper's
 * VecEnv of SubEnvs, Sec. 4.2.2) on one GPU and evaluates an ensemble of actor
 * networks (Sec. 5.2) inside the same rollout.  Everything it computes runs
 * in its own CUDA kernels; there is no CPU fallback.
 *
 * Conventions shared by every call
 *  - Every function returns FR_OK (0) or a negative FR_E* status; no C++
 *    exception crosses the ABI.  fr_last_error() returns a message for the
 *    last failure on the calling thread.
 *  - Handles are opaque, owned by the library and released by *_destroy.
 *  - "device" pointers are CUDA device addresses on the context's device;
 *    "host" pointers are ordinary CPU memory.  Device pointers passed in are
 *    borrowed until the call's work completes on the given stream; host
 *    pointers are read (or written) before the call returns unless stated.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on that stream unless named *_sync or
 *    documented otherwise.
 *  - Money is int64 cents; holdings are integer shares (stock) or lots
 *    (crypto); neither is ever negative.
 */
#ifndef FINRL_GB300_H
#define FINRL_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define FR_OK 0
#define FR_EINVAL (-1)      /* bad argument, shape or configuration        */
#define FR_ENOMEM (-2)      /* allocation failed or HBM budget exceeded     */
#define FR_EBUSY (-3)       /* resource in use                              */
#define FR_ETIMEDOUT (-4)   /* a bounded device wait gave up                */
#define FR_ECUDA (-5)       /* a CUDA runtime call failed                   */
#define FR_ENOTREADY (-6)   /* asynchronous result not ready yet            */
#define FR_ENOTFOUND (-7)   /* unknown ticket                               */
#define FR_ECANCELED (-8)   /* a request cancelled before it completed      */

#define FR_TASK_STOCK 0
#define FR_TASK_CRYPTO 1

#define FR_MAX_ASSETS 32        /* K <= 32: one warp lane per asset          */
#define FR_MAX_INDICATORS 16
#define FR_CRYPTO_FACTORS 8
#define FR_CRYPTO_OBS_DIM 10    /* [cash, position, 8 factors]               */

/* Message describing the last failure on this thread ("" if none). */
const char *fr_last_error(void);

/* Library version string. */
const char *fr_version(void);

/* --------------------------------------------------------------- context */
typedef struct fr_ctx fr_ctx;

/* Create a context on CUDA device `device` that may hold at most
 * `hbm_budget_bytes` of device memory across all objects created from it
 * (0 = no limit).  Creation that would exceed the budget fails with
 * FR_ENOMEM. */
int fr_ctx_create(int device, uint64_t hbm_budget_bytes, fr_ctx **out);
void fr_ctx_destroy(fr_ctx *ctx);
/* Device bytes currently held by objects of this context. */
uint64_t fr_ctx_bytes_in_use(const fr_ctx *ctx);
/* Number of SMs of the context's device. */
int fr_ctx_sm_count(const fr_ctx *ctx);

/* ---------------------------------------------------------------- markets */
typedef struct fr_market fr_market;

/* Market tables, read from host memory at creation and then held resident
 * on the device (the paper keeps simulation data in GPU memory, Sec. 4.3.2).
 *  stock : close int64 [n_days][n_assets] cents (>= 1);
 *          ind float32 [n_days][n_ind][n_assets] technical indicators
 *          (Sec. 3.1, f_t), indicator-major within a day.
 *  crypto: mid int64 [n_seconds] cents per lot (>= 1); spread uint8
 *          [n_seconds] cents; fac float32 [n_seconds][8] factors. */
typedef struct {
    int32_t task;             /* FR_TASK_STOCK or FR_TASK_CRYPTO            */
    int32_t n_days;           /* stock                                      */
    int32_t n_assets;         /* stock, 1..32                               */
    int32_t n_ind;            /* stock, 0..16                               */
    const int64_t *close;     /* host                                       */
    const float *ind;         /* host                                       */
    int64_t n_seconds;        /* crypto                                     */
    const int64_t *mid;       /* host                                       */
    const uint8_t *spread;    /* host                                       */
    const float *fac;         /* host                                       */
    const int64_t *high;      /* host, stock with ind == NULL: see below    */
    const int64_t *low;       /* host                                       */
} fr_market_desc;

/* A stock market given ind == NULL, n_ind == 8 and daily high / low
 * (int64 cents [n_days][n_assets], low <= close <= high) computes its
 * indicator table on the device with market_indicators (below) instead of
 * reading one; the high / low tables are not kept. */
int fr_market_create(fr_ctx *ctx, const fr_market_desc *desc, fr_market **out);
void fr_market_destroy(fr_market *m);
/* Copy a stock market's resident indicator table (float32
 * [n_days][n_ind][n_assets]) to dst (host or device), synchronously. */
int fr_market_copy_indicators(const fr_market *m, float *dst);

/* The 8 technical indicators of the state's f_t (Sec. 3.1; the list of
 * Sec. 6.1), computed on the device from daily close / high / low (device
 * int64 cents [n_days][n_assets]) into ind (device float32
 * [n_days][8][n_assets], indicator-major within a day), each from data up to
 * its own day only:
 *   0  MACD(12, 26) / c          4  CCI-30 / 100
 *   1  (SMA20 + 2 sd20) / c - 1  5  DX-30 / 100
 *   2  (SMA20 - 2 sd20) / c - 1  6  SMA30 / c - 1
 *   3  RSI-30 / 100              7  SMA60 / c - 1
 * Textbook forms in FP64, each operation rounded separately (no fused
 * multiply-add), stored as the float32 rounding of the double:
 *  - windows of n trailing days, shorter at the start (t + 1 < n), summed
 *    from the oldest; sd the population deviation;
 *  - EMA e_t = a c_t + (1 - a) e_{t-1}, a = 2 / (n + 1), e_0 = c_0;
 *  - Wilder w_t = w_{t-1} + (x_t - w_{t-1}) / 30, w_0 = x_0;
 *  - RSI = 100 - 100 / (1 + G / L) over the smoothed gains G and losses L of
 *    c_t - c_{t-1} (0 at t = 0); 100 when L = 0 < G; 50 when G = L = 0;
 *  - CCI = (tp - SMA30(tp)) / (0.015 MAD30(tp)), tp = (h + l + c) / 3, 0 when
 *    the mean absolute deviation is 0;
 *  - DX = 100 |DI+ - DI-| / (DI+ + DI-), DI = 100 DM / TR over the smoothed
 *    directional movements (DM+ = h_t - h_{t-1} when it exceeds l_{t-1} - l_t
 *    and 0, DM- symmetric, both 0 at t = 0) and true range max(h - l,
 *    |h - c_{t-1}|, |l - c_{t-1}|) with c_{-1} = c_0; 0 when DI+ + DI- = 0.
 * Closes must be >= 1.  Asynchronous on `stream`; the tables are borrowed
 * until it completes.  FR_EINVAL for NULL tables or sizes < 1. */
int market_indicators(const int64_t *close, const int64_t *high, const int64_t *low, int32_t n_days,
                      int32_t n_assets, float *ind, void *stream);

/* ------------------------------------------------------------ environments */
typedef struct fr_env fr_env;

/* A batch of N independent environments over one market (the paper's VecEnv
 * of SubEnvs, Sec. 4.2.2; each trajectory is independent, Sec. 4.2.1).
 * Env e trades over the window start[e] .. start[e] + window[e] - 1 (days or
 * seconds): window[e] - 1 steps, after which it is done.
 *  stock : state [b, p, h, f] of Sec. 3.1, observation dimension
 *          D = 1 + 2K + I*K for the market's K assets and I indicators:
 *          [cash*1e-8, p_k*1e-4, h_k*1e-2, f_{i,k} (i outer, k inner)],
 *          each entry the float32 product (float)x * c_f (one rounding for
 *          the conversion, one for the product); assets k >= n_assets[e]
 *          read 0.
 *          Prices are the day's close scaled by (1e4 + bps[e][k]) / 1e4,
 *          rounded half up, floor 1 cent (Sec. 5.1 dataset diversity).
 *          Actions are share changes (Sec. 3.1): sells first, capped at the
 *          holding; then buys in ascending asset order (buy_order
 *          FR_BUY_ASCENDING) or largest requested count first, equal counts
 *          in ascending asset order (FR_BUY_LARGEST_FIRST), each filled as
 *          far as cash allows; fee ceil(notional * fee_bps / 1e4) per order.
 *          The fused rollout kernels take ascending order only; rollouts of
 *          largest-first envs run the unfused path.
 *  crypto: one asset; observation [cash*1e-8, pos/pmax, fac_0..7];
 *          action {0 sell, 1 hold, 2 buy} of one lot at bid = mid - s/2 or
 *          ask = bid + s; long-only, at most pmax lots; no fee.
 *  Reward (both): v_{t+1} - v_t with v = cash + holdings * price
 *  (Sec. 3.1), int64 cents; a float copy is (float)reward * 1e-6f.
 * K > 32, window < 2 or a window past the market end -> FR_EINVAL. */
typedef struct {
    int32_t task;
    int32_t n_envs;           /* N >= 1                                     */
    const int32_t *n_assets;  /* host [N] stock: 1..K (NULL = all K)        */
    const int32_t *window;    /* host [N] >= 2                              */
    const int32_t *start;     /* host [N] >= 0                              */
    const int16_t *bps;       /* host [N][K] stock, -100..100 (NULL = 0)    */
    int64_t init_cash;        /* cents, >= 0                                */
    int32_t hmax;             /* stock: shares per unit action, 1..1e6      */
    int32_t fee_bps;          /* stock: 0..10000                            */
    int32_t pmax;             /* crypto: lots, >= 1                         */
    int32_t auto_reset;       /* 1: a finished env restarts at once         */
    int32_t buy_order;        /* stock: FR_BUY_ASCENDING (0) or
                                 FR_BUY_LARGEST_FIRST (1); crypto: 0        */
} fr_env_desc;

#define FR_BUY_ASCENDING 0
#define FR_BUY_LARGEST_FIRST 1

int env_create(fr_ctx *ctx, const fr_env_desc *desc, const fr_market *market,
               fr_env **out);
void env_destroy(fr_env *env);
/* N, observation dimension D, market assets K (1 for crypto). */
int env_dims(const fr_env *env, int32_t *n_envs, int32_t *obs_dim,
             int32_t *n_assets);

/* reset (Sec. 4.2.2): every env back to its initial state: cash =
 * init_cash, no holdings, step 0, episode accumulators cleared. */
int env_reset(fr_env *env, void *stream);

#define FR_ACT_I32_SHARES 0   /* stock: int32 [N][K] share changes          */
#define FR_ACT_F32_UNIT 1     /* stock: float [N][K] in [-1,1] -> trunc(a*hmax)
                                 shares; NaN/Inf count as 0                  */
#define FR_ACT_U8_DISCRETE 2  /* crypto: uint8 [N] 0 sell, 1 hold, 2 buy    */

typedef struct {
    int32_t kind;             /* FR_ACT_*                                   */
    const void *data;         /* device                                     */
} fr_action;

/* Outputs of one step, each a device pointer or NULL. */
typedef struct {
    int64_t *rew;             /* [N] reward in cents                        */
    float *rew_f32;           /* [N] reward * 1e-6                          */
    uint8_t *done;            /* [N] 1 when the env's window is finished    */
    float *obs;               /* [N][D] observation after the step          */
} fr_step_out;

/* step + reward (Sec. 4.2.2): apply one action to every env.  A done env
 * (without auto_reset) is left unchanged and reports reward 0, done 1. */
int env_step(fr_env *env, const fr_action *action, const fr_step_out *out,
             void *stream);

/* Observation of the current state: obs device float [N][ld], ld >= D. */
int env_observe(fr_env *env, float *obs, int32_t ld, void *stream);

/* Copy of the state: cash [N] int64, holdings [N][K] int32 (crypto: [N]
 * lots), steps taken [N] int32, done [N] uint8 -- device pointers, any NULL. */
int env_get_state(fr_env *env, int64_t *cash, int32_t *hold, int32_t *steps,
                  uint8_t *done, void *stream);

/* Episode metrics [N][3] float64 (device): cumulative return v_T / v_0 - 1,
 * Sharpe ratio (mean - r_f) / std * sqrt(A) of per-period returns
 * (Sharpe equation, Sec. 5.2.1; ddof 1, r_f = 0, A = 252 stock, 1 crypto;
 * 0 with fewer than two periods or zero variance), maximum drawdown
 * min_t v_t / max_{s<=t} v_s - 1 (Sec. 6.1).  Accumulated in FP64 on the
 * device as the env steps.  After an auto-reset at the last step the
 * finished episode is reported. */
int env_metrics(fr_env *env, double *metrics, void *stream);

/* Checkpoint of the whole env state to host memory (synchronous).  With
 * host_buf NULL only *len receives the size needed. */
int env_snapshot(fr_env *env, void *host_buf, size_t cap, size_t *len);
/* Restore a snapshot taken from an env of the same task and shape. */
int env_restore(fr_env *env, const void *host_buf, size_t len);

/* Count of non-finite float actions and out-of-range discrete actions seen
 * since creation (each treated as 0 / hold). */
int env_error_count(fr_env *env, uint64_t *count);

/* -------------------------------------------------------------- ensembles */
typedef struct fr_ensemble fr_ensemble;

#define FR_PREC_FP32 0        /* plain unfused fp32 SIMT path               */
#define FR_PREC_BF16 1        /* tcgen05 BF16 tensor cores, fp32 accumulate */
#define FR_PREC_FP8 2         /* tcgen05 FP8 E4M3 weights+activations, per-
                                 channel weight scales, static activation
                                 scales (ensemble_calibrate_sync)            */
#define FR_PREC_BF16X3 3      /* tcgen05 BF16 with split hi/lo operands:
                                 x ~ hi + lo, three products per step
                                 (hi*hi + lo*hi + hi*lo), fp32-class accuracy
                                 for discrete (argmax / vote) decisions      */
#define FR_PREC_FP16 4        /* tcgen05 FP16 operands (round to nearest even,
                                 saturating at +-65504), fp32 accumulate:
                                 BF16's speed and memory with 10 stored
                                 mantissa bits instead of 7, for inputs,
                                 weights and activations of moderate range
                                 (no counterpart in the paper; an inference
                                 precision option)                           */

#define FR_HEAD_Q 0           /* outputs are the Q-values (DQN, Double DQN)  */
#define FR_HEAD_DUELING 1     /* outputs are [V, A_0 .. A_{n-1}] (Dueling DQN):
                                 Q_a = (V + A_a) - mean_b A_b                */

#define FR_COMBINE_MEAN 0     /* Sec. 5.2.1 weighted average of actions     */
#define FR_COMBINE_VOTE 1     /* Sec. 5.2.2 majority vote of argmax actions */

/* M actors of identical shape (Sec. 6.1 agent networks): L dense layers
 * dims[0] -> ... -> dims[L], ReLU on hidden layers, tanh (out_act = 1) or
 * identity (out_act = 0) on the output.  params: host float [M][P], per
 * layer W_l[out][in] row-major then b_l[out].  weights: host float [M]
 * (MEAN only; NULL = uniform 1/M).  MEAN combines as
 *   a = a_0 + sum_{j>=1} w_j (a_j - a_0),
 * which is the weighted average when the weights sum to one and exactly a_0
 * for identical agents; VOTE takes each agent's argmax (lowest index on
 * ties) and returns the action with the strictly largest count, else 1.
 * heads (VOTE only; Sec. 5.2.2 ensembles of DQN, Double DQN and Dueling DQN
 * agents): per-agent FR_HEAD_*, host [M], NULL = all FR_HEAD_Q.  With any
 * dueling agent the network has dims[L] = n_act + 1 outputs and a plain
 * agent's Q-values are its first n_act outputs; otherwise n_act = dims[L].
 * A dueling agent's Q-values are computed in float32 as
 * Q_a = (y_0 + y_{1+a}) - m, m = (y_1 + ... + y_{n_act}) / n_act summed in
 * index order, each operation rounded once.  Double DQN shares the DQN
 * forward; it differs only in its learning target (ensemble_q_targets). */
typedef struct {
    int32_t n_agents;         /* M, 1..8                                    */
    int32_t n_layers;         /* L, 1..4                                    */
    const int32_t *dims;      /* host [L+1]; hidden widths <= 256           */
    const float *params;      /* host [M][P]                                */
    const float *weights;     /* host [M] or NULL                           */
    int32_t precision;        /* FR_PREC_*                                  */
    int32_t combine;          /* FR_COMBINE_*                               */
    int32_t out_act;          /* 1 tanh, 0 identity                         */
    const int32_t *heads;     /* host [M] FR_HEAD_* (VOTE only) or NULL     */
} fr_ensemble_desc;

int ensemble_create(fr_ctx *ctx, const fr_ensemble_desc *desc,
                    fr_ensemble **out);
void ensemble_destroy(fr_ensemble *ens);

/* Per-agent Q-values after each agent's head: obs device float
 * [n][dims[0]], q device float [M][n][n_act].  VOTE ensembles only. */
int ensemble_q(const fr_ensemble *ens, const float *obs, int32_t n, float *q, void *stream);

/* Learning targets of the DQN family from replay samples (the consumer side
 * of Sec. 3.2 for the crypto agents of Sec. 5.2.2, evaluated on the GPU):
 * for every agent j of `online` and its counterpart in `target` (same
 * shapes, heads and precision class),
 *   a* = argmax_a Q_online_j(s', a) (Double DQN, double_q != 0) or
 *        argmax_a Q_target_j(s', a) (DQN), lowest index on ties;
 *   y_j = r + (done ? 0 : gamma * Q_target_j(s', a*)),
 * float32, each operation rounded once.  next_obs device float
 * [n][dims[0]], rew device float [n], done device uint8 [n] (NULL = none
 * done), y device float [M][n].  The update itself is out of scope. */
int ensemble_q_targets(const fr_ensemble *online, const fr_ensemble *target, const float *next_obs,
                       const float *rew, const uint8_t *done, int32_t n, float gamma, int32_t double_q,
                       float *y, void *stream);

/* FP8 E4M3 ensembles (no counterpart in the paper, whose agents run in
 * fp32; an inference-precision option of the actors).  Weights: row n of
 * layer l holds the E4M3 codes (round to nearest even, saturating at +-448)
 * of W[n][k] * (1 / sw[n]), sw[n] = max_k |W[n][k]| / 448 (1 for a zero
 * row), all float32 operations.  Activations: layer l's input x (the
 * observation for l = 0, else the ReLU output of layer l - 1) is quantised
 * as codes of x * (1 / sx[j][l]) with a static scale per agent j and layer.
 * The FP32 tensor-core accumulator is dequantised as
 * fma(acc, sx[j][l] * sw[n], b[n]); hidden layers then take ReLU, the output
 * tanh or identity.
 * An FP8 ensemble has no activation scales at creation: ensemble_forward,
 * ensemble_act and rollout return FR_ENOTREADY until they are set.
 *  ensemble_set_act_scales: scales host float [M][L], finite and > 0
 *    (FR_EINVAL otherwise or for a non-FP8 ensemble); synchronous.
 *  ensemble_get_act_scales: the current scales into host float [M][L].
 *  ensemble_calibrate_sync: sets sx[j][l] = max |x| / 448 over a calibration
 *    batch obs (device float [n][dims[0]], n >= 1), x the input of layer l
 *    of agent j through the fp32 master weights (1 where the maximum is 0);
 *    runs on `stream` and waits for it. */
int ensemble_set_act_scales(fr_ensemble *ens, const float *scales);
int ensemble_get_act_scales(const fr_ensemble *ens, float *scales);
int ensemble_calibrate_sync(fr_ensemble *ens, const float *obs, int32_t n, void *stream);

/* Per-agent network outputs: obs device float [n][dims[0]] (packed rows),
 * y device float [M][n][dims[L]]. */
int ensemble_forward(const fr_ensemble *ens, const float *obs, int32_t n,
                     float *y, void *stream);

/* Combined action for n observations (obs device float [n][dims[0]]):
 * MEAN -> act device float [n][dims[L]]; VOTE -> act device uint8 [n]. */
int ensemble_act(const fr_ensemble *ens, const float *obs, int32_t n,
                 void *act, void *stream);

/* ensemble_act without any allocation, for callers that must not allocate
 * device memory while they run: a real-time trading or serving loop that
 * reserved all its memory up front and must not stall in the allocator or
 * fail on fragmentation mid-run, or a host application or plugin framework
 * that owns every device buffer and forbids a library from allocating behind
 * its back.  The paper has no counterpart; this is a library convenience.
 * Same arguments, layouts and results as ensemble_act (on the tensor-core
 * precisions it always runs the single-agent kernel, which gives the same
 * results as the large-batch one).  Its scratch is a fixed 16 MiB array
 * inside the library image (held on every GPU that loads the library until
 * the process exits), so no cudaMalloc, cudaFree or other allocating routine
 * is called.  A batch whose scratch would not fit (roughly
 * (2*hidden + out)*M floats per row on the fp32 path, out*M on the
 * tensor-core paths) fails with FR_EINVAL and a message giving the largest
 * batch for this ensemble.  Each call looks up the array's device address
 * on the ensemble's device (a host query that allocates nothing).  After
 * cudaDeviceReset no handle of this library, this call included, may be
 * used again.  All calls share the one
 * array and it keeps the last call's contents: calls whose work overlaps on
 * the GPU (different streams, or different threads) race and must be
 * serialised by the caller. */
int ensemble_act_noalloc(const fr_ensemble *ens, const float *obs, int32_t n,
                         void *act, void *stream);

/* Replace a MEAN ensemble's combine weights (host float [M]); later
 * ensemble_act / rollout calls use them.  FR_EINVAL for VOTE ensembles or
 * non-finite weights. */
int ensemble_set_weights(fr_ensemble *ens, const float *weights);

/* Sharpe-softmax weighting from a validation window (Sec. 5.2.1): each
 * agent trades the validation envs alone (a single-agent ensemble of the
 * same precision) for T steps from their current state; its Sharpe ratio is
 * the mean over the envs of the episode Sharpe (env_metrics); agents with a
 * Sharpe ratio below `threshold` are discarded (when none reaches it, the
 * best agent is kept alone, lowest index on ties); the kept agents' weights
 * are softmax(Sharpe) = exp(S_j - max S) / sum_k exp(S_k - max S), the
 * discarded ones 0, and they become the ensemble's combine weights.  The
 * envs are restored to their state before the call.  sharpe (host double
 * [M]) and weights (host float [M]) receive the results (either may be
 * NULL).  MEAN ensembles only.  Synchronous. */
int ensemble_validate(fr_ensemble *ens, fr_env *val_env, int32_t T, double threshold,
                      double *sharpe, float *weights, void *stream);

/* Error flags raised on the device by the tensor-core kernels of this
 * ensemble (a bounded wait that gave up); 0 when none (synchronous). */
int ensemble_device_errors(const fr_ensemble *ens, uint32_t *flags);

/* ---------------------------------------------------------------- rollout */

/* Optional trajectory: the T x N x D sample tensors of Sec. 4.3.2, each a
 * device pointer or NULL.  Row t holds the observation the step acted on,
 * the combined action, the reward and the done flag. */
typedef struct {
    float *obs;               /* [T][N][obs_ld]                             */
    int32_t obs_ld;           /* >= D (0 = D)                               */
    void *act;                /* stock float [T][N][K]; crypto uint8 [T][N] */
    int64_t *rew;             /* [T][N]                                     */
    float *rew_f32;           /* [T][N]                                     */
    uint8_t *done;            /* [T][N]                                     */
} fr_traj;

/* T steps of observe -> ensemble -> step for every env (the simulation
 * phase of Sec. 3.2, parallel over trajectories as in Sec. 4.2.1).  The
 * ensemble's precision picks the path: FP32 runs the plain unfused kernels
 * (one launch per stage per step); BF16/FP8 run one fused persistent
 * kernel per rollout with tcgen05 tensor-core actors.  metrics: device
 * float64 [N][3] as env_metrics, written at the end, or NULL. */
int rollout(fr_env *env, const fr_ensemble *ens, int32_t T,
            const fr_traj *traj, double *metrics, void *stream);

/* Metrics of stored trajectories on the device (the consumer side of the
 * T x N sample tensors of Sec. 4.3.2).  rew: device int64 [T][N] rewards
 * v_t - v_{t-1}; done: device uint8 [T][N] or NULL.  Env i's periods are
 * its rows up to and including its first done row (all T rows when none);
 * its values are v_0 = v0 (cents, > 0), v_t = v_{t-1} + rew.  out: device
 * double [N][FR_TRAJ_METRICS] (with r_f = 0, A = ann, returns
 * rho_t = v_t / v_{t-1} - 1, ratios with a zero denominator reported as 0):
 *   0 cumulative return v_n / v_0 - 1; 1 Sharpe ratio (Sec. 5.2.1, as
 *   env_metrics); 2 maximum drawdown (<= 0); 3 annual return
 *   (v_n / v_0)^(A/n) - 1; 4 annual volatility sd(rho) sqrt(A) (ddof 1);
 *   5 RoMaD = cumulative return / |MDD|; 6 Sortino = mean(rho) / DD sqrt(A),
 *   DD = sqrt(sum min(rho, 0)^2 / n); 7 Calmar = annual return / |MDD|;
 *   8 Omega = sum max(rho, 0) / sum max(-rho, 0); 9 discounted return
 *   sum_{t=1..n} gamma^t r_t (Sec. 4.3, cents); 10 n.
 * (Sec. 6.1 metric list.)  Asynchronous on the stream. */
#define FR_TRAJ_METRICS 11
int trajectory_metrics(const int64_t *rew, const uint8_t *done, int32_t T, int32_t N, int64_t v0,
                       double ann, double gamma, double *out, void *stream);

/* Exploring rollouts (training producers; no counterpart in the paper's
 * evaluation, which acts greedily): applied by rollout() to the combined
 * action before it is discretised and recorded in the trajectory.
 *  FR_EXPLORE_GAUSSIAN  (stock) a_k + sigma z_k, z_k standard normal;
 *  FR_EXPLORE_EPS_GREEDY (crypto) the voted action is replaced, with
 *      probability floor(eps 2^24) / 2^24, by a uniform action in {0, 1, 2}.
 * Draws are Philox4x32-10 (Salmon et al. 2011) of key = seed and counter
 * (env, global step, asset, 0) for z (Box-Muller in float32 from
 * u = ((x >> 8) + 1/2) 2^-24 of the first two words) and (env, global step,
 * 0, 1) for the greedy draw (replace when word 2 >> 8 is below the
 * threshold; action floor(3 (word 3 >> 8) / 2^24)).  The global step of a
 * rollout's first step is the env's exploration counter, which every
 * rollout advances by T (not part of snapshots).  kind FR_EXPLORE_NONE or a
 * NULL x switches exploration off. */
#define FR_EXPLORE_NONE 0
#define FR_EXPLORE_GAUSSIAN 1
#define FR_EXPLORE_EPS_GREEDY 2
typedef struct {
    int32_t kind;
    float sigma;              /* >= 0, finite                               */
    float eps;                /* 0..1                                       */
    uint64_t seed;
} fr_explore;
int env_set_exploration(fr_env *env, const fr_explore *x);

/* Draw the per-env price perturbations of Sec. 5.1 on the device (each env
 * sees prices shifted by up to +-bps_range basis points per asset; the paper
 * uses +-1%, bps_range = 100).  For env e and asset k < the market's K:
 *   z = splitmix64(seed ^ splitmix64(e << 8 | k)),
 *   bps[e][k] = z mod (2 bps_range + 1) - bps_range,
 * splitmix64 the SplitMix64 output function (Steele, Lea, Flood, OOPSLA
 * 2014): x += 0x9E3779B97F4A7C15, then x ^= x >> 30, x *= 0xBF58476D1CE4E5B9,
 * x ^= x >> 27, x *= 0x94D049BB133111EB, x ^= x >> 31.  Assets >= K get 0.
 * The same draw as backtest_submit's, request env index for e.  Replaces the
 * env's bps table (asynchronous on `stream`); prices use it from the next
 * step on, so call it before env_reset for a fresh episode.  Stock envs only;
 * bps_range in 0..100 (FR_EINVAL otherwise). */
int env_perturb(fr_env *env, uint64_t seed, int32_t bps_range, void *stream);

#define FR_PATH_AUTO 0        /* fused kernel when the pair supports it     */
#define FR_PATH_UNFUSED 1     /* one launch per stage per step              */

/* Choose how rollout() runs this env (default FR_PATH_AUTO).  The fused
 * path covers stock envs over 30 assets with 8 indicators (mean combine,
 * tanh output) and crypto envs (vote combine) for BF16 / BF16X3 ensembles of
 * at most 8 agents; other pairs always run unfused. */
int env_set_rollout_path(fr_env *env, int32_t path);

/* Tile packing of the fused stock rollout (no counterpart in the paper;
 * default on).  When a rollout writes no trajectory, auto-reset is off and
 * the windows differ, the fused kernel processes the envs sorted by window
 * (longest first) in 128-env tiles and stops each tile after its longest
 * window, so short windows do not hold tiles for the whole horizon.  Every
 * env's results are unchanged.  env_tile_packing_efficiency reports, for the
 * current packing, sum over envs of (W - 1) / sum over tiles of 128 x (the
 * tile's longest W - 1) (1.0 when not packed). */
int env_set_tile_packing(fr_env *env, int32_t on);
int env_tile_packing_efficiency(const fr_env *env, float *eff);

/* The fused stock kernel's indicator table: the indicator part of the first
 * layer, W1[:, f] f + b1 for every (day, asset count) (the f block of the
 * state, Sec. 3.1, does not depend on the actions).  on = 1 (the default):
 * built by the first rollout and kept while the ensemble and the envs' asset
 * counts stay the same; on = 0: rebuilt by every rollout on its stream (the
 * cost a producer pays when its actors change between rollouts; the launches
 * are captured with the rollout into a graph).  No counterpart in the paper. */
int env_set_table_cache(fr_env *env, int32_t on);

/* Split fused stock rollouts (no counterpart in the paper).  on = 1 (the
 * default): a fused stock rollout of T >= 128 steps, without tile packing,
 * trajectory outputs or auto-reset, runs as K = min(4, T / 64) launches of
 * the resident kernel (the last T / 8 steps, the one before it T / 4, the
 * others sharing the rest evenly) on an internal stream of the highest
 * priority, and the FP64 metrics replay of each piece runs on `stream`
 * beside the next piece, so that only the last piece's replay follows the
 * kernel.  Events order the two streams, so the rollout is still one
 * ordered operation on `stream` and can be captured into a graph.  Results
 * are those of one launch, bit for bit.  on = 0: always one launch. */
int env_set_rollout_split(fr_env *env, int32_t on);

/* Autotuner of the batched rollouts (no counterpart in the paper: the
 * project's own choice of launch shape).  Times, for this env batch and
 * ensemble, the launch configurations the library has for the pair and keeps
 * the fastest for the env's later rollouts:
 *   path 2  the resident-weight fused stock kernel, tile packing on (packed =
 *           1) or off (only when the windows differ and auto-reset is off);
 *   path 1  the first fused kernel with `stages` weight-ring stages: the most
 *           that fit, the fewest that hold a whole step's weights resident,
 *           and 2 (weights streamed every step);
 *   path 0  the unfused path, with (tiled = 1) or without the large-batch
 *           actor kernel.
 * Each candidate runs a rollout of T_probe steps (1..4096) on the env's own
 * state three times (the first a warm-up; the mean of the other two, timed
 * with CUDA events on `stream`, is reported), the state restored from a host
 * snapshot before each run and at the end, so the env is left as it was.
 * The choice is also kept in a process-wide cache keyed by the pair's shape;
 * a later call with the same shape takes it without timing (cached = 1)
 * unless flags has FR_TUNE_FORCE.  Synchronous.  Tile packing, ring depth
 * and the actor kernel never change results; the three paths compute the
 * same function, each within the stated tolerance of the oracle.
 * env_tune_set pins one configuration (a path that does not apply to a pair
 * falls back as the default does: resident fused, first fused, unfused);
 * path 0..2, stages 0 (the most that fit) or >= 2.
 * env_tune_clear returns the env to the default choice (the resident fused
 * kernel, else the first fused kernel, else unfused; packing on). */
#define FR_TUNE_MAX 8
#define FR_TUNE_FORCE 1
typedef struct {
    int32_t n;                    /* configurations reported                 */
    int32_t chosen;               /* index of the one kept                   */
    int32_t cached;               /* 1: taken from the cache, not timed      */
    int32_t path[FR_TUNE_MAX];
    int32_t packed[FR_TUNE_MAX];
    int32_t stages[FR_TUNE_MAX];
    int32_t tiled[FR_TUNE_MAX];
    float ms[FR_TUNE_MAX];        /* mean time of a T_probe-step rollout     */
} fr_tune_report;
int env_autotune(fr_env *env, const fr_ensemble *ens, int32_t T_probe, int32_t flags, fr_tune_report *out,
                 void *stream);
int env_tune_set(fr_env *env, int32_t path, int32_t packed, int32_t stages, int32_t tiled);
int env_tune_clear(fr_env *env);

/* Kernel timing for roofline measurements (no counterpart in the paper).
 * With on != 0, every later rollout() of this env records two CUDA events
 * on its stream around the launch of its main rollout kernel only (the
 * fused kernel; on the unfused path, nothing is recorded).
 * env_last_kernel_ms waits for the last recorded pair and returns its
 * elapsed milliseconds in *ms; FR_EINVAL when no pair was recorded since
 * timing was switched on.  Timing adds two event records per rollout. */
int env_set_kernel_timing(fr_env *env, int32_t on);
int env_last_kernel_ms(fr_env *env, float *ms);

/* Launch shape of the last resident-weight fused stock rollout of this env
 * (no counterpart in the paper; for roofline accounting): *ctas = thread
 * blocks launched (clusters of 2M, one per SM), *tile_envs = envs per
 * cluster tile (64..128: a batch that does not fill the clusters the GPU
 * holds at once is spread over all of them).  FR_EINVAL before the first
 * such launch or on a NULL argument. */
int env_last_launch_shape(fr_env *env, int32_t *ctas, int32_t *tile_envs);

/* ---------------------------------------------------------- replay buffer */
typedef struct fr_replay fr_replay;

/* The replay buffer of the training process (Sec. 3.2: the reservoir
 * between the simulation phase and the learning phase), resident on the
 * device and fed by rollout trajectories (the T x N x D tensors of
 * Sec. 4.3.2).  A FIFO ring of `capacity` transitions (s, a, r, s', done):
 * s and s' float [D], a float [K] (stock) or uint8 (crypto), r the
 * learner's float reward copy, done uint8; shapes from `env`.  The number
 * of transitions pushed is kept on the device, so push and sample are
 * asynchronous on their stream (and may be captured into a graph).
 *  replay_create: capacity 1..2^31-1; FR_ENOMEM past the context budget.
 *  replay_push: appends the real steps of a T-step trajectory of `env` (obs,
 *    act, rew_f32 and done required; obs_ld as in fr_traj) in (t, env) order.
 *    Row (t, e) is a real step unless the env was done before it: without
 *    auto-reset, done[t-1][e] = 1, or for t = 0 live0[e] = 0 (live0 device
 *    uint8 [N], NULL = all live); with auto-reset every row is real.  s' of
 *    row (t, e) is obs[t+1][e], and last_obs[e] (device, rows obs_ld apart:
 *    the observation after the rollout, env_observe) for t = T - 1 (after
 *    a done row of an auto-reset env s' is the restarted env's first
 *    state; done marks it).  Once full, each new transition replaces the
 *    oldest.
 *  replay_sample: B transitions drawn uniformly with replacement from the
 *    current contents: draw b takes position floor(x * size / 2^32) (0 =
 *    oldest), x the first word of Philox4x32-10 with counter (b, counter low,
 *    counter high, 3) and key (seed low, seed high).  Outputs (device, each
 *    may be NULL): obs and next_obs float [B][D], act float [B][K] or uint8
 *    [B], rew float [B], done uint8 [B], index int64 [B] (the position).  An
 *    empty buffer writes index -1 and nothing else and sets error bit 0.
 *  replay_size_sync: current size (min(pushed, capacity)), transitions ever
 *    pushed and the error bits, after the stream's work so far. */
int replay_create(fr_ctx *ctx, const fr_env *env, int64_t capacity, fr_replay **out);
void replay_destroy(fr_replay *rb);
int replay_push(fr_replay *rb, const fr_env *env, const fr_traj *traj, int32_t T, const float *last_obs,
                const uint8_t *live0, void *stream);
int replay_sample(fr_replay *rb, int32_t B, uint64_t seed, uint64_t counter, float *obs, void *act,
                  float *rew, float *next_obs, uint8_t *done, int64_t *index, void *stream);
int replay_size_sync(fr_replay *rb, int64_t *size, int64_t *pushed, uint32_t *errors, void *stream);

/* ---------------------------------------------------------------- serving */
/* Backtests as requests: many independent backtests (each a group of envs
 * over one window, Sec. 4.2.1 trajectories) served by one GPU with
 * continuous batching.  A server owns one or more pools; a pool is an env
 * batch of `capacity` slots over one market, run with one ensemble in
 * chunks of `chunk_steps` steps on its own stream by its own host thread, so
 * the chunks of different pools (a stock and a crypto pool, say) overlap
 * on the device.  At every chunk boundary a pool retires the requests whose
 * windows are complete (their rows of the episode metrics go to the
 * caller's host buffer) and admits its queued requests in arrival order
 * while the freed slots and the server's HBM budget cover them; a request
 * waits while the one ahead of it in its pool does not fit.  Env state
 * stays resident in the pool; a request that records its trajectory keeps
 * it on the device (Sec. 4.3.2) until the caller fetches or releases it.
 * Submit, poll, fetch and release never wait for a running chunk.  No
 * counterpart in the paper beyond running many trajectories in parallel. */
typedef struct fr_server fr_server;

typedef struct {
    const fr_market *market;  /* the first pool's market (borrowed; outlives
                                 the server)                                */
    const fr_ensemble *ens;   /* the first pool's ensemble (borrowed);
                                 combine/output match the market's task     */
    int32_t capacity;         /* the first pool's env slots, >= 1           */
    int32_t chunk_steps;      /* the first pool's steps per launch, >= 1    */
    int64_t init_cash;        /* cents, >= 0 (every pool)                   */
    int32_t hmax;             /* stock: 1..1e6                              */
    int32_t fee_bps;          /* stock: 0..10000                            */
    int32_t pmax;             /* crypto: >= 1                               */
    uint64_t hbm_budget;      /* bytes of device memory the server may hold
                                 for admitted requests (below); 0 = no server
                                 limit (trajectory buffers are still bounded
                                 by the context's budget)                   */
} fr_server_desc;

/* Create / destroy.  Destroy stops the workers after their current chunks;
 * requests not yet complete are dropped (their tickets become unknown) and
 * trajectories not fetched are freed.
 * A rollout chunk that fails with a CUDA error fails every request and every
 * later submit (the context may be unusable); one that fails otherwise (e.g.
 * FR_ENOMEM when the context's budget cannot cover the rollout's scratch)
 * fails the requests of that chunk with that status, frees their slots, and
 * the pool goes on with its queued requests. */
int fr_server_create(fr_ctx *ctx, const fr_server_desc *desc, fr_server **out);
void fr_server_destroy(fr_server *srv);

/* Add a pool to the server for another (market, ensemble) pair, e.g. the
 * crypto pool beside a stock pool; its worker starts at once.  FR_EINVAL
 * when the ensemble does not match the market's observation and task, or
 * already has a pool in this server. */
int fr_server_add_pool(fr_server *srv, const fr_market *market, const fr_ensemble *ens, int32_t capacity,
                       int32_t chunk_steps);

/* One backtest: n_envs envs, env i over days (or seconds)
 * start + i*start_stride .. + window - 1; stock envs trade the first
 * n_assets assets with per-env per-asset price perturbations drawn from
 * `seed` uniformly in [-bps_range, bps_range] basis points (Sec. 5.1;
 * env_perturb's rule, drawn on the device, with e the env's index within the
 * request).  The request goes to the pool of `ens`, or with ens NULL to the
 * first pool of `task`.  metrics: caller-owned host buffer
 * double [n_envs][3] (cumulative return, Sharpe, max drawdown, as
 * env_metrics), written by the server before the request reports done; it
 * must stay valid until then.  want_traj = 1: the server also records the
 * request's T x N x D trajectory (T = window - 1 rows of n_envs envs:
 * observation, combined action, reward, done, as rollout's fr_traj) into a
 * device buffer of its own, kept after completion until backtest_fetch_traj
 * or backtest_release.
 * HBM budget: a request is charged n_envs times its pool's state bytes per
 * slot, plus with want_traj T * n_envs * (4 D + 4 K + 9) bytes (stock) or
 * T * n_envs * (4 D + 10) (crypto); a pool admits its queue head only when
 * the server's charged bytes plus the head's stay within hbm_budget.  The
 * slot charge returns when the request completes or fails; the trajectory
 * charge when it is fetched or released.
 * Errors at submit: bad fields, a task or ensemble no pool serves, or a
 * window past the market end -> FR_EINVAL; n_envs above the pool's capacity
 * or a charge above hbm_budget (can never fit) -> FR_ENOMEM; a server whose
 * worker failed -> that error.  A request that fits later is queued; one
 * whose trajectory buffer the context's budget cannot hold at admission
 * completes with status FR_ENOMEM. */
typedef struct {
    int32_t n_envs;
    int32_t window;           /* >= 2                                       */
    int32_t start;            /* >= 0                                       */
    int32_t start_stride;     /* >= 0                                       */
    int32_t n_assets;         /* stock: 1..K (0 = K)                        */
    int32_t bps_range;        /* stock: 0..100                              */
    uint64_t seed;
    int32_t want_traj;        /* 0 or 1                                     */
    double *metrics;          /* host [n_envs][3]                           */
    double timeout_s;         /* > 0: a request not complete this long after
                                 submit ends with status FR_ETIMEDOUT (checked
                                 at chunk boundaries); 0 = none             */
    int32_t task;             /* FR_TASK_STOCK or FR_TASK_CRYPTO            */
    const fr_ensemble *ens;   /* the pool's ensemble, or NULL               */
} fr_request;

typedef struct {
    int32_t status;           /* FR_OK, or the error that failed it         */
    int32_t n_envs;
    double queue_s;           /* submit -> admitted into slots              */
    double latency_s;         /* submit -> metrics written                  */
    int32_t task;
    int32_t traj_steps;       /* rows of the kept trajectory (0: none)      */
    uint64_t traj_bytes;      /* device bytes it holds until fetched        */
} fr_result;

int backtest_submit(fr_server *srv, const fr_request *req, uint64_t *ticket);

/* Non-blocking.  Running or queued: FR_ENOTREADY, *done = 0.  Complete:
 * FR_OK, *done = 1, *out filled; the ticket is then released (a later poll
 * returns FR_ENOTFOUND) unless a trajectory is kept, which keeps the ticket
 * until backtest_fetch_traj or backtest_release.  Unknown ticket:
 * FR_ENOTFOUND. */
int backtest_poll(fr_server *srv, uint64_t ticket, fr_result *out, int32_t *done);

/* Copy a completed request's kept trajectory into dst (device or host
 * pointers, each nullable: obs float [T][n_envs][obs_ld] (obs_ld >= D, 0 = D),
 * act float [T][n_envs][K] (stock) or uint8 [T][n_envs] (crypto), rew int64
 * [T][n_envs], done uint8 [T][n_envs]; rew_f32 is not kept and is ignored),
 * on `stream`, wait for the copies, then free the server's copy, return its
 * budget charge and release the ticket.  FR_ENOTREADY while the request
 * runs; FR_ENOTFOUND for a ticket without a kept trajectory. */
int backtest_fetch_traj(fr_server *srv, uint64_t ticket, const fr_traj *dst, void *stream);

/* Free a completed request's kept trajectory without copying it and
 * release the ticket (FR_ENOTREADY while it runs, FR_ENOTFOUND unknown). */
int backtest_release(fr_server *srv, uint64_t ticket);

/* Cancel a request.  Queued: it completes at once with status FR_ECANCELED.
 * Running: it is retired at the next chunk boundary with status
 * FR_ECANCELED (its slots freed, its metrics buffer left unwritten, no
 * trajectory kept).  Complete but not yet polled: no effect.  Either way the
 * ticket is polled as usual.  Unknown ticket: FR_ENOTFOUND.  Other requests
 * are unaffected. */
int backtest_cancel(fr_server *srv, uint64_t ticket);

typedef struct {
    uint64_t submitted, completed, queued, running;
    double env_steps;         /* slot-steps of requests completed (windows) */
    double pool_steps;        /* capacity x steps launched, all pools       */
    double busy_s;            /* wall time of the workers' GPU rounds       */
    uint64_t failed;          /* requests finished with an error other than
                                 FR_ECANCELED and FR_ETIMEDOUT              */
    uint64_t canceled;        /* finished with FR_ECANCELED                 */
    uint64_t timed_out;       /* finished with FR_ETIMEDOUT                 */
    uint64_t bytes_reserved;  /* budget bytes charged now                   */
    uint64_t bytes_peak;      /* the most charged at once                   */
    uint64_t budget;          /* hbm_budget (0 = none)                      */
    uint64_t pools;
} fr_server_stats;

int fr_server_stats_get(fr_server *srv, fr_server_stats *out);

/* ------------------------------------------------- host fault injection
 * For tests of the error paths, process-wide, on the host only: no GPU work
 * is faulted, each injected failure returns the error code the real failure
 * would.  Of the next events of `kind`, the first `skip` proceed and the
 * `count` after them fail; count 0 disarms the kind.
 *  FR_FAULT_ALLOC   a device allocation charged to a context fails: the call
 *                   that needed it returns FR_ENOMEM
 *  FR_FAULT_SUBMIT  backtest_submit rejects the request: FR_EBUSY, nothing
 *                   is queued
 *  FR_FAULT_POLL    backtest_poll drops its answer: FR_ENOTREADY, *done = 0;
 *                   a finished result stays for the next poll
 * FR_EINVAL for an unknown kind or a negative skip / count. */
/* Device check of the bounded waits behind FR_ETIMEDOUT: one block waits,
 * with the limit limit_us (1..2e6), on mbarrier phases that nothing
 * completes, in both forms the fused kernels use (one thread; a whole warp
 * with a warp vote), and once on a phase that does complete.  Synchronous.
 * Returns FR_ETIMEDOUT when a wait gave up -- the designed outcome: *flags =
 * 3 (bit 0 the one-thread wait, bit 1 the warp wait; bit 2 would mean the
 * completed phase was missed) and waited_ns[2] (nullable) the time each of
 * the first two waited -- and the context stays usable.  FR_OK if no wait
 * gave up; FR_ECUDA on a launch or copy error. */
int fr_wait_selftest(fr_ctx *ctx, int32_t limit_us, uint32_t *flags, uint64_t *waited_ns);

#define FR_FAULT_ALLOC 1
#define FR_FAULT_SUBMIT 2
#define FR_FAULT_POLL 3
int fr_fault_inject(int32_t kind, int32_t skip, int32_t count);

#ifdef __cplusplus
}
#endif
#endif /* FINRL_GB300_H */
