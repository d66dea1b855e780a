// fr_fused2.cu -- fused stock rollout with resident weights.
//
// One thread-block cluster of 2M CTAs owns a tile of up to 128 envs for all
// T steps (a batch too small to fill the co-resident clusters is spread over
// all of them, at least 64 envs per tile).  CTA (j, h) -- cluster rank 2j + h -- holds output half h of every
// hidden layer of agent j, so each agent's BF16 weights stay resident in
// shared memory, split over a CTA pair, and are never re-read per step:
//
//   layer 1  the state is [cash, p, h, f] (Sec. 3.1).  Its indicator block f
//            depends only on the day and the env's asset count, never on the
//            actions, so  W1[:, f] f + b1  is precomputed per (day, asset
//            count) into a table Z by a separate GEMM; per step the tensor
//            cores only multiply the 61 trajectory-dependent entries
//            (cash, prices, holdings; K = 64) and the epilogue adds Z;
//   layer 2  full h1 (both halves: the partner writes its half into this
//            CTA's A operand through distributed shared memory), N-half;
//   layer 3  K-split: both halves send their fp32 partial sums of each row
//            straight to the env's owner CTA, which adds them and the bias
//            and applies tanh (one exchange instead of a partner exchange
//            followed by a push of the finished actions).
//
// Env r of the tile is owned by the CTA of rank r mod 2M: one warp per env
// (8 or 16 warps per CTA, one to four envs each), lane = asset, state in
// registers.  The owner combines the agents' actions
// (anchored weighted mean, Sec. 5.2.1), discretises, trades, and writes the
// env's next observation row straight into every CTA's A operand.  The
// step's three cluster exchanges (observation rows, h1 halves, layer-3
// partial sums) are asynchronous stores that complete transaction bytes on
// the receiving CTA's mbarrier, armed once per phase; all waits are bounded
// by the global timer.  The shared buffers need no double buffering: every
// write of step s + 1 depends, through the step's chain, on every read of
// step s.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "fr_env_dev.cuh"
#include "fr_ptx.cuh"
#include "fr_tc.cuh"

namespace fr {

namespace {

// Warps per CTA: 8, or 16 when both hidden widths are multiples of 128 (each
// warp then takes a quarter of its lane quarter's columns, and one or two
// owned envs).  Every warp is an env / epilogue warp; warp 0 also loads the
// weights and issues the MMAs.  16 warps halve each warp's epilogue and owner
// work at 128 registers per thread (8 warps: up to 255).
constexpr int SK2 = 30, SI2 = 8;
constexpr int SD2 = 1 + 2 * SK2 + SI2 * SK2;   // 301
constexpr int NSTATE = 1 + 2 * SK2;            // 61 trajectory-dependent entries
constexpr int KS = 64;                         // their padded K
constexpr int NIND = SI2 * SK2;                // 240 indicator entries
constexpr int64_t VLOG_NONE2 = INT64_MIN;

// One CTA's resident weights: three layers, chunked canonical layout.
struct F2Layer {
    int K, N;             // padded
    int KC, n_chunks;
    uint32_t off;         // byte offset in the CTA image
};

struct F2Plan {
    int M, H1, H2;        // agents, hidden widths
    int fp8;              // E4M3 operands (kind::f8f6f4) instead of BF16
    int esz, ck, kmma;    // operand bytes, elements per 16-byte core row, K per MMA
    int n1, n2;           // N of layer 1 / 2 halves (H/2)
    F2Layer l1, l2, l3;
    uint32_t cta_bytes;   // weights per CTA (multiple of 1024)
    uint32_t a_bytes;     // A operand bytes (max K / 8 * 2048)
};

struct F2Image {
    F2Plan plan;
    uint8_t *img;         // device [M][2][cta_bytes]
    // FP8: dequantisation factors sx[l] * sw[n] [M][3][256] (layer 1: the
    // state columns' codes; layer 3: the 30 outputs) and 1 / sx[l] [M][4]
    float *dq = nullptr;
    float *inv_sx = nullptr;
    uint32_t scale_version = 0;
    float *b2;            // device [M][H2]
    float *b3;            // device [M][32]
    float *wind;          // device [M][240*H1 + H1]: W1 indicator columns transposed ([c][n]), then b1
    const fr_ensemble *owner;
    uint64_t bytes;
};

struct F2Args {
    EnvView v;
    F2Plan plan;
    const uint8_t *img;
    const float *b2, *b3;
    const float *dq, *inv_sx;   // FP8 only
    const float *Z;       // [M][n_ctx][H1]
    const int32_t *slot; // [N] asset-count slot of each env
    const int32_t *perm; // [tiles*tile_rows] env at each tile position (NULL = identity; -1 = empty)
    const int32_t *tile_w; // [tiles] longest window of a tile's envs (NULL = run every tile T steps)
    int n_pos;            // tile positions holding an env index (N, or tiles*tile_rows with perm)
    int tile_rows;        // envs per tile (<= 128; the MMA rows beyond are padding)
    int n_ctx_per_agent;
    float w[MAX_AGENTS];
    int T;
    float *tr_obs;
    int obs_ld;
    float *tr_act;
    int64_t *tr_rew;
    float *tr_rew_f32;
    uint8_t *tr_done;
    int64_t *vlog;
    int32_t *t0_out;      // [N] each env's step count at the launch's start (for the replay)
    unsigned *err;
    Explore ex;           // exploration of the combined actions
};

bool f2_plan(const fr_ensemble *e, F2Plan &p)
{
    if (e->L != 3 || e->dims[0] != SD2 || e->dims[3] != SK2 || e->M > 4 || e->M < 2) return false;
    p.M = e->M;
    p.H1 = e->dims[1];
    p.H2 = e->dims[2];
    p.fp8 = e->precision == FR_PREC_FP8 ? 1 : 0;
    p.esz = p.fp8 ? 1 : 2;
    p.ck = p.fp8 ? 16 : 8;
    p.kmma = p.fp8 ? 32 : 16;
    if (p.H1 % 64 || p.H2 % 64 || p.H1 > 256 || p.H2 > 256) return false;
    p.n1 = p.H1 / 2;
    p.n2 = p.H2 / 2;
    uint32_t off = 0;
    auto mk = [&](F2Layer &l, int K, int N) {
        l.K = K;
        l.N = N;
        int kc = (int)(TC_CHUNK_MAX / (uint32_t)(N * p.esz)) / p.kmma * p.kmma;
        l.KC = std::min(kc, K);
        l.n_chunks = (K + l.KC - 1) / l.KC;
        l.off = off;
        off += (uint32_t)(N * K * p.esz);
    };
    mk(p.l1, KS, p.n1);
    mk(p.l2, p.H1, p.n2);
    mk(p.l3, p.n2, 32);
    p.cta_bytes = (off + 1023u) & ~1023u;
    // A operand: h1 in chunks [0, H1/8) (layer 2), the observation's state
    // part in its own chunks [H1/8, H1/8 + 8) so that the partner's h1 half
    // can never land on an observation this CTA's layer 1 is still reading;
    // h2's half (layer 3) reuses chunks [0, n2/8)
    p.a_bytes = (uint32_t)(p.H1 / p.ck + KS / p.ck) * 2048u;
    return true;
}

// K position in layer 1's operands of state entry k (0 cash, 1..30 prices,
// 31..60 holdings): prices and holdings interleaved by asset, cash last.
__host__ __device__ inline int f2_state_pos(int k) { return k == 0 ? 2 * SK2 : (k <= SK2 ? 2 * (k - 1) : 2 * (k - 1 - SK2) + 1); }

// Rows of a tile owned by one CTA: row r belongs to rank r mod 2M and sits
// at index r / 2M of that CTA's owned rows.  A tile holds tr <= 128 envs
// (rows tr..127 of the MMAs are padding that nothing reads back); the
// owned-row buffers are sized for 128.
__host__ __device__ inline int f2_owned_rows(int M) { return (128 + 2 * M - 1) / (2 * M); }
__host__ __device__ inline int f2_rows_of(int tr, int M, int rank) { return rank < tr ? (tr - 1 - rank) / (2 * M) + 1 : 0; }

// Observation bytes a CTA receives per step from the other CTAs: the 64
// state entries (BF16: 128 bytes, E4M3: 64) and the Z row index (4 bytes)
// of every row of the tile it does not own.
__host__ __device__ inline uint32_t f2_obs_tx_bytes(int M, int rank, int esz, int tr)
{
    return (uint32_t)(tr - f2_rows_of(tr, M, rank)) * (uint32_t)(64 * esz + 4);
}

// h1 bytes a CTA receives per step from its partner: the tile's rows of the
// partner's H1 / 2 columns.
__host__ __device__ inline uint32_t f2_h1_tx_bytes(const F2Plan &p, int tr)
{
    return (uint32_t)tr * (uint32_t)p.n1 * (uint32_t)p.esz;
}

// Layer-3 partial-sum bytes a CTA receives per step from the other 2M - 1
// CTAs: 128 bytes for each of its owned rows from each.
__host__ __device__ inline uint32_t f2_x_tx_bytes(int M, int rank, int tr)
{
    return (uint32_t)(f2_rows_of(tr, M, rank) * (2 * M - 1)) * 128u;
}

// shared-memory carve-up
struct F2Smem {
    uint32_t w, a, xbuf, ctx, bias, bars, total;
};

__host__ __device__ inline F2Smem f2_smem(const F2Plan &p)
{
    F2Smem s;
    s.w = 0;
    s.a = p.cta_bytes;
    // [2M][owned rows][32] fp32 layer-3 partial sums of this CTA's owned
    // rows, one block per sending CTA (agent j, half h at block 2j + h)
    s.xbuf = s.a + p.a_bytes;
    s.ctx = s.xbuf + (uint32_t)(2 * p.M * f2_owned_rows(p.M)) * 128u;   // [128] int32 Z row of each env
    // this CTA's b2 half [128], b3 of every agent [4][32]; FP8: this CTA's
    // dq1 and dq2 halves [128] each, dq3 of every agent [4][32], this
    // agent's 1 / sx[0..2]
    s.bias = s.ctx + 512u;
    s.bars = s.bias + 3072u;
    s.total = s.bars + 256u;
    return s;
}

// pieces of a split rollout (launches of the resident kernel per rollout)
constexpr int F2_PIECES_MAX = 4;

// barrier slots
enum { B_W = 0, B_OBS, B_ACC, B_H1, B_H2, B_X, B_END, B_COUNT };

__device__ __forceinline__ bool f2_wait(uint64_t *bar, uint32_t parity, volatile int *abort, unsigned *err,
                                        unsigned code, bool cluster_scope)
{
    return ptx::warp_wait_all(bar, parity, cluster_scope, abort, err, code, TC_WAIT_NS);
}

// ------------------------------------------------------------- MMA issue
// One layer of this CTA's agent half: K-steps of 16 over the resident
// weight chunks, accumulator in TMEM, completion signalled on `acc`.  Issued
// by lane 0 of env warp 0 at the point where that warp waits on the layer's
// operands anyway; a dedicated issuer warp would make the block 10 warps,
// which caps every thread at 168 registers and makes the env code spill.
// The layer's shape comes by value (K, N, byte offset): a reference would
// take the address of the caller's plan and keep it in local memory.
template <bool FP8>
__device__ __noinline__ void f2_layer(int K, int N, uint32_t off, uint32_t d_tmem, uint32_t a_at, uint32_t w_base,
                                      uint64_t *acc)
{
    using namespace ptx;
    fence_proxy_async_smem();
    tc_fence_after();
    // one MMA per K step of 16 (BF16) or 32 (E4M3) elements: two 16-byte
    // core-matrix columns of A and of B either way
    const uint32_t idesc = FP8 ? idesc_e4m3(128, N) : idesc_bf16(128, N);
    const uint32_t lbo_b = (uint32_t)(N * 16);
    // the layer's resident weights are its K-major core-matrix columns end to
    // end (the image's chunks are contiguous), so both descriptors advance by
    // constant offsets per K = 16 step: 2 columns of A (4,096 B) and of B
    // (2 N 16 B), in the start-address field's 16-byte units
    uint64_t ad = smem_desc(a_at, 2048u, 128u);
    uint64_t bd = smem_desc(w_base + off, lbo_b, 128u);
    const uint64_t b_step = (uint64_t)((2u * lbo_b) >> 4);
    constexpr int KM = FP8 ? 32 : 16;
    if (FP8)
        mma_e4m3(d_tmem, ad, bd, idesc, 0u);
    else
        mma_bf16(d_tmem, ad, bd, idesc, 0u);
    for (int k = KM; k < K; k += KM) {
        ad += 256u;
        bd += b_step;
        if (FP8)
            mma_e4m3(d_tmem, ad, bd, idesc, 1u);
        else
            mma_bf16(d_tmem, ad, bd, idesc, 1u);
    }
    mma_commit(acc);
}

// The executed (and recorded) action explores: a + sigma z of env e, global
// step g, asset k.  Out of line: the step loop stays small when exploration
// is off.
__device__ __noinline__ float f2_explore(Explore x, float act, uint32_t e, uint32_t g, uint32_t k)
{
    return __fadd_rn(act, __fmul_rn(x.sigma, explore_normal(x, e, g, k)));
}

// --------------------------------------------- owner: one env, warp-wide
struct OwnEnv {
    int64_t cash;        // uniform
    int64_t v0;          // uniform: total asset value at the start of the step
    int t, start, W, Ke; // uniform
    int done;            // uniform
    int slot;            // uniform, asset-count slot
    int64_t p;           // this lane's asset price at day start + t
    int32_t h;           // this lane's holding
    int bps;             // this lane's perturbation
};

// Greedy buys in ascending asset order with partial fills, for the case
// where the orders do not all fit in `cash`: lanes whose single share no
// longer fits drop out; a scan finds the first order that does not fit,
// which buys what the remaining cash affords.  Returns the cash left and
// this lane's filled shares (by value: an output reference would put the
// caller's variable in local memory).  cash and the loop state stay
// warp-uniform, so every collective runs on the full warp.
// NARROW: every order's cost and the sum of all of them fit 32 bits, so the
// prefix scan runs on 32-bit values (same sums).
struct Fill {
    int64_t cash, nb;
};

template <bool NARROW>
__device__ __noinline__ Fill own_buy_greedy(int64_t cash, int64_t want, int64_t full, int64_t p, int fee, int lane)
{
    int64_t nb;
    const int64_t one = NARROW ? (int64_t)cost_of32(1u, (uint32_t)p, fee) : cost_of(1, p, fee);
    unsigned pending = __ballot_sync(FULL_MASK, want > 0);
    nb = 0;
    while (pending) {
        bool mine = (pending >> lane) & 1u;
        pending &= ~__ballot_sync(FULL_MASK, mine && one > cash);
        if (!pending) break;
        mine = (pending >> lane) & 1u;
        const int64_t x = mine ? full : 0;
        int64_t pre;
        if (NARROW) {
            uint32_t y = (uint32_t)x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t z = __shfl_up_sync(FULL_MASK, y, o);
                if (lane >= o) y += z;
            }
            pre = (int64_t)y;
        } else {
            pre = warp_incl_scan(x, lane);
        }
        const unsigned fail = __ballot_sync(FULL_MASK, mine && pre > cash);
        if (fail == 0u) {
            if (mine) nb = want;
            cash -= __shfl_sync(FULL_MASK, pre, 31);
            break;
        }
        const int f = __ffs(fail) - 1;
        if (mine && lane < f) nb = want;
        int64_t cf = cash - (pre - x);
        if (lane == f) {
            // the failing order: cf is below its cost, so (NARROW) below 2^32
            const int64_t n = NARROW ? (int64_t)afford32((uint32_t)cf, (uint32_t)p, fee, (uint32_t)want)
                                     : afford(cf, p, fee);
            nb = n;
            cf -= NARROW ? (int64_t)cost_of32((uint32_t)n, (uint32_t)p, fee) : cost_of(n, p, fee);
        }
        cash = __shfl_sync(FULL_MASK, cf, f);
        pending &= ~((2u << f) - 1u);
    }
    return Fill{cash, nb};
}

// fp32 trajectory observation of the step about to be taken (optional output,
// out of line)
__device__ __noinline__ void own_traj_obs(const F2Args &a, float *o, float cv, float pv, float hv, int day, int Ke,
                                          int lane)
{
    if (lane == 0) o[0] = cv;
    if (lane < SK2) {
        o[1 + lane] = pv;
        o[1 + SK2 + lane] = hv;
    }
    const float *f = a.v.ind + (int64_t)day * NIND;
    for (int i = lane; i < NIND; i += 32) o[NSTATE + i] = (i % SK2) < Ke ? __ldg(f + i) : 0.0f;
}

// The next observation row of env r: its 61 state entries in the A
// operand's K order, which puts asset k's price and holding side by side:
// position 2k = price k, 2k + 1 = holding k (k < 30), 60 = cash, 61..63 zero
// (layer 1's weight columns are packed in the same order; the dot product
// does not depend on it).  So lane k's (price, holding) pair is one BF16x2
// word (lane 30: cash and 0; lane 31: 0) and chunk c, positions 8c..8c+7, is
// the words of lanes 4c..4c+3: four shuffles per row.  E4M3: lane k's pair is
// 16 bits, two lanes make a word, chunk c (16 positions) is the words of
// lanes 8c, 8c + 2, 8c + 4, 8c + 6.  Every lane builds the chunk it stores,
// so that the stores to the cluster's CTAs spread over all lanes.
struct ObsWords {
    uint32_t w0, w1, w2, w3;
    int zrow;
    float pv, hv, cv;
};

template <bool NARROW, bool FP8>
__device__ __forceinline__ ObsWords own_words(const F2Args &a, const OwnEnv &s, bool valid, int lane, float inv0)
{
    ObsWords o;
    // NARROW prices are below 2^31: the 32-bit conversion rounds the same
    o.pv = (valid && lane < s.Ke) ? (NARROW ? __fmul_rn(__int2float_rn((int)s.p), 1e-4f) : obs_scale(s.p, 1e-4f))
                                  : 0.0f;
    o.hv = (valid && lane < s.Ke) ? __fmul_rn(__int2float_rn(s.h), 1e-2f) : 0.0f;
    o.cv = valid ? obs_scale(s.cash, 1e-8f) : 0.0f;
    o.zrow = valid ? s.slot * a.v.n_days + s.start + s.t : 0;
    if (FP8) {
        // E4M3 codes of value * (1 / sx[0]) (the agents share the scale)
        const uint32_t pair = lane < SK2 ? e4m3x2(__fmul_rn(o.pv, inv0), __fmul_rn(o.hv, inv0))
                                         : (lane == SK2 ? (e4m3x2(__fmul_rn(o.cv, inv0), 0.0f) & 0xffu) : 0u);
        const uint32_t word = pair | (__shfl_down_sync(FULL_MASK, pair, 1) << 16);   // even lanes
        const int src = 8 * (lane & 3);
        o.w0 = __shfl_sync(FULL_MASK, word, src);
        o.w1 = __shfl_sync(FULL_MASK, word, src + 2);
        o.w2 = __shfl_sync(FULL_MASK, word, src + 4);
        o.w3 = __shfl_sync(FULL_MASK, word, src + 6);
        return o;
    }
    uint32_t word;
    if (lane < SK2) {
        const __nv_bfloat162 ph2 = __floats2bfloat162_rn(o.pv, o.hv);      // .x price, .y holding
        word = *(const uint32_t *)&ph2;
    } else {
        const __nv_bfloat16 cb = __float2bfloat16_rn(o.cv);
        word = lane == SK2 ? (uint32_t)*(const uint16_t *)&cb : 0u;
    }
    const int src = 4 * (lane & 7);
    o.w0 = __shfl_sync(FULL_MASK, word, src);
    o.w1 = __shfl_sync(FULL_MASK, word, src + 1);
    o.w2 = __shfl_sync(FULL_MASK, word, src + 2);
    o.w3 = __shfl_sync(FULL_MASK, word, src + 3);
    return o;
}

// One 16-byte piece of a published row into CTA m: this CTA's own operand by
// a plain store, another CTA's by an asynchronous store that completes its
// bytes on that CTA's observation barrier.
__device__ __forceinline__ void own_put16(const ObsWords &o, uint32_t at, int m, int rank, uint32_t obs_bar)
{
    using namespace ptx;
    if (m == rank) st_shared_v4(at, o.w0, o.w1, o.w2, o.w3);
    else st_async_v4(map_shared_rank(at, (uint32_t)m), o.w0, o.w1, o.w2, o.w3, map_shared_rank(obs_bar, (uint32_t)m));
}

// Row r's chunks to CTAs lane >> 3 and 4 + (lane >> 3) (BF16: 8 chunks) or
// lane >> 2 (E4M3: 4 chunks), its Z row index to CTA `lane`.
template <bool FP8>
__device__ __forceinline__ void own_store(const ObsWords &o, int r, uint32_t a_obs, uint32_t ctx_addr, int M2,
                                          int lane, int rank, uint32_t obs_bar)
{
    using namespace ptx;
    if (FP8) {
        const uint32_t at = a_obs + (uint32_t)(lane & 3) * 2048u + (uint32_t)(r / 8) * 128u + (uint32_t)(r % 8) * 16u;
        const int m = lane >> 2;
        if (m < M2) own_put16(o, at, m, rank, obs_bar);
    } else {
        const uint32_t at = a_obs + (uint32_t)(lane & 7) * 2048u + (uint32_t)(r / 8) * 128u + (uint32_t)(r % 8) * 16u;
        const int m0 = lane >> 3;
        if (m0 < M2) own_put16(o, at, m0, rank, obs_bar);
        if (m0 + 4 < M2) own_put16(o, at, m0 + 4, rank, obs_bar);
    }
    if (lane < M2) {
        const uint32_t c = ctx_addr + 4u * (uint32_t)r;
        if (lane == rank)
            asm volatile("st.shared.u32 [%0], %1;" ::"r"(c), "r"(o.zrow) : "memory");
        else
            st_async_b32(map_shared_rank(c, (uint32_t)lane), (uint32_t)o.zrow,
                         map_shared_rank(obs_bar, (uint32_t)lane));
    }
}

// Publish the next observations of this warp's owned envs: all rows' words
// first (their shuffles overlap), then all stores, then the optional fp32
// trajectory rows.  trow[i] < 0: no trajectory row.
template <int NOWN, bool NARROW, bool FP8>
__device__ __forceinline__ void own_publish_all(const F2Args &a, const OwnEnv *own, const int *orow, const int *eidx,
                                                uint32_t a_obs, uint32_t ctx_addr, int M2, int lane, int64_t tbase,
                                                int rank, uint64_t *obs_bar, float inv0)
{
    ObsWords o[NOWN];
#pragma unroll
    for (int i = 0; i < NOWN; ++i) o[i] = own_words<NARROW, FP8>(a, own[i], eidx[i] >= 0, lane, inv0);
    const uint32_t ob = ptx::smem_u32(obs_bar);
#pragma unroll
    for (int i = 0; i < NOWN; ++i)
        if (orow[i] < a.tile_rows) own_store<FP8>(o[i], orow[i], a_obs, ctx_addr, M2, lane, rank, ob);
    // this CTA's own rows: one local arrival once the warp's plain stores are done
    __syncwarp();
    if (lane == 0) ptx::mbar_arrive(obs_bar);
    if (a.tr_obs) {
#pragma unroll
        for (int i = 0; i < NOWN; ++i) {
            const int e = eidx[i];
            if (e >= 0)
                own_traj_obs(a, a.tr_obs + (tbase + e) * a.obs_ld, o[i].cv, o[i].pv, o[i].hv,
                             own[i].start + own[i].t, own[i].Ke, lane);
        }
    }
}

// NARROW: the env's prices, orders and a step's sells and buys fit 32 bits
// (EnvView::narrow, proved by env_create): the accounting runs in 32-bit
// arithmetic, with the same results.
template <int NOWN, bool NARROW, bool FP8, int W>
__device__ void f2_env_loop(const F2Args &a_in, uint32_t tmem, uint8_t *smem, const F2Smem L_in, uint64_t *bars,
                            volatile int *abort, int warp, int lane, int rank, int tile)
{
    constexpr int PARTS = W / 4;                   // warps sharing a TMEM lane quarter
    constexpr int ZQ = 128 / W;                    // float4 Z values per lane (the warp's columns / 4)
    using namespace ptx;
    const F2Args a = a_in;
    const F2Smem L = L_in;
    const EnvView v = a.v;
    const F2Plan p = a.plan;
    const float w1 = a.w[1], w2 = a.w[2], w3 = a.w[3];
    const int M = p.M, M2 = 2 * M;
    const int j = rank >> 1, hh = rank & 1;
    const int ew = warp;                           // 0..7
    const int q = warp & 3;                        // TMEM lane quarter
    const int col_half = ew >> 2;                  // 0 .. PARTS - 1: which part of the columns this warp reads
    const int r = q * 32 + lane;                   // epilogue row
    const uint32_t tmem_row = tmem + ((uint32_t)(q * 32) << 16);
    const uint32_t a_base = smem_u32(smem + L.a);
    const uint32_t row_off = (uint32_t)(r / 8) * 128u + (uint32_t)(r % 8) * 16u;
    const uint32_t xbuf = smem_u32(smem + L.xbuf);
    const int RO = f2_owned_rows(M);
    const int TR = a.tile_rows;
    const bool row_live = r < TR;                  // this lane's epilogue row holds an env slot
    const bool quarter_live = q * 32 < TR;         // uniform: the warp's lane quarter holds any
    const uint32_t x_tx = f2_x_tx_bytes(M, rank, TR);
    const uint32_t obs_tx = f2_obs_tx_bytes(M, rank, p.esz, TR);
    const uint32_t h1_tx = f2_h1_tx_bytes(p, TR);
    const uint32_t h1r_partner = map_shared_rank(smem_u32(&bars[B_H1]), (uint32_t)(rank ^ 1));
    const uint32_t ctx_addr = smem_u32(smem + L.ctx);
    const int32_t *ctxv = (const int32_t *)(smem + L.ctx);
    uint64_t *obs_ready = &bars[B_OBS], *acc = &bars[B_ACC], *h1r = &bars[B_H1], *h2r = &bars[B_H2];
    uint64_t *xrdy = &bars[B_X];
    const int tile0 = tile * TR;
    const bool issuer = ew == 0;
    const uint32_t w_base = smem_u32(smem + L.w);
    const uint32_t a_obs = a_base + (uint32_t)(p.H1 / p.ck) * 2048u;
    // FP8: this CTA's dequantisation factors and this agent's 1 / sx[l]
    const float *bsm = (const float *)(smem + L.bias);
    const float *dq1s = bsm + 256, *dq2s = bsm + 384, *dq3s = bsm + 512;
    const float inv0 = FP8 ? bsm[640] : 1.0f, inv1 = FP8 ? bsm[641] : 1.0f, inv2 = FP8 ? bsm[642] : 1.0f;
    if (issuer && lane == 0) {
        // resident weights: this CTA's image, loaded once
        const uint8_t *src = a.img + (size_t)rank * p.cta_bytes;
        mbar_arrive_expect_tx(&bars[B_W], p.cta_bytes);
        for (uint32_t o = 0; o < p.cta_bytes; o += TC_CHUNK_MAX) {
            const uint32_t n = min(TC_CHUNK_MAX, p.cta_bytes - o);
            bulk_g2s(smem + L.w + o, src + o, n, &bars[B_W]);
        }
    }

    // owned envs of this warp: rows r0 = rank + M2 * (ew + 8 * i)
    OwnEnv own[NOWN];
    int orow[NOWN], eidx[NOWN];                    // tile row; env index (-1: no env there)
#pragma unroll
    for (int i = 0; i < NOWN; ++i) {
        orow[i] = rank + M2 * (ew + W * i);
        const int pos = tile0 + orow[i];
        eidx[i] = (orow[i] < TR && pos < a.n_pos) ? (a.perm ? a.perm[pos] : pos) : -1;
        const int e = eidx[i];
        OwnEnv &s = own[i];
        s.cash = 0; s.v0 = 0; s.t = 0; s.start = 0; s.W = 2; s.Ke = 0; s.done = 1; s.slot = 0; s.p = 0; s.h = 0;
        s.bps = 0;
        if (e >= 0) {
            s.cash = v.cash[e];
            s.t = v.t[e];
            s.start = v.start[e];
            s.W = v.W[e];
            s.Ke = v.Ke[e];
            s.done = v.done[e];
            s.slot = a.slot[e];
            if (lane < s.Ke) {
                s.h = v.hold[(int64_t)e * KP + lane];
                s.bps = v.bps[(int64_t)e * KP + lane];
                const int64_t c = __ldg(v.close + (int64_t)(s.start + s.t) * SK2 + lane);
                s.p = NARROW ? (int64_t)perturb32((uint32_t)c, s.bps) : perturb(c, s.bps);
            }
        }
        s.v0 = s.cash + warp_sum(s.p * (int64_t)s.h);
        if (e >= 0 && lane == 0) a.t0_out[e] = s.t;
    }
    // observation of step 0
    own_publish_all<NOWN, NARROW, FP8>(a, own, orow, eidx, a_obs, ctx_addr, M2, lane, 0, rank, obs_ready, inv0);

    const float *zbase = a.Z + (size_t)j * a.n_ctx_per_agent * p.H1;
    // The step loop has no early exit: its trip count is uniform, so the warp
    // is provably converged at every warp-collective operation inside it.  A
    // wait that gives up sets the CTA's abort flag; every later wait then
    // returns at once and the remaining steps run through without their data
    // (all of their addresses are independent of it, or clamped).
    // A packed tile runs only until its longest window is over (uniform
    // across the cluster: one value per tile).
    const int T = a.tile_w ? min(a.T, max(a.tile_w[tile] - 1, 0)) : a.T;
    // this lane's word of each owned row in the layer-3 partial-sum buffer
    // (fixed for the launch)
    uint32_t xoff[NOWN];
#pragma unroll
    for (int i = 0; i < NOWN; ++i) {
        const int ri = min(orow[i] / M2, RO - 1);
        xoff[i] = L.xbuf + (uint32_t)ri * 128u + 16u * (uint32_t)((lane >> 2) ^ (ri & 7)) + 4u * (uint32_t)(lane & 3);
    }
    // uniform per launch: read once, not per step
    const bool explore = a.ex.kind == FR_EXPLORE_GAUSSIAN;
    float *const tr_act = a.tr_act;
    if (issuer) f2_wait(&bars[B_W], 0u, abort, a.err, 1u, false);
    for (int s = 0; s < T; ++s) {
        const uint32_t ph = (uint32_t)s & 1u;
        // The next day's closes do not depend on the actions: their loads
        // start here, a whole step of latency before the owners need them.
        int64_t c1[NOWN];
#pragma unroll
        for (int i = 0; i < NOWN; ++i) {
            const OwnEnv &st = own[i];
            c1[i] = (eidx[i] >= 0 && !st.done && lane < st.Ke)
                        ? __ldg(v.close + (int64_t)(st.start + st.t + 1) * SK2 + lane)
                        : 0;
        }
        // ------------------------------------------- E1: + Z + b1 -> ReLU
        // the observation barrier also publishes each env's Z row: read it
        // and start the row's loads while layer 1 runs on the tensor cores
        f2_wait(obs_ready, ph, abort, a.err, 16u, true);
        // arm the next phase: the owner warps' local arrivals follow, the
        // bytes of the other CTAs' rows are expected
        if (issuer && lane == 0 && !*abort) mbar_arrive_expect_tx(obs_ready, obs_tx);
        if (issuer && lane == 0) f2_layer<FP8>(p.l1.K, p.l1.N, p.l1.off, tmem, a_obs, w_base, acc);
        const int nc1 = p.n1 / PARTS;                      // columns per warp (<= 64 / 32)
        const int c01 = col_half * nc1;
        // all of this warp's Z loads in flight at once, one L2 latency
        // clamped: after an aborted wait the row index may be stale
        const int zr = min(max(ctxv[r], 0), a.n_ctx_per_agent - 1);
        const float4 *zrow = (const float4 *)(zbase + (size_t)zr * p.H1 + hh * p.n1 + c01);
        float4 zq[ZQ];
#pragma unroll
        for (int i = 0; i < ZQ; ++i)
            zq[i] = (4 * i < nc1 && row_live) ? __ldg(zrow + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        // The next step's row is the next day's (ctx + 1) for every env that
        // keeps stepping: start pulling it into L1 now, a whole step ahead of
        // its loads (a hint only: a reset env reads its own row, a miss costs
        // what a load costs without it).  One 128-byte line per 32 floats.
        if (row_live && zr + 1 < a.n_ctx_per_agent) {
            const float *znext = zbase + (size_t)(zr + 1) * p.H1 + hh * p.n1 + c01;
#pragma unroll
            for (int i = 0; i < ZQ; i += 8)
                if (4 * i < nc1) asm volatile("prefetch.global.L1 [%0];" ::"l"(znext + 4 * i));
        }
        f2_wait(acc, (uint32_t)(3 * s) & 1u, abort, a.err, 16u, false);
        tc_fence_after();
        if (quarter_live) {                             // uniform; rows beyond the tile are not sent
            const int nc = nc1;
            const int c0 = c01;
            const uint32_t dst_chunk0 = (uint32_t)((hh * p.n1 + c0) / 8);
#pragma unroll
            for (int q4 = 0; q4 < ZQ / 4; ++q4) {
                const int cc = 16 * q4;
                if (cc >= nc) continue;
                uint32_t vv[16];
                __syncwarp();
                tmem_ld16(tmem_row + (uint32_t)(c0 + cc), vv);
                tmem_ld_wait();
                float x[16];
                if constexpr (FP8) {
                    // dequantise the state part, add the table row (indicators + b1)
                    const float *dq = dq1s + c0 + cc;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 z = zq[4 * q4 + i];
                        x[4 * i + 0] = fmaxf(__fmaf_rn(__uint_as_float(vv[4 * i + 0]), dq[4 * i + 0], z.x), 0.0f);
                        x[4 * i + 1] = fmaxf(__fmaf_rn(__uint_as_float(vv[4 * i + 1]), dq[4 * i + 1], z.y), 0.0f);
                        x[4 * i + 2] = fmaxf(__fmaf_rn(__uint_as_float(vv[4 * i + 2]), dq[4 * i + 2], z.z), 0.0f);
                        x[4 * i + 3] = fmaxf(__fmaf_rn(__uint_as_float(vv[4 * i + 3]), dq[4 * i + 3], z.w), 0.0f);
                    }
                    uint32_t w[4];
                    e4m3_pack16(x, inv1, w);
                    const uint32_t at = a_base + (uint32_t)((hh * p.n1 + c0 + cc) / 16) * 2048u + row_off;
                    if (row_live) {
                        st_shared_v4(at, w[0], w[1], w[2], w[3]);
                        st_async_v4(map_shared_rank(at, (uint32_t)(rank ^ 1)), w[0], w[1], w[2], w[3], h1r_partner);
                    }
                } else {
                    // + Z, then ReLU inside the BF16 conversion
                    uint32_t w0[4], w1[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 z = zq[4 * q4 + i];
                        const uint32_t lo = relu_bf16x2(__uint_as_float(vv[4 * i + 0]) + z.x,
                                                        __uint_as_float(vv[4 * i + 1]) + z.y);
                        const uint32_t hi = relu_bf16x2(__uint_as_float(vv[4 * i + 2]) + z.z,
                                                        __uint_as_float(vv[4 * i + 3]) + z.w);
                        if (i < 2) {
                            w0[2 * i] = lo;
                            w0[2 * i + 1] = hi;
                        } else {
                            w1[2 * i - 4] = lo;
                            w1[2 * i - 3] = hi;
                        }
                    }
                    const uint32_t at = a_base + (dst_chunk0 + (uint32_t)(cc / 8)) * 2048u + row_off;
                    if (row_live) {
                        st_shared_v4(at, w0[0], w0[1], w0[2], w0[3]);
                        st_shared_v4(at + 2048u, w1[0], w1[1], w1[2], w1[3]);
                        // the partner's copy: asynchronous stores that complete
                        // their bytes on the partner's h1 barrier
                        const uint32_t pt = map_shared_rank(at, (uint32_t)(rank ^ 1));
                        st_async_v4(pt, w0[0], w0[1], w0[2], w0[3], h1r_partner);
                        st_async_v4(pt + 2048u, w1[0], w1[1], w1[2], w1[3], h1r_partner);
                    }
                }
            }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(h1r);
        if (issuer) {
            f2_wait(h1r, ph, abort, a.err, 4u, true);
            if (lane == 0 && !*abort) mbar_arrive_expect_tx(h1r, h1_tx);     // arm the next phase
            if (lane == 0) f2_layer<FP8>(p.l2.K, p.l2.N, p.l2.off, tmem, a_base, w_base, acc);
            __syncwarp();
        }
        // ------------------------------------------------- E2: + b2 -> ReLU
        f2_wait(acc, (uint32_t)(3 * s + 1) & 1u, abort, a.err, 16u, false);
        tc_fence_after();
        {
            const float *b2 = (const float *)(smem + L.bias);
            const int nc = quarter_live ? p.n2 / PARTS : 0;     // uniform
            const int c0 = col_half * (p.n2 / PARTS);
            for (int cc = 0; cc < nc; cc += 16) {
                uint32_t vv[16];
                __syncwarp();
                tmem_ld16(tmem_row + (uint32_t)(c0 + cc), vv);
                tmem_ld_wait();
                float x[16];
                if constexpr (FP8) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        x[i] = fmaxf(__fmaf_rn(__uint_as_float(vv[i]), dq2s[c0 + cc + i], b2[c0 + cc + i]), 0.0f);
                    uint32_t w[4];
                    e4m3_pack16(x, inv2, w);
                    st_shared_v4(a_base + (uint32_t)((c0 + cc) / 16) * 2048u + row_off, w[0], w[1], w[2], w[3]);
                } else {
                    // + b2 (four per shared load), then ReLU inside the BF16
                    // conversion
                    const float4 *b4 = (const float4 *)(b2 + c0 + cc);
                    uint32_t w0[4], w1[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 bb = b4[i];
                        const uint32_t lo = relu_bf16x2(__uint_as_float(vv[4 * i + 0]) + bb.x,
                                                        __uint_as_float(vv[4 * i + 1]) + bb.y);
                        const uint32_t hi = relu_bf16x2(__uint_as_float(vv[4 * i + 2]) + bb.z,
                                                        __uint_as_float(vv[4 * i + 3]) + bb.w);
                        if (i < 2) {
                            w0[2 * i] = lo;
                            w0[2 * i + 1] = hi;
                        } else {
                            w1[2 * i - 4] = lo;
                            w1[2 * i - 3] = hi;
                        }
                    }
                    const uint32_t at = a_base + (uint32_t)((c0 + cc) / 8) * 2048u + row_off;
                    st_shared_v4(at, w0[0], w0[1], w0[2], w0[3]);
                    st_shared_v4(at + 2048u, w1[0], w1[1], w1[2], w1[3]);
                }
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(h2r);
        if (issuer) {
            f2_wait(h2r, ph, abort, a.err, 8u, false);
            if (lane == 0) f2_layer<FP8>(p.l3.K, p.l3.N, p.l3.off, tmem + 128u, a_base, w_base, acc);
            __syncwarp();
        }
        // --------------------------------- E3: partial sums to the owners
        f2_wait(acc, (uint32_t)(3 * s + 2) & 1u, abort, a.err, 16u, false);
        tc_fence_after();
        if (quarter_live) {
            // every warp of the lane quarter reads its part of the 32 columns
            // (EC = 32 / PARTS of them, EC / 4 16-byte groups)
            constexpr int EC = 32 / PARTS;
            uint32_t vv[EC];
            __syncwarp();
            if constexpr (EC == 8)
                tmem_ld8(tmem_row + 128u + (uint32_t)(EC * col_half), vv);
            else
                tmem_ld16(tmem_row + 128u + (uint32_t)(EC * col_half), vv);
            tmem_ld_wait();
            // row r's partial sums to block `rank` of its owner's buffer, at
            // owned row r / 2M; column group k stored at group k ^ (row & 7),
            // so that the owner's per-lane reads of one row are conflict-free.
            // Another CTA's rows go by asynchronous stores that complete bytes
            // on the owner's barrier (no fence here); this CTA's own rows by
            // plain stores and one local arrival per warp.
            const uint32_t ri = (uint32_t)(r / M2);
            const uint32_t owner = (uint32_t)(r % M2);
            const uint32_t at = xbuf + ((uint32_t)rank * (uint32_t)RO + ri) * 128u;
            const uint32_t k0 = (uint32_t)(EC / 4 * col_half);
            if (!row_live) {
                // a padding row: nothing to send
            } else if (owner == (uint32_t)rank) {
#pragma unroll
                for (int k = 0; k < EC / 4; ++k)
                    st_shared_v4(at + 16u * ((k0 + (uint32_t)k) ^ (ri & 7u)), vv[4 * k], vv[4 * k + 1],
                                 vv[4 * k + 2], vv[4 * k + 3]);
            } else {
                const uint32_t dst = map_shared_rank(at, owner);
                const uint32_t rbar = map_shared_rank(smem_u32(xrdy), owner);
#pragma unroll
                for (int k = 0; k < EC / 4; ++k)
                    st_async_v4(dst + 16u * ((k0 + (uint32_t)k) ^ (ri & 7u)), vv[4 * k], vv[4 * k + 1],
                                vv[4 * k + 2], vv[4 * k + 3], rbar);
            }
        }
        __syncwarp();                               // every warp arrives, sending or not
        if (lane == 0) mbar_arrive(xrdy);
        tc_fence_before();
        // --------------------------------------------- owners: trade, publish
        // The owned envs are processed in lockstep, so that their reductions
        // overlap instead of forming one long dependent chain per env.
        int64_t p1[NOWN];
        bool run[NOWN];                                 // uniform: env exists and is not done
#pragma unroll
        for (int i = 0; i < NOWN; ++i) {
            const OwnEnv &st = own[i];
            run[i] = eidx[i] >= 0 && !st.done;
            const bool ok = run[i] && lane < st.Ke;
            p1[i] = ok ? (NARROW ? (int64_t)perturb32((uint32_t)c1[i], st.bps) : perturb(c1[i], st.bps)) : 0;
        }
        f2_wait(xrdy, ph, abort, a.err, 64u, true);
        // arm the next phase: one arrival, the bytes the other CTAs send
        if (ew == 0 && lane == 0 && !*abort) mbar_arrive_expect_tx(xrdy, x_tx);
        const int fee = v.fee_bps;
        int64_t nsell[NOWN], want[NOWN], full[NOWN], ssum[NOWN], bsum[NOWN], vsum[NOWN], wsum[NOWN];
        // The owned envs' actions first, all envs together, then (only when
        // asked for) exploration and the recorded actions, then the trades'
        // reductions: no out-of-line call sits between the envs' chains.
        float actv[NOWN];
#pragma unroll
        for (int i = 0; i < NOWN; ++i) {
            // agent jj's action for this lane's asset: tanh(partial of half 0
            // + partial of half 1 + b3), rounded to fp16
            const uint8_t *xr = smem + xoff[i];
            const float *b3s = (const float *)(smem + L.bias) + 128;
            auto agent_act = [&](int jj) {
                const float p0 = *(const float *)(xr + (size_t)(2 * jj) * RO * 128);
                const float p1 = *(const float *)(xr + (size_t)(2 * jj + 1) * RO * 128);
                // FP8: the two halves' sums of codes dequantised together (one
                // output channel, one factor)
                const float pre = FP8 ? __fmaf_rn(__fadd_rn(p0, p1), dq3s[32 * jj + lane], b3s[32 * jj + lane])
                                      : __fadd_rn(__fadd_rn(p0, p1), b3s[32 * jj + lane]);
                const float y = lane < SK2 ? tanh_approx(pre) : 0.0f;
                return __half2float(__float2half_rn(y));
            };
            // combine (anchored weighted mean) for this lane's asset
            const float a0 = agent_act(0);
            float act = a0;
#pragma unroll
            for (int jj = 1; jj < 4; ++jj) {
                if (jj < M) {
                    const float aj = agent_act(jj);
                    const float wj = jj == 1 ? w1 : (jj == 2 ? w2 : w3);
                    act = __fadd_rn(act, __fmul_rn(wj, __fsub_rn(aj, a0)));
                }
            }
            actv[i] = act;
        }
        if (explore || tr_act) {
#pragma unroll
            for (int i = 0; i < NOWN; ++i) {
                const int e = eidx[i];
                if (explore && e >= 0 && lane < SK2)
                    actv[i] = f2_explore(a.ex, actv[i], (uint32_t)e, a.ex.g0 + (uint32_t)s, (uint32_t)lane);
                if (tr_act && e >= 0 && lane < SK2) tr_act[((int64_t)s * v.N + e) * SK2 + lane] = actv[i];
            }
        }
#pragma unroll
        for (int i = 0; i < NOWN; ++i) {
            const OwnEnv &st = own[i];
            const float act = actv[i];
            const bool live = run[i] && lane < st.Ke;
            float ac = isfinite(act) ? act : 0.0f;
            ac = fminf(fmaxf(ac, -1.0f), 1.0f);
            const int32_t qa = live ? (int32_t)__fmul_rz(ac, (float)v.hmax) : 0;
            const int64_t hcur = st.h;
            // sells capped at the holding; buys as ordered (the common case:
            // every order fits); the value after both at the next prices
            nsell[i] = qa < 0 ? min((int64_t)(-qa), hcur) : 0;
            want[i] = qa > 0 ? (int64_t)qa : 0;
            if (NARROW) {
                // orders of at most hmax shares: notionals, fees and a step's
                // sums below 2^32; holdings int32 (one 32 x 32 -> 64 product)
                const uint32_t p32 = (uint32_t)st.p, gs = (uint32_t)nsell[i] * p32;
                const uint32_t f32 = cost_of32((uint32_t)want[i], p32, fee);
                full[i] = (int64_t)f32;
                ssum[i] = (int64_t)__reduce_add_sync(FULL_MASK, gs - fee_of32(gs, fee));
                bsum[i] = (int64_t)__reduce_add_sync(FULL_MASK, f32);
                vsum[i] = warp_sum_redux(
                    (int64_t)((uint64_t)(uint32_t)p1[i] * (uint32_t)(hcur - nsell[i] + want[i])));
                // the wanted shares at the next prices (each below an order's
                // notional bound, their sum below 2^32)
                wsum[i] = (int64_t)__reduce_add_sync(FULL_MASK, (uint32_t)p1[i] * (uint32_t)want[i]);
            } else {
                wsum[i] = 0;
                const int64_t gs = nsell[i] * st.p;
                full[i] = cost_of(want[i], st.p, fee);
                ssum[i] = warp_sum_redux(gs - fee_of(gs, fee));
                bsum[i] = warp_sum_redux(full[i]);
                vsum[i] = warp_sum_redux(p1[i] * (hcur - nsell[i] + want[i]));
            }
        }
        // trades: every env's common case (all buys fit) first, then the
        // greedy partial fills of the envs whose buys do not all fit, then
        // the state updates
        int64_t cashv[NOWN], nbv[NOWN], v1v[NOWN];
        bool greedy[NOWN];
#pragma unroll
        for (int i = 0; i < NOWN; ++i) {
            const int64_t cash1 = own[i].cash + ssum[i];
            cashv[i] = cash1 - bsum[i];
            nbv[i] = want[i];
            v1v[i] = cashv[i] + vsum[i];
            greedy[i] = run[i] && bsum[i] > cash1;
        }
#pragma unroll
        for (int i = 0; i < NOWN; ++i) {
            if (!greedy[i]) continue;                  // uniform
            const OwnEnv &st = own[i];
            const int64_t cash1 = st.cash + ssum[i];
            if (NARROW) {
                // the value without the wanted buys, plus what was filled
                const bool can = want[i] > 0 && (int64_t)cost_of32(1u, (uint32_t)st.p, fee) <= cash1;
                if (!__any_sync(FULL_MASK, can)) {     // no order affords one share
                    cashv[i] = cash1;
                    nbv[i] = 0;
                    v1v[i] = cash1 + vsum[i] - wsum[i];
                } else {
                    const Fill fl = own_buy_greedy<true>(cash1, want[i], full[i], st.p, fee, lane);
                    cashv[i] = fl.cash;
                    nbv[i] = fl.nb;
                    v1v[i] = fl.cash + vsum[i] - wsum[i] +
                             (int64_t)__reduce_add_sync(FULL_MASK, (uint32_t)p1[i] * (uint32_t)fl.nb);
                }
            } else {
                const Fill fl = own_buy_greedy<false>(cash1, want[i], full[i], st.p, fee, lane);
                cashv[i] = fl.cash;
                nbv[i] = fl.nb;
                v1v[i] = fl.cash + warp_sum_redux(p1[i] * (st.h - nsell[i] + fl.nb));
            }
        }
#pragma unroll
        for (int i = 0; i < NOWN; ++i) {
            const int e = eidx[i];
            const bool valid = e >= 0;
            OwnEnv &st = own[i];
            const int64_t row = (int64_t)s * v.N + e;
            int64_t rew = 0, vlog = VLOG_NONE2;
            bool dn_out = true;
            if (run[i]) {
                const int64_t v1 = v1v[i];
                rew = v1 - st.v0;
                st.t += 1;
                st.done = st.t == st.W - 1;
                dn_out = st.done;
                vlog = st.done ? -v1 - 1 : v1;
                st.cash = cashv[i];
                st.h = (int32_t)(st.h - nsell[i] + nbv[i]);
                st.p = p1[i];
                st.v0 = v1;
                if (st.done && v.auto_reset) {
                    st.cash = v.init_cash;
                    st.v0 = v.init_cash;
                    st.t = 0;
                    st.done = 0;
                    st.h = 0;
                    const int64_t c0 = lane < st.Ke ? __ldg(v.close + (int64_t)st.start * SK2 + lane) : 1;
                    st.p = lane < st.Ke ? (NARROW ? (int64_t)perturb32((uint32_t)c0, st.bps) : perturb(c0, st.bps)) : 0;
                }
            }
            if (valid && lane == 0) {
                if (a.tr_rew) a.tr_rew[row] = rew;
                if (a.tr_rew_f32) a.tr_rew_f32[row] = reward_f32(rew);
                if (a.tr_done) a.tr_done[row] = dn_out ? 1 : 0;
                a.vlog[row] = vlog;
            }
        }
        if (s + 1 < T)
            own_publish_all<NOWN, NARROW, FP8>(a, own, orow, eidx, a_obs, ctx_addr, M2, lane,
                                               (int64_t)(s + 1) * v.N, rank, obs_ready, inv0);
    }
    // the other CTAs' asynchronous stores of the last step have landed
    // before this CTA can exit, also when a wait gave up and the loop ran on
    // without its data (bounded; a no-op when the last phase completed)
    if (T > 0 && ew == 0 && lane == 0) {
        volatile int no_abort = 0;
        mbar_wait_cluster(obs_ready, (uint32_t)(T - 1) & 1u, &no_abort, a.err, 32u, TC_WAIT_NS);
        mbar_wait_cluster(h1r, (uint32_t)(T - 1) & 1u, &no_abort, a.err, 32u, TC_WAIT_NS);
        mbar_wait_cluster(xrdy, (uint32_t)(T - 1) & 1u, &no_abort, a.err, 32u, TC_WAIT_NS);
    }
    // every MMA this CTA issued has completed before TMEM is released, also
    // when a wait gave up and the loop ran on without its data
    if (issuer && lane == 0) {
        mma_commit(&bars[B_END]);
        volatile int no_abort = 0;
        mbar_wait(&bars[B_END], 0u, &no_abort, a.err, 256u, TC_WAIT_NS);
    }
    __syncwarp();
    // state back to global memory (steps and accumulators: metrics replay);
    // the steps a packed tile did not run are no-steps in the value log
#pragma unroll
    for (int i = 0; i < NOWN; ++i) {
        const int e = eidx[i];
        if (e < 0) continue;
        for (int s = T + lane; s < a.T; s += 32) a.vlog[(int64_t)s * v.N + e] = VLOG_NONE2;
        if (lane == 0) {
            v.cash[e] = own[i].cash;
            v.done[e] = own[i].done ? 1 : 0;
            v.t[e] = own[i].t;
        }
        if (lane < SK2) v.hold[(int64_t)e * KP + lane] = lane < own[i].Ke ? own[i].h : 0;
    }
}

template <bool NARROW, bool FP8, int W>
__global__ void __launch_bounds__(32 * W, 1) k_rollout_stock2(const __grid_constant__ F2Args a)
{
    using namespace ptx;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const F2Plan &p = a.plan;
    const F2Smem L = f2_smem(p);
    uint64_t *bars = (uint64_t *)(smem + L.bars);
    uint32_t *tmem_slot = (uint32_t *)(bars + B_COUNT);
    volatile int *abort = (volatile int *)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rank = (int)cluster_ctarank();
    const int tile = blockIdx.y;

    if (threadIdx.x == 0) {
        mbar_init(&bars[B_W], 1);
        // this CTA's owner warps (its own rows) plus one arming arrival per
        // phase that expects the other CTAs' rows; phase 0 armed here
        mbar_init(&bars[B_OBS], (uint32_t)W + 1u);
        mbar_arrive_expect_tx(&bars[B_OBS], f2_obs_tx_bytes(p.M, rank, p.esz, a.tile_rows));
        mbar_init(&bars[B_ACC], 1);
        // this CTA's E1 warps plus one arming arrival per phase that expects
        // the partner's half; phase 0 armed here
        mbar_init(&bars[B_H1], (uint32_t)W + 1u);
        mbar_arrive_expect_tx(&bars[B_H1], f2_h1_tx_bytes(p, a.tile_rows));
        mbar_init(&bars[B_H2], (uint32_t)W);                       // this CTA's E2 warps
        // this CTA's W E3 warps, plus one arming arrival per phase that
        // expects the other CTAs' bytes; phase 0 armed here
        mbar_init(&bars[B_X], (uint32_t)W + 1u);
        mbar_arrive_expect_tx(&bars[B_X], f2_x_tx_bytes(p.M, rank, a.tile_rows));
        mbar_init(&bars[B_END], 1);                                // the issuer's last commit
        *abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        __syncwarp();
        tmem_alloc(tmem_slot, 256u);
        tmem_relinquish();
    }
    if (warp == 2) {
        // this CTA's b2 half (epilogue 2) and every agent's b3 (owners)
        float *bs = (float *)(smem + L.bias);
        const int jj = rank >> 1, h2 = rank & 1;
        for (int i = lane; i < 128; i += 32) bs[i] = i < p.n2 ? a.b2[(size_t)jj * p.H2 + h2 * p.n2 + i] : 0.0f;
        for (int i = lane; i < 4 * 32; i += 32) bs[128 + i] = i < p.M * 32 ? a.b3[i] : 0.0f;
        if (FP8) {
            for (int i = lane; i < 128; i += 32) {
                bs[256 + i] = i < p.n1 ? a.dq[((size_t)jj * 3 + 0) * 256 + h2 * p.n1 + i] : 0.0f;
                bs[384 + i] = i < p.n2 ? a.dq[((size_t)jj * 3 + 1) * 256 + h2 * p.n2 + i] : 0.0f;
                bs[512 + i] = i < p.M * 32 ? a.dq[((size_t)(i / 32) * 3 + 2) * 256 + (i % 32)] : 0.0f;
            }
            if (lane < 3) bs[640 + lane] = a.inv_sx[(size_t)jj * 4 + lane];
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    cluster_sync_all();
    const uint32_t tmem = *tmem_slot;

    {
        // owned envs per env warp: ceil(ceil(tile_rows / 2M) / 8), at least 2
        // (at 128 rows: 4, 3, 2 for M = 2..4)
        const int per_warp = (f2_rows_of(a.tile_rows, p.M, 0) + W - 1) / W;
        if (W == 16) {
            // 16 warps: at most ceil(ceil(128 / 4) / 16) = 2 envs per warp
            if (per_warp <= 1) f2_env_loop<1, NARROW, FP8, W>(a, tmem, smem, L, bars, abort, warp, lane, rank, tile);
            else f2_env_loop<2, NARROW, FP8, W>(a, tmem, smem, L, bars, abort, warp, lane, rank, tile);
        } else {
            switch (per_warp) {
            case 4: f2_env_loop<4, NARROW, FP8, W>(a, tmem, smem, L, bars, abort, warp, lane, rank, tile); break;
            case 3: f2_env_loop<3, NARROW, FP8, W>(a, tmem, smem, L, bars, abort, warp, lane, rank, tile); break;
            default: f2_env_loop<2, NARROW, FP8, W>(a, tmem, smem, L, bars, abort, warp, lane, rank, tile); break;
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, 256u);
    }
    __syncwarp();
    cluster_sync_all();
}

// The indicator table: Z[j][ctx][n] = sum_c W1_j[n][c] x[ctx][c] + b1_j[n]
// over the 240 indicator entries c, with x[ctx][i*30 + k] = ind[day][i][k]
// for assets k < the slot's count, else 0 (ctx = slot * days + day).  A block
// takes ZT_ROWS contexts x ZT_COLS outputs of one agent.  The contexts' rows
// and the tile's weight columns (read [c][n]) are copied into shared memory
// by asynchronous 16-byte copies issued all at once, so the block waits for
// memory once rather than once per indicator entry; each thread then sums
// ZT_ROWS / 8 contexts x 2 outputs, in c order in fp32.  40 contexts per
// block: 1,000 contexts x 256 outputs x 3 agents make 300 blocks, one wave
// at two blocks (100 KB of shared memory each) per SM.
constexpr int ZT_ROWS = 40, ZT_COLS = 64, ZT_RPT = ZT_ROWS / 8;
static_assert(ZT_ROWS % 8 == 0 && ZT_ROWS <= 256, "8 warps of ZT_RPT rows; one thread per row's slot");
constexpr uint32_t ZT_SMEM = (uint32_t)(ZT_ROWS * NIND + NIND * ZT_COLS + ZT_ROWS) * 4u;

__global__ void __launch_bounds__(256) k_ztable(const float *__restrict__ ind, int n_days,
                                                 const int32_t *__restrict__ slot_ke, int n_ctx,
                                                 const float *__restrict__ wind, int H1, float *__restrict__ Z)
{
    extern __shared__ __align__(16) float zsm[];
    float *xs = zsm;                               // [ZT_ROWS][NIND]
    float *ws = zsm + ZT_ROWS * NIND;              // [NIND][ZT_COLS]
    int *kes = (int *)(ws + NIND * ZT_COLS);       // [ZT_ROWS] assets of each row's slot
    const int j = blockIdx.z, n0 = blockIdx.y * ZT_COLS, ctx0 = blockIdx.x * ZT_ROWS;
    const int tid = threadIdx.x;
    // H1 is a multiple of 64 and the buffers are 256-byte aligned, so every
    // copy below starts on a 16-byte boundary
    const float *w = wind + (size_t)j * ((size_t)H1 * NIND + H1);
    for (int i = tid; i < NIND * (ZT_COLS / 4); i += blockDim.x) {
        const int c = i / (ZT_COLS / 4), q = i % (ZT_COLS / 4);
        ptx::cp_async16(ptx::smem_u32(ws + c * ZT_COLS + q * 4), w + (size_t)c * H1 + n0 + q * 4);
    }
    for (int i = tid; i < ZT_ROWS * (NIND / 4); i += blockDim.x) {
        const int r = i / (NIND / 4), q = i % (NIND / 4), ctx = ctx0 + r;
        float *dst = xs + r * NIND + q * 4;
        if (ctx < n_ctx)
            ptx::cp_async16(ptx::smem_u32(dst), ind + (size_t)(ctx % n_days) * NIND + q * 4);
        else
            *(float4 *)dst = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    ptx::cp_async_commit();
    if (tid < ZT_ROWS) kes[tid] = ctx0 + tid < n_ctx ? slot_ke[(ctx0 + tid) / n_days] : SK2;
    ptx::cp_async_wait<0>();
    __syncthreads();
    // zero the assets a row's slot does not hold
    for (int i = tid; i < ZT_ROWS * NIND; i += blockDim.x) {
        const int r = i / NIND, c = i % NIND;
        if (c % SK2 >= kes[r]) xs[i] = 0.0f;
    }
    __syncthreads();
    const int tn = tid & 31, tr = tid >> 5;        // outputs n0 + 2 tn + {0, 1}, rows ZT_RPT tr + {0 ..}
    const float *xr = xs + tr * ZT_RPT * NIND;
    float a0[ZT_RPT], a1[ZT_RPT];
#pragma unroll
    for (int r = 0; r < ZT_RPT; ++r) a0[r] = a1[r] = 0.0f;
#pragma unroll 2
    for (int c = 0; c < NIND; c += 4) {
        float2 wv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) wv[k] = *(const float2 *)(ws + (c + k) * ZT_COLS + 2 * tn);
#pragma unroll
        for (int r = 0; r < ZT_RPT; ++r) {
            const float4 x = *(const float4 *)(xr + r * NIND + c);
            a0[r] = fmaf(x.x, wv[0].x, a0[r]);
            a1[r] = fmaf(x.x, wv[0].y, a1[r]);
            a0[r] = fmaf(x.y, wv[1].x, a0[r]);
            a1[r] = fmaf(x.y, wv[1].y, a1[r]);
            a0[r] = fmaf(x.z, wv[2].x, a0[r]);
            a1[r] = fmaf(x.z, wv[2].y, a1[r]);
            a0[r] = fmaf(x.w, wv[3].x, a0[r]);
            a1[r] = fmaf(x.w, wv[3].y, a1[r]);
        }
    }
    const float2 b = __ldg((const float2 *)(w + (size_t)H1 * NIND + n0 + 2 * tn));
    float *zj = Z + (size_t)j * n_ctx * H1;
#pragma unroll
    for (int r = 0; r < ZT_RPT; ++r) {
        const int ctx = ctx0 + tr * ZT_RPT + r;
        if (ctx < n_ctx) *(float2 *)(zj + (size_t)ctx * H1 + n0 + 2 * tn) = make_float2(a0[r] + b.x, a1[r] + b.y);
    }
}

inline uint16_t bf16_rne(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (uint16_t)(u >> 16);
}

inline uint32_t coff(int N, int n, int kk)
{
    return (uint32_t)((kk / 8) * (N * 16) + (n / 8) * 128 + (n % 8) * 16 + (kk % 8) * 2);
}

}  // namespace

// ------------------------------------------------------------------ host
struct F2Cache {
    F2Image im;
};

static void f2_free(fr_ctx *ctx, F2Image &im)
{
    dev_free(ctx, im.img, (uint64_t)im.plan.M * 2 * im.plan.cta_bytes);
    dev_free(ctx, im.b2, (uint64_t)im.plan.M * im.plan.H2 * 4);
    dev_free(ctx, im.b3, (uint64_t)im.plan.M * 32 * 4);
    dev_free(ctx, im.wind, (uint64_t)im.plan.M * (im.plan.H1 * NIND + im.plan.H1) * 4);
    dev_free(ctx, im.dq, (uint64_t)im.plan.M * 3 * 256 * 4);
    dev_free(ctx, im.inv_sx, (uint64_t)im.plan.M * 4 * 4);
    im.img = nullptr;
    im.dq = im.inv_sx = nullptr;
}

// Build the per-CTA resident images of an ensemble (host packing, once;
// FP8 again whenever the activation scales change).  FP8 weights are the
// actor kernel's: codes of W[n][k] * (1 / sw[n]) with its per-row scales
// sw[n] (the whole row's, indicator columns included, which enter through
// the fp32 table unquantised), dequantised by sx[l] * sw[n].
static int f2_build(const fr_ensemble *e, F2Image &im)
{
    F2Plan &p = im.plan;
    const TcImage *t = e->tc;
    std::vector<float> host((size_t)e->M * e->P);
    FR_CUDA(cudaMemcpy(host.data(), e->params, host.size() * 4, cudaMemcpyDeviceToHost));
    std::vector<uint8_t> img((size_t)p.M * 2 * p.cta_bytes, 0);
    std::vector<float> b2((size_t)p.M * p.H2), b3((size_t)p.M * 32, 0.0f);
    std::vector<float> wind((size_t)p.M * (p.H1 * NIND + p.H1));
    std::vector<float> dq(p.fp8 ? (size_t)p.M * 3 * 256 : 0, 0.0f), inv_sx(p.fp8 ? (size_t)p.M * 4 : 0, 1.0f);
    int cur_j = 0, cur_l = 0;            // agent and layer being packed (FP8 row scales)
    auto put = [&](uint8_t *base, const F2Layer &l, int n, int k, float w) {
        const int c = k / l.KC, kk = k % l.KC;
        if (p.fp8) {
            // n: row within this CTA's half; the global row is resolved by the caller
            const uint8_t q = (uint8_t)__nv_cvt_float_to_fp8(w, __NV_SATFINITE, __NV_E4M3);
            base[l.off + (size_t)c * l.N * l.KC + (size_t)(kk / 16) * (l.N * 16) + (size_t)(n / 8) * 128 +
                 (size_t)(n % 8) * 16 + (size_t)(kk % 16)] = q;
            return;
        }
        const uint16_t b = bf16_rne(w);
        memcpy(base + l.off + (size_t)c * l.N * l.KC * 2 + coff(l.N, n, kk), &b, 2);
    };
    // FP8 operand of global row n of layer l: w * (1 / sw[n])
    auto wq = [&](int n, float w) { return p.fp8 ? w * (1.0f / t->sw[cur_j][cur_l][n]) : w; };
    for (int j = 0; j < p.M; ++j) {
        const float *P = host.data() + (size_t)j * e->P;
        const float *W1 = P + e->w_off[0], *B1 = P + e->b_off[0];
        const float *W2 = P + e->w_off[1], *B2 = P + e->b_off[1];
        const float *W3 = P + e->w_off[2], *B3 = P + e->b_off[2];
        cur_j = j;
        for (int hh = 0; hh < 2; ++hh) {
            uint8_t *base = img.data() + (size_t)(2 * j + hh) * p.cta_bytes;
            cur_l = 0;
            for (int n = 0; n < p.n1; ++n)
                for (int k = 0; k < NSTATE; ++k)
                    put(base, p.l1, n, f2_state_pos(k), wq(hh * p.n1 + n, W1[(size_t)(hh * p.n1 + n) * SD2 + k]));
            cur_l = 1;
            for (int n = 0; n < p.n2; ++n)
                for (int k = 0; k < p.H1; ++k)
                    put(base, p.l2, n, k, wq(hh * p.n2 + n, W2[(size_t)(hh * p.n2 + n) * p.H1 + k]));
            cur_l = 2;
            for (int n = 0; n < SK2; ++n)
                for (int k = 0; k < p.n2; ++k) put(base, p.l3, n, k, wq(n, W3[(size_t)n * p.H2 + hh * p.n2 + k]));
        }
        if (p.fp8) {
            const int width[3] = {p.H1, p.H2, SK2};
            for (int l = 0; l < 3; ++l) {
                for (int n = 0; n < width[l]; ++n) dq[((size_t)j * 3 + l) * 256 + n] = t->sx[j][l] * t->sw[j][l][n];
                inv_sx[(size_t)j * 4 + l] = 1.0f / t->sx[j][l];
            }
        }
        for (int n = 0; n < p.H2; ++n) b2[(size_t)j * p.H2 + n] = B2[n];
        for (int n = 0; n < SK2; ++n) b3[(size_t)j * 32 + n] = B3[n];
        float *wi = wind.data() + (size_t)j * (p.H1 * NIND + p.H1);
        for (int n = 0; n < p.H1; ++n) {
            for (int c = 0; c < NIND; ++c) wi[(size_t)c * p.H1 + n] = W1[(size_t)n * SD2 + NSTATE + c];
            wi[(size_t)p.H1 * NIND + n] = B1[n];
        }
    }
    int rc;
    if ((rc = dev_alloc(e->ctx, (void **)&im.img, img.size())) ||
        (rc = dev_alloc(e->ctx, (void **)&im.b2, b2.size() * 4)) ||
        (rc = dev_alloc(e->ctx, (void **)&im.b3, b3.size() * 4)) ||
        (rc = dev_alloc(e->ctx, (void **)&im.wind, wind.size() * 4)) ||
        (p.fp8 && (rc = dev_alloc(e->ctx, (void **)&im.dq, dq.size() * 4))) ||
        (p.fp8 && (rc = dev_alloc(e->ctx, (void **)&im.inv_sx, inv_sx.size() * 4)))) {
        f2_free(e->ctx, im);
        return rc;
    }
    if (p.fp8) {
        FR_CUDA(cudaMemcpy(im.dq, dq.data(), dq.size() * 4, cudaMemcpyHostToDevice));
        FR_CUDA(cudaMemcpy(im.inv_sx, inv_sx.data(), inv_sx.size() * 4, cudaMemcpyHostToDevice));
        im.scale_version = t->scale_version;
    }
    FR_CUDA(cudaMemcpy(im.img, img.data(), img.size(), cudaMemcpyHostToDevice));
    FR_CUDA(cudaMemcpy(im.b2, b2.data(), b2.size() * 4, cudaMemcpyHostToDevice));
    FR_CUDA(cudaMemcpy(im.b3, b3.data(), b3.size() * 4, cudaMemcpyHostToDevice));
    FR_CUDA(cudaMemcpy(im.wind, wind.data(), wind.size() * 4, cudaMemcpyHostToDevice));
    im.owner = e;
    return FR_OK;
}

bool f2_supported(const fr_env *env, const fr_ensemble *e)
{
    const EnvView &v = env->v;
    if (v.task != FR_TASK_STOCK || v.K != SK2 || v.I != SI2 || e->combine != FR_COMBINE_MEAN ||
        e->out_act != 1 || v.buy_order != FR_BUY_ASCENDING)
        return false;
    // FP8: the owners publish one set of observation codes to every agent,
    // so the agents must share the first layer's activation scale
    if (e->precision != FR_PREC_BF16 && !(e->precision == FR_PREC_FP8 && e->tc && e->tc->scaled && e->tc->shared_l0))
        return false;
    F2Plan p;
    if (!f2_plan(e, p)) return false;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, env->ctx->device) != cudaSuccess)
        return false;
    return f2_smem(p).total + 1024u <= (uint32_t)optin;
}

// Clusters of a launch configuration the GPU holds at once, cached per
// kernel, cluster size and device (a host query, made at the first rollout
// of a shape; later calls, graph captures included, read the cache).
struct F2Occ {
    const void *kern;
    unsigned cluster;
    int device, n;
};
static std::vector<F2Occ> g_f2_occ;
static std::mutex g_f2_occ_mu;

static cudaError_t f2_max_clusters(const void *kern, const cudaLaunchConfig_t &cfg, int device, int *n)
{
    std::lock_guard<std::mutex> lk(g_f2_occ_mu);
    const unsigned cl = cfg.attrs[0].val.clusterDim.x;
    for (const F2Occ &o : g_f2_occ)
        if (o.kern == kern && o.cluster == cl && o.device == device) {
            *n = o.n;
            return cudaSuccess;
        }
    cudaLaunchConfig_t c = cfg;
    c.gridDim = dim3(cl, 1, 1);
    int k = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&k, kern, &c);
    if (e != cudaSuccess) return e;
    g_f2_occ.push_back(F2Occ{kern, cl, device, k});
    *n = k;
    return cudaSuccess;
}

// images are cached per ensemble (keyed by handle); released with the ensemble
struct F2Entry {
    const fr_ensemble *ens;
    F2Image im;
};
static std::vector<F2Entry> g_f2;
static std::mutex g_f2_mu;

void f2_release(const fr_ensemble *e)
{
    std::lock_guard<std::mutex> lk(g_f2_mu);
    for (size_t i = 0; i < g_f2.size(); ++i) {
        if (g_f2[i].ens == e) {
            f2_free(e->ctx, g_f2[i].im);
            g_f2.erase(g_f2.begin() + (long)i);
            return;
        }
    }
}

int f2_rollout(fr_env *env, const fr_ensemble *e, int T, const fr_traj *traj, double *metrics, cudaStream_t s)
{
    const EnvView &v = env->v;
    F2Image imv;
    bool found = false;
    {
        std::lock_guard<std::mutex> lk(g_f2_mu);
        for (size_t i = 0; i < g_f2.size(); ++i) {
            if (g_f2[i].ens != e) continue;
            if (g_f2[i].im.plan.fp8 && g_f2[i].im.scale_version != e->tc->scale_version) {
                // new activation scales: repack (the old image may still be
                // read by launches in flight on this stream)
                FR_CUDA(cudaStreamSynchronize(s));
                f2_free(e->ctx, g_f2[i].im);
                g_f2.erase(g_f2.begin() + (long)i);
                break;
            }
            imv = g_f2[i].im;
            found = true;
        }
        if (!found) {
            F2Entry en{};
            en.ens = e;
            if (!f2_plan(e, en.im.plan)) {
                set_error("fused rollout: unsupported ensemble shape");
                return FR_EINVAL;
            }
            int rc = f2_build(e, en.im);
            if (rc) return rc;
            g_f2.push_back(en);
            imv = en.im;
        }
    }
    const F2Image *im = &imv;
    const F2Plan &p = im->plan;
    if (T == 0) {
        if (metrics) FR_CUDA(launch_env_metrics(v, metrics, s));
        return FR_OK;
    }
    // asset-count slots of this env batch (host side, from the device copy)
    if (env->slot_of_env == nullptr) {
        std::vector<int32_t> ke(v.N);
        FR_CUDA(cudaMemcpy(ke.data(), v.Ke, 4ull * v.N, cudaMemcpyDeviceToHost));
        std::vector<int32_t> kes;
        for (int x : ke)
            if (std::find(kes.begin(), kes.end(), x) == kes.end()) kes.push_back(x);
        std::vector<int32_t> slot(v.N);
        for (int i = 0; i < v.N; ++i) slot[i] = (int32_t)(std::find(kes.begin(), kes.end(), ke[i]) - kes.begin());
        env->n_slots = (int)kes.size();
        int rc = dev_alloc(env->ctx, (void **)&env->slot_of_env, 4ull * v.N + 4ull * 32);
        if (rc) return rc;
        env->slot_ke = env->slot_of_env + v.N;
        FR_CUDA(cudaMemcpy(env->slot_of_env, slot.data(), 4ull * v.N, cudaMemcpyHostToDevice));
        FR_CUDA(cudaMemcpy(env->slot_ke, kes.data(), 4ull * kes.size(), cudaMemcpyHostToDevice));
        env->z_serial = 0;
    }
    const int n_ctx = env->n_slots * v.n_days;
    // the table Z in its own buffer, rebuilt only when the ensemble or the
    // env's asset-count slots change; the value log in the env's scratch
    const uint64_t x_b = 0;
    const uint64_t z_b = (uint64_t)p.M * n_ctx * p.H1 * 4;
    if (env->zbuf_bytes < x_b + z_b) {
        FR_CUDA(cudaStreamSynchronize(s));
        dev_free(env->ctx, env->zbuf, env->zbuf_bytes);
        env->zbuf = nullptr;
        env->zbuf_bytes = 0;
        int rc = dev_alloc(env->ctx, &env->zbuf, x_b + z_b);
        if (rc) return rc;
        env->zbuf_bytes = x_b + z_b;
        env->z_serial = 0;
    }
    // the value log, then one [N] array of start step counts per launch
    const uint64_t t0_b = ((uint64_t)v.N * 4 + 255) & ~255ull;
    const uint64_t vlog_b = (((uint64_t)T * v.N * 8 + 255) & ~255ull) + (uint64_t)F2_PIECES_MAX * t0_b;
    if (env->scratch_bytes < vlog_b) {
        FR_CUDA(cudaStreamSynchronize(s));
        dev_free(env->ctx, env->scratch, env->scratch_bytes);
        env->scratch = nullptr;
        env->scratch_bytes = 0;
        int rc = dev_alloc(env->ctx, &env->scratch, vlog_b);
        if (rc) return rc;
        env->scratch_bytes = vlog_b;
    }
    int64_t *vlog = (int64_t *)env->scratch;
    int32_t *t0a = (int32_t *)((char *)env->scratch + (((uint64_t)T * v.N * 8 + 255) & ~255ull));
    float *Z = (float *)((char *)env->zbuf + x_b);
    if (env->z_serial != e->serial || env->z_cache_off) {
        // Z[j][ctx][n] = W1_j[n, indicators] . x[ctx] + b1_j[n]
        FR_CUDA(set_max_smem_once((const void *)k_ztable, env->ctx->device));
        k_ztable<<<dim3((unsigned)ceil_div(n_ctx, ZT_ROWS), (unsigned)(p.H1 / ZT_COLS), (unsigned)p.M), 256,
                   ZT_SMEM, s>>>(v.ind, v.n_days, env->slot_ke, n_ctx, im->wind, p.H1, Z);
        FR_CUDA(cudaGetLastError());
        env->z_serial = e->serial;
    }

    // Tile packing (no trajectory, no auto-reset, windows of different
    // lengths): envs sorted by window, longest first, into 128-env tiles, each
    // tile running until its longest window is over; the longest tiles get
    // the lowest block indices, so they start first when the grid takes more
    // than one wave.  Every env's arithmetic is unchanged.
    const bool want_traj = traj->obs || traj->act || traj->rew || traj->rew_f32 || traj->done;
    const bool may_pack = !want_traj && !v.auto_reset && v.N > 128 && !env->pack_off;
    const int tiles = (int)ceil_div(v.N, 128);
    if (may_pack && env->pack_state == 0) {
        std::vector<int32_t> W(v.N);
        FR_CUDA(cudaMemcpy(W.data(), v.W, 4ull * v.N, cudaMemcpyDeviceToHost));
        bool uniform = true;
        for (int i = 1; i < v.N; ++i) uniform = uniform && W[i] == W[0];
        if (uniform) {
            env->pack_state = 1;
        } else {
            std::vector<int32_t> order(v.N);
            for (int i = 0; i < v.N; ++i) order[i] = i;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return W[x] > W[y]; });
            std::vector<int32_t> perm((size_t)tiles * 128, -1), tw(tiles, 2);
            double used = 0.0, spent = 0.0;
            for (int i = 0; i < v.N; ++i) {
                perm[i] = order[i];
                used += W[order[i]] - 1;
            }
            for (int t = 0; t < tiles; ++t) {
                tw[t] = W[order[(size_t)t * 128]];
                spent += 128.0 * (tw[t] - 1);
            }
            if (!env->pack_perm) {
                int rc = dev_alloc(env->ctx, (void **)&env->pack_perm, 4ull * tiles * 128);
                if (rc) return rc;
                rc = dev_alloc(env->ctx, (void **)&env->pack_tile_w, 4ull * tiles);
                if (rc) return rc;
            }
            FR_CUDA(cudaMemcpy(env->pack_perm, perm.data(), 4ull * tiles * 128, cudaMemcpyHostToDevice));
            FR_CUDA(cudaMemcpy(env->pack_tile_w, tw.data(), 4ull * tiles, cudaMemcpyHostToDevice));
            env->pack_efficiency = spent > 0 ? (float)(used / spent) : 1.0f;
            env->pack_state = 2;
        }
    }
    const bool packed = may_pack && env->pack_state == 2;

    // 16 warps when every warp's share of a hidden layer is whole 16-column
    // groups (H1, H2 multiples of 128), else 8
    const int W = (p.H1 % 128 == 0 && p.H2 % 128 == 0) ? 16 : 8;
    void (*kern)(F2Args);
    if (W == 16)
        kern = v.narrow ? (p.fp8 ? k_rollout_stock2<true, true, 16> : k_rollout_stock2<true, false, 16>)
                        : (p.fp8 ? k_rollout_stock2<false, true, 16> : k_rollout_stock2<false, false, 16>);
    else
        kern = v.narrow ? (p.fp8 ? k_rollout_stock2<true, true, 8> : k_rollout_stock2<true, false, 8>)
                        : (p.fp8 ? k_rollout_stock2<false, true, 8> : k_rollout_stock2<false, false, 8>);
    FR_CUDA(set_max_smem_once((const void *)kern, env->ctx->device));
    const uint32_t smem = f2_smem(p).total + 1024u;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3((unsigned)(32 * W), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)(2 * p.M);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // Envs per tile: 128 when the tiles fill the clusters the GPU holds at
    // once (or are packed by window); otherwise the envs are spread evenly
    // over that many clusters (at least 64 per tile), so that a batch of a
    // few thousand envs uses every SM it can: each step's owner work and
    // exchanges shrink with the rows, its MMAs (128 rows) do not.
    int TR = 128;
    if (!packed) {
        int nc = 0;
        FR_CUDA(f2_max_clusters((const void *)kern, cfg, env->ctx->device, &nc));
        if (nc > 0) TR = (int)std::min<int64_t>(128, std::max<int64_t>(64, ceil_div(v.N, nc)));
    }

    F2Args a;
    memset(&a, 0, sizeof(a));
    a.perm = packed ? env->pack_perm : nullptr;
    a.tile_w = packed ? env->pack_tile_w : nullptr;
    a.n_pos = packed ? tiles * 128 : v.N;
    a.tile_rows = TR;
    a.v = v;
    a.plan = p;
    a.img = im->img;
    a.b2 = im->b2;
    a.b3 = im->b3;
    a.dq = im->dq;
    a.inv_sx = im->inv_sx;
    a.Z = Z;
    a.slot = env->slot_of_env;
    a.n_ctx_per_agent = n_ctx;
    for (int jj = 0; jj < MAX_AGENTS; ++jj) a.w[jj] = e->host_weights[jj];
    a.T = T;
    a.tr_obs = traj->obs;
    a.obs_ld = traj->obs_ld ? traj->obs_ld : v.D;
    a.tr_act = (float *)traj->act;
    a.tr_rew = traj->rew;
    a.tr_rew_f32 = traj->rew_f32;
    a.tr_done = traj->done;
    a.vlog = vlog;
    a.t0_out = t0a;
    a.err = e->tc->err;
    a.ex = explore_of(env, env->explore_step);
    cfg.gridDim = dim3((unsigned)(2 * p.M), (unsigned)ceil_div(v.N, TR), 1);
    env->last_ctas = (int)(cfg.gridDim.x * cfg.gridDim.y);
    env->last_tile = TR;
    // Split rollout: the FP64 replay of a rollout's value log is a chain of
    // dependent divisions per env that no parallelism shortens.  Long
    // rollouts without packing, trajectory outputs or auto-reset run as K
    // launches (K = T / 64, at most 4) on an internal stream of the highest
    // priority; the replay of each piece runs on `stream` on the idle SMs
    // while the next piece's launch runs, so only the last piece's replay
    // (a short piece: T / 8 steps) follows the kernel.  Events order the
    // two streams, so the rollout stays one ordered (and graph-capturable)
    // operation on `stream`.  Every env's arithmetic is that of one launch
    // (a rollout in pieces is the same rollout).
    const int K = (!packed && !want_traj && !v.auto_reset && !env->split_off) ? std::min(F2_PIECES_MAX, T / 64) : 1;
    FR_CUDA(env_time_mark(env, 0, s));
    if (K <= 1) {
        FR_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
        FR_CUDA(env_time_mark(env, 1, s));
        FR_CUDA(launch_metrics_replay(v, vlog, T, metrics, s, t0a));
        return FR_OK;
    }
    if (!env->split_stream) {
        int lo = 0, hi = 0;
        FR_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        FR_CUDA(cudaStreamCreateWithPriority(&env->split_stream, cudaStreamNonBlocking, hi));
        for (int i = 0; i <= F2_PIECES_MAX; ++i)
            FR_CUDA(cudaEventCreateWithFlags(&env->split_ev[i], cudaEventDisableTiming));
        env->split_prio = hi;
    }
    cudaLaunchConfig_t cfg2 = cfg;
    cudaLaunchAttribute attr2[2];
    attr2[0] = attr[0];
    attr2[1].id = cudaLaunchAttributePriority;
    attr2[1].val.priority = env->split_prio;
    cfg2.attrs = attr2;
    cfg2.numAttrs = 2;
    cfg2.stream = env->split_stream;
    FR_CUDA(cudaEventRecord(env->split_ev[F2_PIECES_MAX], s));
    FR_CUDA(cudaStreamWaitEvent(env->split_stream, env->split_ev[F2_PIECES_MAX], 0));
    // the pieces' ends: the last piece is short (T / 8), so that the replay
    // left after the kernel is short, the one before it T / 4, and the
    // others share the rest evenly (80, 80, 64 and 32 steps at T = 256;
    // measured 1.720 ms per rollout against 1.747 with 74, 75, 75 and 32)
    int ends[F2_PIECES_MAX];
    {
        const int tl = std::max(16, T / 8), tp = std::max(16, T / 4);
        const int head = K >= 3 ? T - tl - tp : T - tl;        // the evenly shared steps
        const int nh = K >= 3 ? K - 2 : K - 1;                 // pieces sharing them
        for (int k = 0; k < nh; ++k) ends[k] = (k + 1) * head / nh;
        if (K >= 3) ends[K - 2] = T - tl;
        ends[K - 1] = T;
    }
    int s0 = 0;
    for (int k = 0; k < K; ++k) {
        const int Tk = ends[k] - s0;
        F2Args b = a;
        b.T = Tk;
        b.vlog = vlog + (int64_t)s0 * v.N;
        b.t0_out = (int32_t *)((char *)t0a + (uint64_t)k * t0_b);
        b.ex.g0 = a.ex.g0 + (uint32_t)s0;
        FR_CUDA(cudaLaunchKernelEx(&cfg2, kern, b));               // steps [s0, s0 + Tk)
        FR_CUDA(cudaEventRecord(env->split_ev[k], env->split_stream));
        s0 += Tk;
    }
    s0 = 0;
    for (int k = 0; k < K; ++k) {
        const int Tk = ends[k] - s0;
        FR_CUDA(cudaStreamWaitEvent(s, env->split_ev[k], 0));
        if (k == K - 1) FR_CUDA(env_time_mark(env, 1, s));
        FR_CUDA(launch_metrics_replay(v, vlog + (int64_t)s0 * v.N, Tk, k == K - 1 ? metrics : nullptr, s,
                                      (const int32_t *)((const char *)t0a + (uint64_t)k * t0_b)));
        s0 += Tk;
    }
    return FR_OK;
}

}  // namespace fr
