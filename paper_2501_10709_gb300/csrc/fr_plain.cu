// fr_plain.cu -- the plain, unfused FP32 actor path: one SIMT dense-layer
// kernel launch per layer (all agents of the ensemble in one grid), then a
// separate combine launch.  It is the comparison path for the fused BF16
// rollout and the fp32 reference the tensor-core kernels are held to.
#include "fr_common.cuh"

namespace fr {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// Y[a][r][o] = act( sum_k X[a][r][k] * W_a[o][k] + b_a[o] ), ACT: 0 ReLU,
// 1 tanh, 2 identity.  W_a / b_a live at P + a*p_stride + w_off / b_off.
template <int ACT>
__global__ void __launch_bounds__(NT) k_dense_f32(const float *__restrict__ X, int64_t x_stride, int ldx,
                                                  const float *__restrict__ P, int64_t p_stride,
                                                  int64_t w_off, int64_t b_off,
                                                  float *__restrict__ Y, int64_t y_stride, int ldy,
                                                  int n, int fin, int fout)
{
    const int a = blockIdx.z;
    X += a * x_stride;
    const float *W = P + a * p_stride + w_off;
    const float *B = P + a * p_stride + b_off;
    Y += a * y_stride;
    __shared__ float As[BK][BM + 1];
    __shared__ float Bs[BK][BN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    for (int k0 = 0; k0 < fin; k0 += BK) {
        for (int i = threadIdx.x; i < BM * BK; i += NT) {
            const int r = i / BK, kk = i % BK;
            const int gr = row0 + r, gk = k0 + kk;
            As[kk][r] = (gr < n && gk < fin) ? X[(int64_t)gr * ldx + gk] : 0.0f;
        }
        for (int i = threadIdx.x; i < BN * BK; i += NT) {
            const int o = i / BK, kk = i % BK;
            const int go = col0 + o, gk = k0 + kk;
            Bs[kk][o] = (go < fout && gk < fin) ? W[(int64_t)go * fin + gk] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = row0 + ty * 4 + i;
        if (r >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int o = col0 + tx * 4 + j;
            if (o >= fout) continue;
            float y = acc[i][j] + B[o];
            if (ACT == 0) y = fmaxf(y, 0.0f);
            else if (ACT == 1) y = tanhf(y);
            Y[(int64_t)r * ldy + o] = y;
        }
    }
}

// a = a_0 + sum_{j>=1} w_j (a_j - a_0), rounded at every operation
__global__ void k_combine_mean(const float *__restrict__ Y, int64_t y_stride, int ldy,
                               const float *__restrict__ w, int M, int n, int K,
                               float *__restrict__ out, int ldo)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * K) return;
    const int64_t r = i / K, k = i % K;
    const float a0 = Y[r * ldy + k];
    float acc = a0;
    for (int j = 1; j < M; ++j)
        acc = __fadd_rn(acc, __fmul_rn(w[j], __fsub_rn(Y[j * y_stride + r * ldy + k], a0)));
    out[r * ldo + k] = acc;
}

// per-agent argmax (lowest index on ties), then the action with the strictly
// largest count, else hold (1)
__global__ void k_combine_vote(const float *__restrict__ Y, int64_t y_stride, int ldy, int M,
                               int n, int nact, uint32_t dueling, uint8_t *__restrict__ out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int cnt[3] = {0, 0, 0};
    for (int j = 0; j < M; ++j) {
        const int best = HeadQ(Y + j * y_stride + (int64_t)r * ldy, (dueling >> j) & 1u, nact).argmax();
        if (best < 3) cnt[best]++;
    }
    int best = 0, bc = cnt[0];
    bool tie = false;
    for (int c = 1; c < 3; ++c) {
        if (cnt[c] > bc) { bc = cnt[c]; best = c; tie = false; }
        else if (cnt[c] == bc) tie = true;
    }
    out[r] = (uint8_t)(tie ? 1 : best);
}

// Q-values after each agent's head: q[j][r][a], a < nact.
__global__ void k_heads(const float *__restrict__ Y, int64_t y_stride, int ldy, int M, int n, int nact,
                        uint32_t dueling, float *__restrict__ q)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * n) return;
    const int j = (int)(i / n), r = (int)(i % n);
    const HeadQ h(Y + j * y_stride + (int64_t)r * ldy, (dueling >> j) & 1u, nact);
    for (int a = 0; a < nact; ++a) q[i * nact + a] = h.q(a);
}

// DQN / Double DQN learning targets y[j][r] = r + (done ? 0 : gamma Q_target(s', a*)).
__global__ void k_q_targets(const float *__restrict__ Yon, const float *__restrict__ Ytg, int64_t y_stride, int ldy,
                            int M, int n, int nact, uint32_t dueling, const float *__restrict__ rew,
                            const uint8_t *__restrict__ done, float gamma, int double_q, float *__restrict__ y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * n) return;
    const int j = (int)(i / n), r = (int)(i % n);
    const bool d = (dueling >> j) & 1u;
    const HeadQ tg(Ytg + j * y_stride + (int64_t)r * ldy, d, nact);
    const int a = double_q ? HeadQ(Yon + j * y_stride + (int64_t)r * ldy, d, nact).argmax() : tg.argmax();
    const float rr = rew[r];
    y[i] = (done && done[r]) ? rr : __fadd_rn(rr, __fmul_rn(gamma, tg.q(a)));
}

}  // namespace

cudaError_t launch_heads(const float *Y, int64_t y_stride, int ldy, int M, int n, int nact, uint32_t dueling,
                         float *q, cudaStream_t s)
{
    k_heads<<<ceil_div((int64_t)M * n, 256), 256, 0, s>>>(Y, y_stride, ldy, M, n, nact, dueling, q);
    return cudaGetLastError();
}

cudaError_t launch_q_targets(const float *Yon, const float *Ytg, int64_t y_stride, int ldy, int M, int n, int nact,
                             uint32_t dueling, const float *rew, const uint8_t *done, float gamma, int double_q,
                             float *y, cudaStream_t s)
{
    k_q_targets<<<ceil_div((int64_t)M * n, 256), 256, 0, s>>>(Yon, Ytg, y_stride, ldy, M, n, nact, dueling, rew,
                                                               done, gamma, double_q, y);
    return cudaGetLastError();
}

cudaError_t launch_dense_f32(const float *X, int64_t x_stride, int ldx, const float *P,
                             int64_t p_stride, int64_t w_off, int64_t b_off, float *Y,
                             int64_t y_stride, int ldy, int n, int fin, int fout, int act, int M,
                             cudaStream_t s)
{
    dim3 grid(ceil_div(fout, BN), ceil_div(n, BM), M);
    if (act == 0)
        k_dense_f32<0><<<grid, NT, 0, s>>>(X, x_stride, ldx, P, p_stride, w_off, b_off, Y, y_stride, ldy, n, fin, fout);
    else if (act == 1)
        k_dense_f32<1><<<grid, NT, 0, s>>>(X, x_stride, ldx, P, p_stride, w_off, b_off, Y, y_stride, ldy, n, fin, fout);
    else
        k_dense_f32<2><<<grid, NT, 0, s>>>(X, x_stride, ldx, P, p_stride, w_off, b_off, Y, y_stride, ldy, n, fin, fout);
    return cudaGetLastError();
}

namespace {
// Maximum of |x| over `count` floats of matrix j (at x + j * stride), as float
// bits atomically maxed into out[j * out_stride] (non-negative floats order
// like their bit patterns).
__global__ void k_absmax(const float *__restrict__ x, int64_t stride, int64_t count, unsigned *out,
                         int out_stride)
{
    const float *xj = x + (int64_t)blockIdx.y * stride;
    float m = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(xj[i]));
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + (int64_t)blockIdx.y * out_stride, __float_as_uint(m));
}
}  // namespace

cudaError_t launch_absmax(const float *x, int64_t stride, int64_t count, int M, unsigned *out, int out_stride,
                          cudaStream_t s)
{
    const long long b = ((long long)count + 255) / 256;
    const unsigned blocks = (unsigned)(b < 1024 ? (b > 0 ? b : 1) : 1024);
    k_absmax<<<dim3(blocks, M), 256, 0, s>>>(x, stride, count, out, out_stride);
    return cudaGetLastError();
}

cudaError_t launch_combine_mean(const float *Y, int64_t y_stride, int ldy, const float *w, int M,
                                int n, int K, float *out, int ldo, cudaStream_t s)
{
    const int64_t tot = (int64_t)n * K;
    k_combine_mean<<<ceil_div(tot, 256), 256, 0, s>>>(Y, y_stride, ldy, w, M, n, K, out, ldo);
    return cudaGetLastError();
}

cudaError_t launch_combine_vote(const float *Y, int64_t y_stride, int ldy, int M, int n, int nact,
                                uint32_t dueling, uint8_t *out, cudaStream_t s)
{
    k_combine_vote<<<ceil_div(n, 256), 256, 0, s>>>(Y, y_stride, ldy, M, n, nact, dueling, out);
    return cudaGetLastError();
}

}  // namespace fr
