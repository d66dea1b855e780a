// fr_metrics.cu -- the Sec. 6.1 metric list and the Sec. 4.3 discounted
// trajectory return, computed on the device from a stored trajectory (the
// consumer side of the T x N sample tensors).  One thread per env walks its
// rows in time order in FP64; every operation is an explicitly rounded
// intrinsic, so no FMA contraction changes a result.
#include "fr_common.cuh"
#include "fr_env_dev.cuh"

namespace fr {
namespace {

__global__ void k_traj_metrics(int T, int N, const int64_t *__restrict__ rew, const uint8_t *__restrict__ done,
                               int64_t v0, double ann, double gamma, double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double mu = 0.0, m2 = 0.0, mdd = 0.0, down2 = 0.0, up = 0.0, dn = 0.0, disc = 0.0, g = 1.0;
    int64_t peak = v0, vlast = v0, v = v0;
    int n = 0;
    for (int t = 0; t < T; ++t) {
        const int64_t r = rew[(int64_t)t * N + i];
        const int64_t v1 = v + r;
        const double rho = __dsub_rn(__ddiv_rn((double)v1, (double)v), 1.0);
        n += 1;
        acc_push(mu, m2, mdd, peak, vlast, n, v, v1);
        if (rho < 0.0) {
            down2 = __dadd_rn(down2, __dmul_rn(rho, rho));
            dn = __dadd_rn(dn, -rho);
        } else {
            up = __dadd_rn(up, rho);
        }
        g = __dmul_rn(g, gamma);
        disc = __dadd_rn(disc, __dmul_rn(g, (double)r));
        v = v1;
        if (done && done[(int64_t)t * N + i]) break;
    }
    double *o = out + (int64_t)i * 11;
    acc_final(mu, m2, mdd, vlast, v0, n, ann, o);
    const double nd = (double)n;
    const double cr = o[0], dd_max = -o[2];
    const double annual = n > 0 ? __dsub_rn(pow(__ddiv_rn((double)vlast, (double)v0), __ddiv_rn(ann, nd)), 1.0) : 0.0;
    o[3] = annual;
    o[4] = n >= 2 ? __dmul_rn(__dsqrt_rn(__ddiv_rn(m2, __dsub_rn(nd, 1.0))), __dsqrt_rn(ann)) : 0.0;
    o[5] = dd_max != 0.0 ? __ddiv_rn(cr, dd_max) : 0.0;
    const double ddown = n > 0 ? __dsqrt_rn(__ddiv_rn(down2, nd)) : 0.0;
    o[6] = ddown != 0.0 ? __dmul_rn(__ddiv_rn(mu, ddown), __dsqrt_rn(ann)) : 0.0;
    o[7] = dd_max != 0.0 ? __ddiv_rn(annual, dd_max) : 0.0;
    o[8] = dn != 0.0 ? __ddiv_rn(up, dn) : 0.0;
    o[9] = disc;
    o[10] = nd;
}

}  // namespace
}  // namespace fr

using namespace fr;

extern "C" int trajectory_metrics(const int64_t *rew, const uint8_t *done, int32_t T, int32_t N, int64_t v0,
                                  double ann, double gamma, double *out, void *stream)
{
    FR_NVTX("trajectory_metrics");
    FR_CHECK(T >= 0 && N >= 0 && v0 > 0 && ann > 0.0 && isfinite(gamma), FR_EINVAL,
             "trajectory_metrics: need T, N >= 0, v0 > 0, ann > 0, finite gamma");
    if (N == 0) return FR_OK;
    FR_CHECK(out && (rew || T == 0), FR_EINVAL, "trajectory_metrics: NULL rew or out");
    cudaStream_t s = (cudaStream_t)stream;
    k_traj_metrics<<<ceil_div(N, 128), 128, 0, s>>>(T, N, rew, done, v0, ann, gamma, out);
    FR_CUDA(cudaGetLastError());
    return FR_OK;
}
