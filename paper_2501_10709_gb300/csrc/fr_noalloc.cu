// fr_noalloc.cu -- ensemble_act for callers that must not allocate.
//
// ensemble_act takes its scratch (the hidden activations of the plain fp32
// path and the per-agent outputs before they are combined) from the
// stream-ordered allocator.  Some callers cannot allow that: a real-time
// loop that reserved its memory up front and must not stall in (or fail in)
// the allocator mid-run, or a plugin host that owns every device buffer and
// forbids the library to allocate behind its back.  ensemble_act_noalloc runs the
// same kernels on a scratch area that is part of this library's image: a
// file-scope device array of fixed size that every GPU loading the library
// holds until the process exits.  It calls no cudaMalloc, cudaFree or other
// allocating routine.
#include "fr_common.cuh"

namespace fr {
namespace {

// Scratch for one call: 16 MiB.  A call needs (2 * hidden_max + out) * M
// floats per observation row on the fp32 path and out * M floats per row on
// the tensor-core paths; larger batches are rejected.
constexpr uint64_t kNoAllocFloats = (16ull << 20) / sizeof(float);

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address comes from
// the runtime, looked up on every call (a host query that allocates
// nothing; no address is kept that a device reset could leave stale).
int scratch_address(float **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                                 "cudaGetSymbolAddress(scratch)");
    *out = (float *)p;
    return FR_OK;
}

}  // namespace
}  // namespace fr

using namespace fr;

extern "C" int ensemble_act_noalloc(const fr_ensemble *e, const float *obs, int32_t n, void *act,
                                    void *stream)
{
    FR_NVTX("ensemble_act_noalloc");
    FR_CHECK(e && n >= 0, FR_EINVAL, "ensemble_act_noalloc: bad argument");
    if (n == 0) return FR_OK;
    FR_CHECK(obs && act, FR_EINVAL, "ensemble_act_noalloc: NULL obs or act");
    const int out = e->dims[e->L];
    int wmax = 0;
    for (int l = 1; l < e->L; ++l) wmax = wmax > e->dims[l] ? wmax : e->dims[l];
    const uint64_t hidden = e->precision == FR_PREC_FP32 ? 2ull * e->M * (uint64_t)n * wmax : 0;
    const uint64_t need = hidden + (uint64_t)e->M * n * out;
    const uint64_t per_row = need / (uint64_t)n;
    FR_CHECK(need <= kNoAllocFloats, FR_EINVAL,
             "ensemble_act_noalloc: %d rows need %llu scratch floats; the fixed scratch holds %llu "
             "(at most %llu rows for this ensemble)",
             n, (unsigned long long)need, (unsigned long long)kNoAllocFloats,
             (unsigned long long)(kNoAllocFloats / per_row));
    FR_CUDA(cudaSetDevice(e->ctx->device));
    float *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    // Every element of both regions is written before it is read, so
    // nothing has to start at zero: y first (per-agent outputs), then the
    // two hidden-layer buffers of the fp32 path.
    float *y = scratch;
    float *hid = scratch + (uint64_t)e->M * n * out;
    cudaStream_t s = (cudaStream_t)stream;
    if (e->precision == FR_PREC_FP32) {
        FR_CUDA(forward_plain(e, obs, e->dims[0], n, y, hid, s));
    } else {
        rc = tc_forward(e, obs, e->dims[0], n, y, s);
        if (rc) return rc;
    }
    if (e->combine == FR_COMBINE_MEAN)
        FR_CUDA(launch_combine_mean(y, (int64_t)n * out, out, e->weights, e->M, n, out, (float *)act, out, s));
    else
        FR_CUDA(launch_combine_vote(y, (int64_t)n * out, out, e->M, n, e->n_act, e->dueling, (uint8_t *)act, s));
    return FR_OK;
}
