// Gather ceiling of a product on a given index stream (a measurement aid, not
// part of the paper's method): sum of val[k] * x[idx[k]] with one gather and
// one DFMA per entry, no row structure, the loads issued as the product
// kernels issue them.
#include "internal.cuh"

namespace spmv {

constexpr int kProbeBlocks = 152 * 8, kProbeThreads = 256;
static_assert(kProbeBlocks * kProbeThreads == SPMV_PROBE_PARTIALS, "partial count");

__global__ void __launch_bounds__(kProbeThreads) k_probe_gather(const int32_t* __restrict__ idx,
                                                                const double* __restrict__ val, int64_t nnz,
                                                                const double* __restrict__ x, double* __restrict__ out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;  // four entries in flight per thread
    int64_t k = t;
    for (; k + 3 * stride < nnz; k += 4 * stride) {
        s0 = fma(__ldcs(val + k), dev::ldx(x, __ldcs(idx + k)), s0);
        s1 = fma(__ldcs(val + k + stride), dev::ldx(x, __ldcs(idx + k + stride)), s1);
        s2 = fma(__ldcs(val + k + 2 * stride), dev::ldx(x, __ldcs(idx + k + 2 * stride)), s2);
        s3 = fma(__ldcs(val + k + 3 * stride), dev::ldx(x, __ldcs(idx + k + 3 * stride)), s3);
    }
    for (; k < nnz; k += stride) s0 = fma(__ldcs(val + k), dev::ldx(x, __ldcs(idx + k)), s0);
    out[t] = (s0 + s1) + (s2 + s3);
}

}  // namespace spmv

using namespace spmv;

extern "C" int spmv_probe_gather(const int32_t* idx, const double* val, int64_t nnz, const double* x,
                                 double* partial, cudaStream_t stream) {
    if (nnz < 0 || !partial || (nnz > 0 && (!idx || !val || !x))) return set_error(SPMV_ERR_INVALID_ARG, "bad argument");
    k_probe_gather<<<kProbeBlocks, kProbeThreads, 0, stream>>>(idx, val, nnz, x, partial);
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}
