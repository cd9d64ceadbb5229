// Gather ceiling of a product on a given index stream: a measurement aid of
// the benchmark, not part of the library's C ABI and not part of the paper's
// method.  It is built into its own shared library (libspmv_probe.so), which
// only the benchmark loads.
//
// spmv_probe_gather sums val[k] * x[idx[k]] over k < nnz with one random
// gather and one DFMA per entry and no row structure: a grid-stride stream
// over the arrays, idx and val read with coalesced streaming loads and x
// gathered through the read-only path, as the product kernels issue them.
// Its time on a matrix's own idx/val is the practical roofline of an SpMV on
// that matrix when the gathers, not HBM, bound it.
//
//   int spmv_probe_partials(void);
//       Partial sums one call writes on the current device (threads of the
//       launch: 8 blocks of 256 per SM).
//   int spmv_probe_gather(const int32_t* idx, const double* val, int64_t nnz,
//                         const double* x, double* partial, int64_t n_partial,
//                         cudaStream_t stream);
//       idx, val: nnz entries; x: indexed by idx; partial: n_partial doubles,
//       at least spmv_probe_partials(); all device memory.  Overwrites
//       partial[0 .. spmv_probe_partials()) with one partial sum per thread
//       (their sum is the total).  Asynchronous, one launch.  Returns 0, or -1
//       for a bad argument, -4 when the launch fails.
#include <cstdint>

#include <cuda_runtime.h>

#define PROBE_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

int probe_blocks() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1) {
        (void)cudaGetLastError();
        return 0;
    }
    return sms * kBlocksPerSm;
}

__global__ void __launch_bounds__(kThreads) k_probe_gather(const int32_t* __restrict__ idx,
                                                           const double* __restrict__ val, int64_t nnz,
                                                           const double* __restrict__ x, double* __restrict__ out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;  // four entries in flight per thread
    int64_t k = t;
    for (; k + 3 * stride < nnz; k += 4 * stride) {
        s0 = fma(__ldcs(val + k), __ldg(x + __ldcs(idx + k)), s0);
        s1 = fma(__ldcs(val + k + stride), __ldg(x + __ldcs(idx + k + stride)), s1);
        s2 = fma(__ldcs(val + k + 2 * stride), __ldg(x + __ldcs(idx + k + 2 * stride)), s2);
        s3 = fma(__ldcs(val + k + 3 * stride), __ldg(x + __ldcs(idx + k + 3 * stride)), s3);
    }
    for (; k < nnz; k += stride) s0 = fma(__ldcs(val + k), __ldg(x + __ldcs(idx + k)), s0);
    out[t] = (s0 + s1) + (s2 + s3);
}

}  // namespace

PROBE_API int spmv_probe_partials(void) { return probe_blocks() * kThreads; }

PROBE_API int spmv_probe_gather(const int32_t* idx, const double* val, int64_t nnz, const double* x, double* partial,
                                int64_t n_partial, cudaStream_t stream) {
    const int blocks = probe_blocks();
    if (blocks < 1 || nnz < 0 || !partial || n_partial < (int64_t)blocks * kThreads || (nnz > 0 && (!idx || !val || !x)))
        return -1;
    k_probe_gather<<<blocks, kThreads, 0, stream>>>(idx, val, nnz, x, partial);
    if (cudaGetLastError() != cudaSuccess) return -4;
    return 0;
}
