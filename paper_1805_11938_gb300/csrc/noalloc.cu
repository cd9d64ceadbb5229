// spmv_csr_run_noalloc: y = A x straight from a caller's CSR arrays, with no
// handle and no device allocation of any kind.
//
// Who needs it: callers that cannot call cudaMalloc at the moment they need a
// product -- code that runs under a memory manager which has already reserved
// every device byte (a framework's caching allocator, an application's own
// pool), or latency-critical paths that must not enter the CUDA allocator,
// whose calls can synchronise the whole device.  They pass inputs and outputs
// they already own; the little scratch the method needs lives in this file's
// static device array instead.
//
// Method: the same segmented-sum scheme as the CSR5 kernels, on the plain CSR
// order.  The nonzeros are cut into tiles of 32 x kNaSigma; lane c of the warp
// for tile t walks nonzeros t*S + c*kNaSigma .. + kNaSigma - 1, finding its
// first row by binary search in ptr and later rows by walking ptr, with one
// DFMA per nonzero; partial sums across lanes are joined by a segmented
// suffix sum over the lanes.  The part of a row that continues from an
// earlier tile is stored in the scratch array (carry) and a second launch adds
// those carries in tile order and zeroes the empty rows.
//
// Scratch: kNaMaxTiles tiles (one double and one int each, 6 MiB), so at most
// kNaMaxTiles * 32 * kNaSigma = 536,870,912 nonzeros; larger inputs are
// rejected with SPMV_ERR_TOO_LARGE.  Every GPU that loads this library holds
// the array until the process exits.  Nothing in it has to start at zero:
// every entry a call reads was written earlier in that same call.  All calls
// share the one array, so two calls whose kernels overlap on the GPU (on
// different streams) race and give wrong results; order them on one stream
// or synchronise between them.
#include <mutex>

#include "internal.cuh"
#include "kernels.cuh"

namespace spmv {
namespace {

constexpr int kNaSigma = 32;
constexpr int64_t kNaTile = 32LL * kNaSigma;
constexpr int64_t kNaMaxTiles = 1LL << 19;

struct NaScratch {
    double carry[kNaMaxTiles];   // partial sum of the row a tile begins inside of
    int32_t row0[kNaMaxTiles];   // row holding the tile's first nonzero
};

static __device__ __align__(256) NaScratch g_na_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
NaScratch* g_na_addr[kMaxDevices] = {};

// Device address of this device's copy of g_na_scratch (looked up once per
// device, with that device current).
int na_scratch(NaScratch** out) {
    int dev = 0;
    SPMV_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(SPMV_ERR_INVALID_ARG, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_na_addr[dev] = static_cast<NaScratch*>(p);
    }
    *out = g_na_addr[dev];
    return SPMV_OK;
}

__global__ void __launch_bounds__(256) k_na_tiles(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                                  const double* __restrict__ val, int32_t m, int64_t nnz,
                                                  int64_t ntiles, const double* __restrict__ x, double* __restrict__ y,
                                                  NaScratch* __restrict__ sc) {
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    const int64_t base = t * kNaTile;
    const int64_t k0 = base + (int64_t)lane * kNaSigma;
    const int64_t k1 = k0 + kNaSigma < nnz ? k0 + kNaSigma : nnz;
    // rows: the row holding k0 (or, for an idle lane, none)
    int32_t row = -1, end = 0;
    if (k0 < nnz) {
        row = dev::row_of_nnz(ptr, m, k0);
        end = ptr[row + 1];
    }
    const int32_t trow = __shfl_sync(dev::kFull, row, 0);
    const bool cont = ptr[trow] != base;  // the tile begins inside row trow
    // segments: `head` = part of the lane's first row begun before k0 (if it
    // was), complete rows are written directly, `cur` = the open last segment
    double cur = 0.0, head = 0.0;
    bool own = (k0 < nnz) && (ptr[row] == k0 || lane == 0);
    const bool first_owned = own;
    int nseg = (k0 < nnz) ? 1 : 0;
    for (int64_t k = k0; k < k1; ++k) {
        if (k == end) {  // the segment ends before k
            if (own) {
                if (row == trow && cont && lane == 0 && nseg == 1) sc->carry[t] = cur;
                else y[row] = cur;
            } else {
                head = cur;
            }
            cur = 0.0;
            own = true;
            ++nseg;
            do {
                ++row;
                end = ptr[row + 1];
            } while (end == k);
        }
        cur = fma(__ldcs(val + k), dev::ldx(x, __ldcs(idx + k)), cur);
    }
    // lanes whose whole range continues a row begun earlier pass it on
    const bool has_start = (k0 < nnz) && (first_owned || nseg > 1);
    if (!has_start) head = cur;
    // T_c = head_c + (lane c holds no segment start ? T_{c+1} : 0)
    double T = head;
    int stop = has_start;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const double Tn = __shfl_down_sync(dev::kFull, T, d);
        const int sn = __shfl_down_sync(dev::kFull, stop, d);
        if (!stop && lane + d < 32) {
            T += Tn;
            stop = sn;
        }
    }
    double next = __shfl_down_sync(dev::kFull, T, 1);
    if (lane == 31) next = 0.0;
    if (has_start) {
        const double tot = cur + next;
        if (own && lane == 0 && nseg == 1 && cont) sc->carry[t] = tot;  // whole lane 0 continues an earlier row
        else y[row] = tot;
    }
    if (lane == 0) sc->row0[t] = trow;
}

// Adds each continuing row's carries in tile order; zeroes the empty rows.
__global__ void __launch_bounds__(256) k_na_calibrate(const int32_t* __restrict__ ptr, int32_t m, int64_t ntiles,
                                                      double* __restrict__ y, const NaScratch* __restrict__ sc) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t i = g; i < m; i += (int64_t)gridDim.x * blockDim.x)
        if (ptr[i + 1] == ptr[i]) y[i] = 0.0;
    for (int64_t t = g; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = sc->row0[t];
        const int64_t start = ptr[r];
        if (start == t * kNaTile) continue;                                  // tile t begins row r
        if (t > 0 && sc->row0[t - 1] == r && start < (t - 1) * kNaTile) continue;  // not the first continuing tile
        double acc = sc->carry[t];
        for (int64_t u = t + 1; u < ntiles && sc->row0[u] == r; ++u) acc += sc->carry[u];
        y[r] += acc;
    }
}

}  // namespace
}  // namespace spmv

using namespace spmv;

extern "C" SPMV_API int spmv_csr_run_noalloc(const spmv_csr* csr, const double* x, double* y, cudaStream_t stream) {
    if (!csr || !x || !y) return set_error(SPMV_ERR_INVALID_ARG, "csr, x or y is NULL");
    if (csr->m <= 0 || csr->n <= 0 || csr->nnz < 0 || !csr->ptr || (csr->nnz > 0 && (!csr->idx || !csr->val)))
        return set_error(SPMV_ERR_INVALID_ARG, "malformed csr argument");
    if ((const void*)x == (const void*)y) return set_error(SPMV_ERR_INVALID_ARG, "x and y must not alias");
    const int64_t ntiles = (csr->nnz + kNaTile - 1) / kNaTile;
    if (ntiles > kNaMaxTiles)
        return set_error(SPMV_ERR_TOO_LARGE, "spmv_csr_run_noalloc handles at most %lld nonzeros (got %lld)",
                         (long long)(kNaMaxTiles * kNaTile), (long long)csr->nnz);
    NaScratch* sc = nullptr;
    SPMV_TRY(na_scratch(&sc));
    if (ntiles > 0)
        k_na_tiles<<<grid_for(ntiles * 32, 256), 256, 0, stream>>>(csr->ptr, csr->idx, csr->val, csr->m, csr->nnz,
                                                                   ntiles, x, y, sc);
    const int64_t n2 = ntiles > csr->m ? ntiles : csr->m;
    const int g = grid_capped(n2, 256, 32);
    k_na_calibrate<<<g, 256, 0, stream>>>(csr->ptr, csr->m, ntiles, y, sc);
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}
