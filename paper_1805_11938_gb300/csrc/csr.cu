// CSR (Sec. II-B "CSR"): y_i = sum of val[k] * x[idx[k]] over row i's range.
// The handle keeps a copy of the CSR arrays plus the nonzero tiles' first
// rows (see build_csr_tiles); each warp of a 256-thread block processes one
// tile of kCsrW nonzeros.
#include <algorithm>

#include "internal.cuh"

namespace spmv {

// Warp w of the grid takes tiles w, w + warps, ... (tiles hold equal numbers
// of nonzeros, so the static split is balanced).
template <bool ADD>
__global__ void __launch_bounds__(256) k_csr_tiles(dev::CsrArgs a) {
    extern __shared__ __align__(16) unsigned char csr_smem[];
    dev::CsrWarpSmem* S = reinterpret_cast<dev::CsrWarpSmem*>(csr_smem);
    dev::pdl_wait();  // launched early (launch_pdl): wait for the kernel ahead
    const int w = threadIdx.x >> 5;
    const int32_t stride = (int32_t)gridDim.x * dev::kCsrWarps;
    for (int32_t t = (int32_t)blockIdx.x * dev::kCsrWarps + w; t < a.ntiles; t += stride)
        dev::csr_tile<ADD>(a, t, S[w], threadIdx.x & 31);
}

__global__ void __launch_bounds__(256) k_csr_zero(dev::CsrArgs a) {
    dev::pdl_wait();
    dev::csr_zero(a, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

int csr_prepare(CsrTiles& ct) {
    // per device: the attribute belongs to the current context
    SPMV_CUDA(cudaFuncSetAttribute(k_csr_tiles<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)dev::kCsrSmemBytes));
    SPMV_CUDA(cudaFuncSetAttribute(k_csr_tiles<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)dev::kCsrSmemBytes));
    int dev = 0, sms = 0, per_sm = 0;
    SPMV_CUDA(cudaGetDevice(&dev));
    SPMV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SPMV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_csr_tiles<false>, 256, dev::kCsrSmemBytes));
    // two waves of resident blocks, warps striding over the tiles (measured:
    // power-law 2e6 119 -> 110 us and rows of 100 251 -> 219 us against one
    // tile per warp; one wave and four waves slightly slower)
    const int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1) * 2;
    ct.grid = (int32_t)std::min<int64_t>(cap, ceil_div(ct.n, dev::kCsrWarps));
    return SPMV_OK;
}

dev::CsrArgs csr_tile_args(const CsrTiles& ct, const int32_t* ptr, const int32_t* idx, const double* val,
                           const int32_t* row_map, const double* x, double* y) {
    return dev::CsrArgs{ct.tile_row, ptr,  idx,          val,  row_map, ct.slot_head, ct.slot_tail,
                        ct.cnt,      ct.rows, (int32_t)ct.nnz, ct.n, x,       y};
}

int csr_tiles_launch(const CsrTiles& ct, const int32_t* ptr, const int32_t* idx, const double* val,
                     const int32_t* row_map, const double* x, double* y, bool add, cudaStream_t s) {
    const dev::CsrArgs a = csr_tile_args(ct, ptr, idx, val, row_map, x, y);
    if (ct.n > 0) {
        if (add) launch_pdl(k_csr_tiles<true>, dim3(ct.grid), dim3(256), dev::kCsrSmemBytes, s, a);
        else launch_pdl(k_csr_tiles<false>, dim3(ct.grid), dim3(256), dev::kCsrSmemBytes, s, a);
    } else if (!add && ct.rows > 0) {
        launch_pdl(k_csr_zero, dim3(grid_for(ct.rows, 256)), dim3(256), 0, s, a);
    }
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

int csr_convert(spmv_handle* h, const spmv_csr* c, cudaStream_t s) {
    if (h->params.csr_block_nnz != 0 && h->params.csr_block_nnz != dev::kCsrW)
        return set_error(SPMV_ERR_INVALID_ARG, "csr_block_nnz must be 0 or %d (got %d)", dev::kCsrW,
                         h->params.csr_block_nnz);
    h->params.csr_block_nnz = dev::kCsrW;
    SPMV_TRY(copy_csr(h, c, s));
    SPMV_TRY(build_csr_tiles(h, h->cu, h->ptr, h->m, h->nnz, "", s));
    SPMV_TRY(csr_prepare(h->cu));
    h->stored_slots = h->nnz;
    h->aux[0] = h->cu.n;
    return SPMV_OK;
}

int csr_run(const spmv_handle* h, const double* x, double* y, cudaStream_t s) {
    return csr_tiles_launch(h->cu, h->ptr, h->idx, h->val, nullptr, x, y, false, s);
}

}  // namespace spmv
