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

// Rows of similar length: V lanes per row (dev::csr_lanes_row), no shared
// memory, no joins.  The tiles above pay for their generality (any mix of
// row lengths) with staging and segmentation work that regular rows do not
// need (the 27-point stencil: 1.28 ms with tiles, 0.87 ms with V = 4).
template <int V>
__global__ void __launch_bounds__(256) k_csr_lanes(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                                   const double* __restrict__ val, const double* __restrict__ x,
                                                   double* __restrict__ y, int32_t m) {
    dev::pdl_wait();  // launched early (launch_pdl): wait for the kernel ahead
    dev::csr_lanes_row<V>(ptr, idx, val, x, y, m, (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / V,
                          (int)(threadIdx.x & (V - 1)));
}

// Automatic choice of V: the smallest power of two giving each lane at most
// about this many of the row's entries, and at most 16 lanes.  Measured over
// banded, stencil, block-diagonal and uniform-random matrices (mean row length
// 3 to 130) it picks the fastest V or one within about 10 % of it; the tiles
// were 1.2-1.8x slower on all of them.
constexpr int kCsrLaneEntries = 8;
constexpr int kCsrMaxLanes = 16;

int csr_convert(spmv_handle* h, const spmv_csr* c, cudaStream_t s) {
    const int32_t b = h->params.csr_block_nnz;
    if (!(b == 0 || b == dev::kCsrW || b == -2 || b == -4 || b == -8 || b == -16 || b == -32))
        return set_error(SPMV_ERR_INVALID_ARG, "csr_block_nnz must be 0, %d or -V with V in {2, 4, 8, 16, 32} (got %d)",
                         dev::kCsrW, b);
    SPMV_TRY(copy_csr(h, c, s));
    SPMV_TRY(build_csr_tiles(h, h->cu, h->ptr, h->m, h->nnz, "", s));  // also what a batch runs
    SPMV_TRY(csr_prepare(h->cu));
    int32_t lanes = b < 0 ? -b : 0;
    if (b == 0) {  // automatic: lanes per row when the rows are of similar length
        Scratch tmp;
        int32_t* len = nullptr;
        SPMV_TRY(tmp.get(&len, (size_t)h->m + 1));
        SPMV_TRY(row_lengths(h->ptr, h->m, len, s));
        int32_t longest = 0;
        SPMV_TRY(max_i32(len, h->m, &longest, s, tmp));
        const double mean = (double)h->nnz / (double)h->m;
        if ((double)longest <= 2.0 * mean + 8.0) {
            lanes = 2;
            while (lanes < kCsrMaxLanes && lanes * kCsrLaneEntries < mean) lanes *= 2;
        }
    }
    h->csr_lanes = lanes;
    h->params.csr_block_nnz = lanes ? -lanes : dev::kCsrW;
    h->stored_slots = h->nnz;
    h->aux[0] = h->cu.n;
    h->aux[1] = lanes;
    return SPMV_OK;
}

int csr_run(const spmv_handle* h, const double* x, double* y, cudaStream_t s) {
    if (h->csr_lanes == 0) return csr_tiles_launch(h->cu, h->ptr, h->idx, h->val, nullptr, x, y, false, s);
    const int64_t threads = (int64_t)h->m * h->csr_lanes;
    const dim3 grid((unsigned)ceil_div(threads, 256)), block(256);
    switch (h->csr_lanes) {
        case 2: launch_pdl(k_csr_lanes<2>, grid, block, 0, s, h->ptr, h->idx, h->val, x, y, h->m); break;
        case 4: launch_pdl(k_csr_lanes<4>, grid, block, 0, s, h->ptr, h->idx, h->val, x, y, h->m); break;
        case 8: launch_pdl(k_csr_lanes<8>, grid, block, 0, s, h->ptr, h->idx, h->val, x, y, h->m); break;
        case 16: launch_pdl(k_csr_lanes<16>, grid, block, 0, s, h->ptr, h->idx, h->val, x, y, h->m); break;
        default: launch_pdl(k_csr_lanes<32>, grid, block, 0, s, h->ptr, h->idx, h->val, x, y, h->m); break;
    }
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

}  // namespace spmv
