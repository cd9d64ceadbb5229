// CSR5 (Sec. II-B "CSR5", Table I): the nonzeros are cut into tiles of
// omega x sigma = 32 x sigma entries (omega = the warp width), each stored
// transposed so one tile row is 32 consecutive values; a tile descriptor
// (tile_ptr, bit flags, y_off, seg_off) lets a warp compute the tile's
// segmented sums without the row pointers.  Layout and flag conventions:
//   * column c of tile t holds nonzeros t*S + c*sigma + r, slot (r, c) is
//     stored at t*S + r*32 + c; the last tile is padded (col 0, value +0.0);
//   * a slot is flagged when it starts a row, and the first slot of every
//     tile is flagged (Table I's tile 1); flags[t*32 + c] has bit r set for
//     flagged slot (r, c);
//   * tile_ptr[t] = the row holding nonzero t*S, tile_ptr[ntiles] = m;
//   * y_off[t*32 + c] = flagged slots of tile t in lanes before c;
//     seg_off[t] bit c = lane c holds no flagged slot;
//   * a tile whose row span contains an empty row lists the row of every
//     flagged slot (empty_rows[empty_ptr[t] ..]).
// The product is one launch, one warp per tile; rows crossing tile
// boundaries are joined by the last of their tiles to finish (see csr5_tile),
// and the tile warps share out the zeroing of the empty rows.
#include "internal.cuh"
#include "kernels.cuh"

namespace spmv {

using dev::row_of_nnz;

__global__ void k_tile_ptr(const int32_t* __restrict__ ptr, int32_t m, int64_t nnz, int64_t nt, int64_t S,
                           int32_t* __restrict__ tile_ptr) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < nt) tile_ptr[t] = row_of_nnz(ptr, m, t * S);
    else if (t == nt) tile_ptr[nt] = m;
}

// One thread per (tile, lane): the lane's flag bits.
__global__ void k_flags(const int32_t* __restrict__ ptr, int32_t m, int64_t nnz, int64_t nt, int32_t sigma,
                        uint32_t* __restrict__ flags) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nt * 32) return;
    const int64_t t = g >> 5;
    const int c = (int)(g & 31);
    const int64_t k0 = t * 32LL * sigma + (int64_t)c * sigma;
    uint32_t f = 0;
    if (k0 < nnz) {
        int32_t row = row_of_nnz(ptr, m, k0);
        for (int r = 0; r < sigma; ++r) {
            const int64_t k = k0 + r;
            if (k >= nnz) break;
            while (ptr[row + 1] <= k) ++row;  // next nonempty row
            if (ptr[row] == k || (c == 0 && r == 0)) f |= 1u << r;
        }
    }
    flags[g] = f;
}

// One warp per tile: y_off (exclusive flag counts over lanes) and seg_off.
__global__ void k_desc(const uint32_t* __restrict__ flags, int64_t nt, int32_t* __restrict__ y_off,
                       uint32_t* __restrict__ seg_off, int32_t* __restrict__ nflag) {
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= nt) return;
    const int nf = __popc(flags[t * 32 + lane]);
    int inc = nf;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(dev::kFull, inc, d);
        if (lane >= d) inc += v;
    }
    y_off[t * 32 + lane] = inc - nf;
    const unsigned none = __ballot_sync(dev::kFull, nf == 0);
    if (lane == 0) seg_off[t] = none;
    if (lane == 31) nflag[t] = inc;
}

__global__ void k_tiles(const int32_t* __restrict__ idx, const double* __restrict__ val, int64_t nnz, int64_t nt,
                        int32_t sigma, int32_t* __restrict__ tidx, double* __restrict__ tval) {
    const int64_t S = 32LL * sigma;
    for (int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; slot < nt * S;
         slot += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = slot / S, w = slot % S, r = w >> 5, c = w & 31;
        const int64_t k = t * S + c * sigma + r;
        if (k < nnz) {
            tidx[slot] = idx[k];
            tval[slot] = val[k];
        } else {
            tidx[slot] = 0;
            tval[slot] = 0.0;
        }
    }
}

__global__ void k_empty_flag(const int32_t* __restrict__ ptr, int32_t m, int32_t* __restrict__ e) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i <= m) e[i] = (i < m && ptr[i + 1] == ptr[i]) ? 1 : 0;
}

// cnt[t] = number of flagged slots if tile t's row span holds an empty row, else 0.
__global__ void k_listed(const int32_t* __restrict__ ptr, int32_t m, int64_t nnz, int64_t nt, int64_t S,
                         const int32_t* __restrict__ tile_ptr, const int32_t* __restrict__ E,
                         const int32_t* __restrict__ nflag, int32_t* __restrict__ cnt) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t > nt) return;
    if (t == nt) {
        cnt[nt] = 0;
        return;
    }
    const int64_t last = (t + 1) * S - 1 < nnz - 1 ? (t + 1) * S - 1 : nnz - 1;
    const int32_t lr = row_of_nnz(ptr, m, last);
    cnt[t] = (E[lr] - E[tile_ptr[t]] > 0) ? nflag[t] : 0;
}

__global__ void k_list_rows(const int32_t* __restrict__ ptr, int32_t m, int64_t nnz, int64_t nt, int32_t sigma,
                            const uint32_t* __restrict__ flags, const int32_t* __restrict__ y_off,
                            const int32_t* __restrict__ eptr, int32_t* __restrict__ erows) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= nt * 32) return;
    const int64_t t = g >> 5;
    if (eptr[t + 1] == eptr[t]) return;
    const int c = (int)(g & 31);
    const uint32_t f = flags[g];
    const int64_t k0 = t * 32LL * sigma + (int64_t)c * sigma;
    int j = 0;
    for (int r = 0; r < sigma; ++r)
        if ((f >> r) & 1u) erows[eptr[t] + y_off[g] + j++] = row_of_nnz(ptr, m, k0 + r);
}

__global__ void k_compact_rows(const int32_t* __restrict__ f, const int32_t* __restrict__ off, int32_t m,
                               int32_t* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m && f[i]) out[off[i]] = (int32_t)i;
}

int csr5_convert(spmv_handle* h, const spmv_csr* c, cudaStream_t s) {
    const int32_t m = c->m;
    if (h->params.csr5_omega != 0 && h->params.csr5_omega != 32)
        return set_error(SPMV_ERR_INVALID_ARG, "csr5_omega must be 32, the warp width (got %d)", h->params.csr5_omega);
    const int32_t sigma = h->params.csr5_sigma ? h->params.csr5_sigma : 32;
    if (sigma < 1 || sigma > 32) return set_error(SPMV_ERR_INVALID_ARG, "csr5_sigma must be in [1, 32] (got %d)", sigma);
    h->params.csr5_omega = 32;
    h->params.csr5_sigma = sigma;
    h->csr5_sigma = sigma;
    const int64_t S = 32LL * sigma;
    const int64_t nt = ceil_div(c->nnz, S);
    h->ntiles = nt;
    const int64_t bytes = nt * S * 12 + nt * (32 * 8 + 8 + 8) + (int64_t)m * 8;
    const int64_t cap = resolve_cap(h->params);
    if (bytes > cap) return set_error(SPMV_ERR_TOO_LARGE, "CSR5 needs %lld bytes, cap %lld", (long long)bytes, (long long)cap);
    SPMV_TRY(h->alloc(&h->ptr, (size_t)m + 1, "ptr"));
    SPMV_CUDA(cudaMemcpyAsync(h->ptr, c->ptr, sizeof(int32_t) * ((size_t)m + 1), cudaMemcpyDeviceToDevice, s));
    SPMV_TRY(h->alloc(&h->tile_ptr, (size_t)nt + 1, "tile_ptr"));
    SPMV_TRY(h->alloc(&h->flags, (size_t)nt * 32, "flags"));
    SPMV_TRY(h->alloc(&h->y_off, (size_t)nt * 32, "y_off"));
    SPMV_TRY(h->alloc(&h->seg_off, (size_t)nt, "seg_off"));
    SPMV_TRY(h->alloc(&h->tile_idx, (size_t)(nt * S), "tile_idx"));
    SPMV_TRY(h->alloc(&h->tile_val, (size_t)(nt * S), "tile_val"));
    SPMV_TRY(h->alloc(&h->slot_head, (size_t)nt, nullptr));
    SPMV_TRY(h->alloc(&h->slot_tail, (size_t)nt, nullptr));
    SPMV_TRY(h->alloc(&h->join_cnt, (size_t)nt, nullptr));
    if (nt > 0) SPMV_CUDA(cudaMemsetAsync(h->join_cnt, 0, sizeof(unsigned) * (size_t)nt, s));
    SPMV_TRY(h->alloc(&h->empty_ptr, (size_t)nt + 1, "empty_ptr"));
    Scratch tmp;
    int32_t *nflag = nullptr, *E = nullptr, *cnt = nullptr, *zoff = nullptr;
    SPMV_TRY(tmp.get(&nflag, (size_t)nt + 1));
    SPMV_TRY(tmp.get(&E, (size_t)m + 2));
    SPMV_TRY(tmp.get(&zoff, (size_t)m + 2));
    SPMV_TRY(tmp.get(&cnt, (size_t)nt + 1));
    k_tile_ptr<<<grid_for(nt + 1, 256), 256, 0, s>>>(c->ptr, m, c->nnz, nt, S, h->tile_ptr);
    if (nt > 0) {
        k_flags<<<grid_for(nt * 32, 256), 256, 0, s>>>(c->ptr, m, c->nnz, nt, sigma, h->flags);
        k_desc<<<grid_for(nt * 32, 256), 256, 0, s>>>(h->flags, nt, h->y_off, h->seg_off, nflag);
        int g = grid_capped(nt * S, 256, 64);
        k_tiles<<<g, 256, 0, s>>>(c->idx, c->val, c->nnz, nt, sigma, h->tile_idx, h->tile_val);
    }
    // empty rows: flags, prefix counts, and the rows listed per tile
    k_empty_flag<<<grid_for((int64_t)m + 1, 256), 256, 0, s>>>(c->ptr, m, E);
    SPMV_CUDA(cudaGetLastError());
    int32_t* eflag = nullptr;
    SPMV_TRY(tmp.get(&eflag, (size_t)m + 1));
    SPMV_CUDA(cudaMemcpyAsync(eflag, E, sizeof(int32_t) * ((size_t)m + 1), cudaMemcpyDeviceToDevice, s));
    SPMV_TRY(exclusive_scan<int32_t>(eflag, zoff, (int64_t)m + 1, s, tmp));  // zoff[i] = empty rows before i
    k_listed<<<grid_for(nt + 1, 256), 256, 0, s>>>(c->ptr, m, c->nnz, nt, S, h->tile_ptr, zoff, nflag, cnt);
    SPMV_CUDA(cudaGetLastError());
    SPMV_TRY(exclusive_scan<int32_t>(cnt, h->empty_ptr, nt, s, tmp));
    int32_t nlisted = 0, nzero = 0;
    SPMV_CUDA(cudaMemcpyAsync(&nlisted, h->empty_ptr + nt, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA(cudaMemcpyAsync(&nzero, zoff + m, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA(cudaStreamSynchronize(s));
    SPMV_TRY(h->alloc(&h->empty_rows, (size_t)(nlisted > 0 ? nlisted : 1), "empty_rows"));
    h->arrays["empty_rows"].count = nlisted;
    if (nlisted > 0)
        k_list_rows<<<grid_for(nt * 32, 256), 256, 0, s>>>(c->ptr, m, c->nnz, nt, sigma, h->flags, h->y_off,
                                                            h->empty_ptr, h->empty_rows);
    h->n_zero_rows = nzero;
    SPMV_TRY(h->alloc(&h->zero_rows, (size_t)(nzero > 0 ? nzero : 1), "zero_rows"));
    h->arrays["zero_rows"].count = nzero;
    if (nzero > 0) k_compact_rows<<<grid_for(m, 256), 256, 0, s>>>(eflag, zoff, m, h->zero_rows);
    SPMV_CUDA(cudaGetLastError());
    SPMV_CUDA(cudaStreamSynchronize(s));
    h->stored_slots = nt * S;
    h->aux[0] = nt;
    h->aux[1] = nlisted;
    h->aux[2] = nzero;
    return SPMV_OK;
}

__global__ void __launch_bounds__(256) k_csr5(dev::Csr5Args a) {
    dev::pdl_wait();  // launched early (launch_pdl): wait for the kernel ahead
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t < a.ntiles) dev::csr5_tile(a, t, threadIdx.x & 31);
}

__global__ void __launch_bounds__(256) k_csr5_zero(dev::Csr5Args a) {
    dev::pdl_wait();
    dev::csr5_zero_all(a, blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
}

dev::Csr5Args csr5_args(const spmv_handle* h, const double* x, double* y) {
    return dev::Csr5Args{h->ptr, h->tile_ptr, h->flags, h->tile_idx, h->tile_val, h->empty_ptr, h->empty_rows,
                         h->slot_head, h->slot_tail, h->join_cnt, h->zero_rows, h->n_zero_rows, h->nnz, h->ntiles,
                         h->csr5_sigma, x, y};
}

int csr5_run(const spmv_handle* h, const double* x, double* y, cudaStream_t s) {
    const dev::Csr5Args a = csr5_args(h, x, y);
    if (h->ntiles > 0) launch_pdl(k_csr5, dim3(grid_for(h->ntiles * 32, 256)), dim3(256), 0, s, a);
    else if (h->n_zero_rows > 0) launch_pdl(k_csr5_zero, dim3(grid_for(h->n_zero_rows, 256)), dim3(256), 0, s, a);
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

__global__ void k_untile(const int32_t* __restrict__ tidx, const double* __restrict__ tval, int64_t nnz, int32_t sigma,
                         int32_t* __restrict__ idx, double* __restrict__ val) {
    const int64_t S = 32LL * sigma;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = k / S, w = k % S, c = w / sigma, r = w % sigma;
        const int64_t slot = t * S + r * 32 + c;
        idx[k] = tidx[slot];
        val[k] = tval[slot];
    }
}

int csr5_to_csr(const spmv_handle* h, int32_t* ptr, int32_t* idx, double* val, cudaStream_t s) {
    SPMV_CUDA(cudaMemcpyAsync(ptr, h->ptr, sizeof(int32_t) * ((size_t)h->m + 1), cudaMemcpyDeviceToDevice, s));
    if (h->nnz > 0) {
        int g = grid_capped(h->nnz, 256, 64);
        k_untile<<<g, 256, 0, s>>>(h->tile_idx, h->tile_val, h->nnz, h->csr5_sigma, idx, val);
    }
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

}  // namespace spmv
