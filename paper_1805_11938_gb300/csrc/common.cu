// Shared host helpers and small device utilities: errors, allocation, CSR
// validation, exclusive scan, row lengths and the CSR nonzero tiles.
#include <atomic>
#include <cstring>
#include <mutex>

#include "internal.cuh"
#include "kernels.cuh"

namespace spmv {

static thread_local std::string g_last_error;
static std::atomic<int> g_fail_alloc_countdown{0};

int set_error(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

const char* last_error() { return g_last_error.c_str(); }
void clear_error() { g_last_error.clear(); }

int cuda_error(cudaError_t e, const char* what) {
    cudaGetLastError();  // clear a sticky-free error so the next call starts clean
    return set_error(SPMV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void debug_fail_alloc(int k) { g_fail_alloc_countdown.store(k); }

int sm_count() {
    static std::atomic<int> cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return 1;
    }
    int n = cached[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
            (void)cudaGetLastError();
            n = 1;
        }
        cached[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

int dev_malloc(void** p, size_t bytes) {
    int c = g_fail_alloc_countdown.load();
    while (c > 0) {
        if (g_fail_alloc_countdown.compare_exchange_weak(c, c - 1)) {
            if (c == 1) {
                *p = nullptr;
                return set_error(SPMV_ERR_ALLOC, "device allocation of %zu bytes failed (injected)", bytes);
            }
            break;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(SPMV_ERR_ALLOC, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    return SPMV_OK;
}

void dev_free(void* p) {
    if (p) cudaFree(p);
}

// ------------------------------------------------------------ validation

// bit 1: ptr[0] != 0 or ptr[m] != nnz; bit 2: ptr decreases; bit 4: column out of range
__global__ void k_validate_ptr(const int32_t* __restrict__ ptr, int32_t m, int64_t nnz, int* err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > m) return;
    if (i == 0 && ptr[0] != 0) atomicOr(err, 1);
    if (i == m && ptr[m] != nnz) atomicOr(err, 1);
    if (i < m && ptr[i + 1] < ptr[i]) atomicOr(err, 2);
}

__global__ void k_validate_idx(const int32_t* __restrict__ idx, int64_t nnz, int32_t n, int* err) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int bad = 0;
    for (; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = idx[k];
        bad |= (c < 0) | (c >= n);
    }
    if (__any_sync(dev::kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(err, 4);
}

int validate_csr(const spmv_csr* c, cudaStream_t s) {
    if (!c) return set_error(SPMV_ERR_INVALID_ARG, "csr is NULL");
    if (c->m <= 0 || c->n <= 0) return set_error(SPMV_ERR_INVALID_ARG, "m and n must be positive (m=%d n=%d)", c->m, c->n);
    if (c->nnz < 0) return set_error(SPMV_ERR_INVALID_ARG, "nnz must be >= 0");
    if (c->nnz > 2147483647LL) return set_error(SPMV_ERR_INDEX_OVERFLOW, "nnz %lld does not fit int32 row pointers", (long long)c->nnz);
    if (!c->ptr) return set_error(SPMV_ERR_INVALID_ARG, "csr.ptr is NULL");
    if (c->nnz > 0 && (!c->idx || !c->val)) return set_error(SPMV_ERR_INVALID_ARG, "csr.idx or csr.val is NULL");
    Scratch tmp;
    int* err = nullptr;
    SPMV_TRY(tmp.get(&err, 1));
    SPMV_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    k_validate_ptr<<<grid_for((int64_t)c->m + 1, 256), 256, 0, s>>>(c->ptr, c->m, c->nnz, err);
    if (c->nnz > 0) {
        int g = grid_capped(c->nnz, 256, 32);
        k_validate_idx<<<g, 256, 0, s>>>(c->idx, c->nnz, c->n, err);
    }
    SPMV_CUDA(cudaGetLastError());
    int h = 0;
    SPMV_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA(cudaStreamSynchronize(s));
    if (h & 1) return set_error(SPMV_ERR_INVALID_ARG, "malformed CSR: ptr[0] != 0 or ptr[m] != nnz");
    if (h & 2) return set_error(SPMV_ERR_INVALID_ARG, "malformed CSR: row pointers decrease");
    if (h & 4) return set_error(SPMV_ERR_INVALID_ARG, "malformed CSR: column index outside [0, n)");
    return SPMV_OK;
}

// ------------------------------------------------------------------ scan
//
// Exclusive scan in three passes: tile sums (2048 items per 256-thread
// block), a single-block scan of the tile sums, and a block scan of each tile
// offset by its tile's prefix.  out has n + 1 entries; out[n] is the total.

constexpr int kScanItems = 8;
constexpr int kScanTile = 256 * kScanItems;

template <class T>
__device__ __forceinline__ T block_exclusive_scan256(T v, T* sh, T* total) {
    // sh: 8 entries
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = __shfl_up_sync(dev::kFull, inc, d);
        if (l >= d) inc += o;
    }
    if (l == 31) sh[w] = inc;
    __syncthreads();
    T wpre = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i < w) wpre += sh[i];
        tot += sh[i];
    }
    __syncthreads();
    *total = tot;
    return wpre + inc - v;
}

template <class T>
__global__ void k_scan_tiles(const T* __restrict__ in, int64_t n, T* __restrict__ tile_sums) {
    __shared__ T sh[8];
    const int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += in[base + i];
    T tot;
    block_exclusive_scan256<T>(s, sh, &tot);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

template <class T>
__global__ void k_scan_sums(T* __restrict__ sums, int64_t nt, T* __restrict__ total_out) {
    __shared__ T sh[8];
    T carry = 0;
    for (int64_t b = 0; b < nt; b += kScanTile) {
        const int64_t base = b + threadIdx.x * kScanItems;
        T v[kScanItems];
        T s = 0;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            v[i] = base + i < nt ? sums[base + i] : 0;
            s += v[i];
        }
        T tot;
        T pre = block_exclusive_scan256<T>(s, sh, &tot) + carry;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            if (base + i < nt) sums[base + i] = pre;
            pre += v[i];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

template <class T>
__global__ void k_scan_apply(const T* __restrict__ in, int64_t n, const T* __restrict__ tile_pre, T* __restrict__ out) {
    __shared__ T sh[8];
    const int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    T tot;
    T pre = block_exclusive_scan256<T>(s, sh, &tot) + tile_pre[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = pre;
        pre += v[i];
    }
}

template <class T>
int exclusive_scan(const T* in, T* out, int64_t n, cudaStream_t s, Scratch& tmp) {
    const int64_t nt = ceil_div(n > 0 ? n : 1, kScanTile);
    T* sums = nullptr;
    SPMV_TRY(tmp.get(&sums, (size_t)nt));
    k_scan_tiles<T><<<(unsigned)nt, 256, 0, s>>>(in, n, sums);
    k_scan_sums<T><<<1, 256, 0, s>>>(sums, nt, out + n);
    k_scan_apply<T><<<(unsigned)nt, 256, 0, s>>>(in, n, sums, out);
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

template int exclusive_scan<int32_t>(const int32_t*, int32_t*, int64_t, cudaStream_t, Scratch&);
template int exclusive_scan<int64_t>(const int64_t*, int64_t*, int64_t, cudaStream_t, Scratch&);

// ------------------------------------------------------------ row lengths

__global__ void k_row_lengths(const int32_t* __restrict__ ptr, int32_t m, int32_t* __restrict__ len) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) len[i] = ptr[i + 1] - ptr[i];
}

int row_lengths(const int32_t* ptr, int32_t m, int32_t* len, cudaStream_t s) {
    k_row_lengths<<<grid_for(m, 256), 256, 0, s>>>(ptr, m, len);
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

__global__ void k_max_i32(const int32_t* __restrict__ a, int64_t n, int32_t* out) {
    int32_t v = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v = max(v, a[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(dev::kFull, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}

int max_i32(const int32_t* a, int64_t n, int32_t* result_host, cudaStream_t s, Scratch& tmp) {
    int32_t* d = nullptr;
    SPMV_TRY(tmp.get(&d, 1));
    SPMV_CUDA(cudaMemsetAsync(d, 0, sizeof(int32_t), s));
    int g = grid_capped(n, 256, 16);
    if (n > 0) k_max_i32<<<g, 256, 0, s>>>(a, n, d);
    SPMV_CUDA(cudaGetLastError());
    SPMV_CUDA(cudaMemcpyAsync(result_host, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA(cudaStreamSynchronize(s));
    return SPMV_OK;
}

int copy_csr(spmv_handle* h, const spmv_csr* c, cudaStream_t s) {
    SPMV_TRY(h->alloc(&h->ptr, (size_t)c->m + 1, "ptr"));
    SPMV_TRY(h->alloc(&h->idx, (size_t)c->nnz, "idx"));
    SPMV_TRY(h->alloc(&h->val, (size_t)c->nnz, "val"));
    SPMV_CUDA(cudaMemcpyAsync(h->ptr, c->ptr, sizeof(int32_t) * ((size_t)c->m + 1), cudaMemcpyDeviceToDevice, s));
    if (c->nnz > 0) {
        SPMV_CUDA(cudaMemcpyAsync(h->idx, c->idx, sizeof(int32_t) * (size_t)c->nnz, cudaMemcpyDeviceToDevice, s));
        SPMV_CUDA(cudaMemcpyAsync(h->val, c->val, sizeof(double) * (size_t)c->nnz, cudaMemcpyDeviceToDevice, s));
    }
    return SPMV_OK;
}

int64_t resolve_cap(const spmv_params& p) {
    if (p.max_bytes > 0) return p.max_bytes;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (int64_t)(0.9 * (double)fr);
}

// ------------------------------------------------------------- CSR tiles
//
// Tile u covers nonzeros [u*W, (u+1)*W); tile_row[u] is the first row whose
// pointer is at or after u*W (a lower bound over ptr[0..rows]), so the rows
// starting in tile u are tile_row[u] .. tile_row[u+1]-1.  tile_row[ntiles] =
// rows, so the last tile also takes the trailing empty rows.

__global__ void k_tile_row(const int32_t* __restrict__ ptr, int32_t rows, int32_t nt, int32_t* __restrict__ tile_row) {
    const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (u > nt) return;
    if (u == nt) {
        tile_row[nt] = rows;
        return;
    }
    const int64_t k = u * dev::kCsrW;
    int32_t lo = 0, hi = rows;  // ptr[rows] = nnz > k
    while (lo < hi) {
        const int32_t mid = lo + (hi - lo) / 2;
        if (ptr[mid] >= k) hi = mid;
        else lo = mid + 1;
    }
    tile_row[u] = lo;
}

int build_csr_tiles(spmv_handle* h, CsrTiles& ct, const int32_t* ptr, int32_t rows, int64_t nnz, const char* prefix,
                    cudaStream_t s) {
    ct.rows = rows;
    ct.nnz = nnz;
    ct.n = (int32_t)ceil_div(nnz, dev::kCsrW);
    std::string pre = prefix ? prefix : "";
    SPMV_TRY(h->alloc(&ct.tile_row, (size_t)ct.n + 1, (pre + "tile_row").c_str()));
    SPMV_TRY(h->alloc(&ct.slot_head, (size_t)ct.n + 1, nullptr));
    SPMV_TRY(h->alloc(&ct.slot_tail, (size_t)ct.n + 1, nullptr));
    SPMV_TRY(h->alloc(&ct.cnt, (size_t)ct.n + 1, nullptr));
    SPMV_CUDA(cudaMemsetAsync(ct.cnt, 0, sizeof(unsigned) * ((size_t)ct.n + 1), s));
    k_tile_row<<<grid_for((int64_t)ct.n + 1, 256), 256, 0, s>>>(ptr, rows, ct.n, ct.tile_row);
    SPMV_CUDA(cudaGetLastError());
    SPMV_CUDA(cudaStreamSynchronize(s));
    return SPMV_OK;
}

}  // namespace spmv
