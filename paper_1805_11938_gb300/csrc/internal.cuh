// Internal host-side declarations of the SpMV library (not part of the ABI).
#pragma once

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/spmv.h"
#include "kernels.cuh"

namespace spmv {

constexpr int kThreads = 256;      // block size of the SpMV kernels
constexpr int kEllLongRow = 64;    // ELL rows longer than this go to the warp-per-row kernel
constexpr int kSellUnitWidth = 64;   // SELL slices wider than this are split over several warps
constexpr int kCsr5Omega = 32;     // CSR5 tile width = warp width

int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);
#define SPMV_CUDA(call)                                         \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return ::spmv::cuda_error(e_, #call); \
    } while (0)
#define SPMV_TRY(call)                    \
    do {                                  \
        int s_ = (call);                  \
        if (s_ != SPMV_OK) return s_;     \
    } while (0)

// Device allocation with the test hook of spmv_debug_fail_alloc.
int dev_malloc(void** p, size_t bytes);
void dev_free(void* p);

// Temporaries of one call, freed when the object goes out of scope (after the
// call has synchronised its stream).
struct Scratch {
    std::vector<void*> ptrs;
    template <class T>
    int get(T** p, size_t count) {
        void* q = nullptr;
        SPMV_TRY(dev_malloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16));
        ptrs.push_back(q);
        *p = static_cast<T*>(q);
        return SPMV_OK;
    }
    ~Scratch() {
        for (void* q : ptrs) dev_free(q);
    }
};

struct NamedArray {
    const void* ptr;
    int64_t count;
    int32_t elem_bytes;
};

// CSR nonzero tiles (also used for the HYB COO tail): n tiles of kCsrW
// nonzeros, tile_row[u] = first row starting at or after u*kCsrW.
struct CsrTiles {
    int32_t* tile_row = nullptr;  // n + 1 entries
    int32_t n = 0;
    int32_t rows = 0;
    int64_t nnz = 0;
    int32_t grid = 0;             // persistent grid of the tile kernel
    double* slot_head = nullptr;  // per tile, for rows crossing tiles
    double* slot_tail = nullptr;
    unsigned* cnt = nullptr;
};

struct EllPart {  // column-major ELL: slot s of row i at s*ld + i
    int32_t K = 0;
    int64_t ld = 0;
    int32_t* row_len = nullptr;  // ld entries (zero padded)
    int32_t* col = nullptr;
    double* val = nullptr;
    int32_t* long_rows = nullptr;  // rows longer than kEllLongRow
    int32_t n_long = 0;
};

}  // namespace spmv

struct spmv_handle {
    int32_t fmt = 0, m = 0, n = 0;
    int64_t nnz = 0;
    spmv_params params{};
    int64_t device_bytes = 0;
    int64_t stored_slots = 0;
    int64_t aux[4] = {0, 0, 0, 0};
    int device = 0;
    std::vector<void*> owned;
    std::map<std::string, spmv::NamedArray> arrays;

    // CSR (also the kept ptr of CSR5)
    int32_t* ptr = nullptr;
    int32_t* idx = nullptr;
    double* val = nullptr;
    spmv::CsrTiles cu;
    int32_t csr_lanes = 0;  // CSR product: 0 = warp tiles, V = V lanes per row

    // CSR5
    int32_t csr5_sigma = 0;
    int64_t ntiles = 0;
    int32_t* tile_ptr = nullptr;
    uint32_t* flags = nullptr;  // per (tile, lane): bit r = slot (r, lane) starts a segment
    int32_t* y_off = nullptr;
    uint32_t* seg_off = nullptr;  // per tile: bit c = lane c holds no flagged slot
    int32_t* tile_idx = nullptr;
    double* tile_val = nullptr;
    int32_t* empty_ptr = nullptr;
    int32_t* empty_rows = nullptr;
    int32_t* zero_rows = nullptr;  // the matrix's empty rows (y = 0)
    int32_t n_zero_rows = 0;
    double* slot_head = nullptr;  // per tile: its part of a row begun in an earlier tile
    double* slot_tail = nullptr;  // per tile: its open last segment
    unsigned* join_cnt = nullptr; // per start tile: tickets of the row's tiles (reset after use)

    // ELL and the ELL part of HYB
    spmv::EllPart ell;

    // SELL-C-sigma
    int32_t sell_C = 32, sell_sigma = 1;
    int64_t n_slices = 0;
    int64_t* slice_ptr = nullptr;
    int32_t* perm = nullptr;
    int32_t* sell_len = nullptr;  // per sorted position, padded to a multiple of C
    int32_t* sell_col = nullptr;
    double* sell_val = nullptr;
    int2* sell_units = nullptr;   // {slice, chunk or -1}, n_sell_units + 1 entries
    int32_t n_sell_units = 0;
    double* sell_partial = nullptr;
    unsigned* sell_counters = nullptr;
    // SELL column panels: panel p covers columns [p*panel_cols, (p+1)*panel_cols)
    // and is a SELL handle of its own; all panels share the parent's row order
    // (perm, owned by the parent), and sell_ys holds the partial sums per
    // sorted position between panels; after the last panel, y[i] =
    // sell_ys[sell_ipos[i]] (rows in order, whole sectors written).  panel_pos[p][j] is the CSR position of
    // its entry j (for the way back).  ptr keeps the CSR row pointers.
    double* sell_ys = nullptr;
    int32_t* sell_ipos = nullptr;  // panels: row -> sorted position (the inverse of perm)
    bool sell_ident = false;       // one panel whose sort moved no row: y written without perm
    int32_t panel_cols = 0;
    std::vector<spmv_handle*> panels;
    std::vector<int32_t*> panel_pos;

    // HYB COO tail, grouped by row: tail row r_t = tail_rows[t], entries tail_ptr[t]..tail_ptr[t+1]
    int64_t n_tail = 0;
    int32_t n_tail_rows = 0;
    int32_t* tail_rows = nullptr;
    int32_t* tail_ptr = nullptr;
    int32_t* tail_col = nullptr;
    double* tail_val = nullptr;
    spmv::CsrTiles tail_units;

    template <class T>
    int alloc(T** p, size_t count, const char* name) {
        void* q = nullptr;
        size_t bytes = count * sizeof(T);
        SPMV_TRY(spmv::dev_malloc(&q, bytes > 0 ? bytes : 16));
        owned.push_back(q);
        device_bytes += (int64_t)bytes;
        *p = static_cast<T*>(q);
        if (name) arrays[name] = spmv::NamedArray{q, (int64_t)count, (int32_t)sizeof(T)};
        return SPMV_OK;
    }
    ~spmv_handle() {
        for (spmv_handle* c : panels) delete c;
        for (void* q : owned) spmv::dev_free(q);
    }
};

namespace spmv {

// ---- shared host helpers (common.cu)
int validate_csr(const spmv_csr* c, cudaStream_t s);
template <class T>
int exclusive_scan(const T* in, T* out, int64_t n, cudaStream_t s, Scratch& tmp);  // out[n] = total
int row_lengths(const int32_t* ptr, int32_t m, int32_t* len, cudaStream_t s);
int max_i32(const int32_t* a, int64_t n, int32_t* result_host, cudaStream_t s, Scratch& tmp);
int copy_csr(spmv_handle* h, const spmv_csr* c, cudaStream_t s);
int64_t resolve_cap(const spmv_params& p);
// Nonzero tiles over the CSR arrays (ptr, rows, nnz).
int build_csr_tiles(spmv_handle* h, CsrTiles& ct, const int32_t* ptr, int32_t rows, int64_t nnz, const char* prefix,
                    cudaStream_t s);

// ---- per-format conversion and launch
int csr_convert(spmv_handle* h, const spmv_csr* c, cudaStream_t s);
int csr_run(const spmv_handle* h, const double* x, double* y, cudaStream_t s);
dev::CsrArgs csr_tile_args(const CsrTiles& ct, const int32_t* ptr, const int32_t* idx, const double* val,
                           const int32_t* row_map, const double* x, double* y);
int csr_tiles_launch(const CsrTiles& ct, const int32_t* ptr, const int32_t* idx, const double* val,
                     const int32_t* row_map, const double* x, double* y, bool add, cudaStream_t s);
// Opens the tile kernels' dynamic shared memory and sizes their persistent grid.
int csr_prepare(CsrTiles& ct);

int csr5_convert(spmv_handle* h, const spmv_csr* c, cudaStream_t s);
int csr5_run(const spmv_handle* h, const double* x, double* y, cudaStream_t s);
int csr5_to_csr(const spmv_handle* h, int32_t* ptr, int32_t* idx, double* val, cudaStream_t s);

int ell_build(spmv_handle* h, EllPart& e, const spmv_csr* c, int32_t K, const int32_t* len, bool hyb,
              cudaStream_t s);
int ell_convert(spmv_handle* h, const spmv_csr* c, cudaStream_t s);
int ell_launch(const EllPart& e, int32_t m, int32_t long_len, const double* x, double* y, cudaStream_t s);
int ell_run(const spmv_handle* h, const double* x, double* y, cudaStream_t s);
int ell_to_csr(const spmv_handle* h, int32_t* ptr, int32_t* idx, double* val, cudaStream_t s);

int sell_convert(spmv_handle* h, const spmv_csr* c, cudaStream_t s);
int sell_run(const spmv_handle* h, const double* x, double* y, cudaStream_t s);
int sell_to_csr(const spmv_handle* h, int32_t* ptr, int32_t* idx, double* val, cudaStream_t s);

int hyb_convert(spmv_handle* h, const spmv_csr* c, cudaStream_t s);
int hyb_run(const spmv_handle* h, const double* x, double* y, cudaStream_t s);
int hyb_to_csr(const spmv_handle* h, int32_t* ptr, int32_t* idx, double* val, cudaStream_t s);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int grid_for(int64_t n, int per_block) {
    int64_t g = ceil_div(n, per_block);
    return (int)(g < 1 ? 1 : (g > 0x7fffffff ? 0x7fffffff : g));
}

// Streaming multiprocessors of the current device (queried once per device).
int sm_count();

// grid_for, capped at blocks_per_sm blocks per SM of the current device (for
// grid-stride kernels, whose blocks loop over the rest).
inline int grid_capped(int64_t n, int per_block, int blocks_per_sm) {
    const int g = grid_for(n, per_block);
    const int cap = sm_count() * blocks_per_sm;
    return g < cap ? g : cap;
}

// Launch with programmatic stream serialization: the kernel's blocks may get
// resident while the kernel ahead of it in the stream is still finishing
// (that kernel lets them in with dev::pdl_trigger(), or simply by ending).
// Every kernel launched this way calls dev::pdl_wait() before it touches
// memory, which returns once the kernel ahead has completed and its writes
// are visible, so stream order is kept.
template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

}  // namespace spmv
