// Batched SpMV: many independent products y_b = A_b x_b, each matrix in its
// own format, in one CUDA graph of persistent launches, one per task family
// present in the batch:
//     memset(counters) -> CSR5 / ELL / zero-row tasks -> SELL tasks (one
//     launch per slice height C = 32, 64, 128) -> CSR tiles -> HYB tails
// Each family gets a kernel of its own so that it keeps the register budget
// and occupancy of the format's own kernel (SELL: 8 blocks per SM at C = 32)
// instead of the worst case of all families; the CSR tile tasks (CSR
// matrices and HYB COO tails) stage their nonzeros in shared memory, which
// only their kernel reserves (the others leave the SM's storage to L1, where
// the small x vectors of the batch stay cached).  The HYB tails add into y
// after the ELL part of their matrix is written, so they come last.
//
// The work lists are built once on the host from the handles' unit counts:
// task = {matrix, kind, index}.  Each launch is a grid of (SMs x resident
// blocks) 256-thread blocks that take tasks from an atomic counter until the
// list is exhausted (no block ever waits on another).  run uploads the x/y
// pointer tables when they change and replays the graph.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "kernels.cuh"

namespace spmv {

enum TaskKind : int32_t {
    T_CSR = 0,       // 8 CSR tiles (warp each)
    T_CSR5 = 1,      // 8 CSR5 tiles (warp each)
    T_ELL = 2,       // 512 ELL rows
    T_ELL_LONG = 3,  // one long ELL row
    T_SELL = 4,      // 8 SELL units (warp each)
    T_CSR5_ZERO = 5, // 256 empty rows of a CSR5 matrix without nonzeros
    T_HYB_TAIL = 6,  // 8 HYB tail tiles, adding into y
    T_CSR_ZERO = 7,  // 256 rows of a CSR matrix without nonzeros
    T_CSR_LANES = 8  // 256 / V rows of a CSR matrix on the lanes-per-row path
};

struct MatDesc {
    int32_t fmt, sell_r;
    int32_t csr_lanes;  // CSR: V lanes per row, 0 for the tiles
    int32_t ell_nb;
    const int32_t* long_rows;
    dev::CsrArgs csr;   // CSR, or the HYB tail (ADD)
    dev::Csr5Args csr5;
    dev::EllArgs ell;   // ELL, or the ELL part of HYB
    dev::SellArgs sell;
};

struct BatchDev {
    const MatDesc* mats;
    const int4* tasks;
    int32_t n_tasks;
    unsigned* counter;
    const double* const* xs;
    double* const* ys;
};

// Task families, one kernel each (the list index in spmv_batch).
enum Family : int { F_OTHER = 0, F_SELL1 = 1, F_SELL2 = 2, F_SELL4 = 3, F_CSR = 4, F_TAIL = 5, F_COUNT = 6 };

template <int FAM>
__global__ void __launch_bounds__(256, FAM == F_SELL1 ? 8 : (FAM == F_SELL2 ? 5 : 4)) k_batch(BatchDev B) {
    extern __shared__ __align__(16) unsigned char batch_smem[];
    dev::CsrWarpSmem* S = reinterpret_cast<dev::CsrWarpSmem*>(batch_smem);  // CSR tiles: one slice per warp
    __shared__ double red[8];
    __shared__ int task_sh;
    if constexpr (FAM == F_CSR || FAM == F_TAIL) {
        // CSR tiles: warp-sized items (task, tile), each warp taking every
        // (grid x 8)-th, with no counter and no block barrier (tiles hold
        // equal numbers of nonzeros, so the static split is balanced;
        // measured on the 512-matrix batch in CSR: 7.24 -> 6.17 ms)
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int64_t n_items = (int64_t)B.n_tasks * 8;
        for (int64_t it = (int64_t)blockIdx.x * 8 + warp; it < n_items; it += (int64_t)gridDim.x * 8) {
            const int4 t = B.tasks[it >> 3];
            const int32_t u = t.z * 8 + (int32_t)(it & 7);
            dev::CsrArgs a = B.mats[t.x].csr;
            if (u < a.ntiles) {
                a.x = B.xs[t.x];
                a.y = B.ys[t.x];
                dev::csr_tile<FAM == F_TAIL>(a, u, S[warp], lane);
            }
        }
    } else {
        // the other families take tasks of 8 units from a counter (SELL units are
        // often a few dozen gathers: one descriptor read per 8 of them; measured
        // on the 512-matrix batch in SELL: 4.20 ms against 4.81 striding units)
        for (;;) {
            if (threadIdx.x == 0) task_sh = (int)atomicAdd(B.counter, 1u);
            __syncthreads();
            const int ti = task_sh;
            __syncthreads();
            if (ti >= B.n_tasks) break;
            const int4 t = B.tasks[ti];
            const MatDesc& md = B.mats[t.x];
            const double* x = B.xs[t.x];
            double* y = B.ys[t.x];
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            if constexpr (FAM == F_SELL1 || FAM == F_SELL2 || FAM == F_SELL4) {
                constexpr int R = FAM == F_SELL1 ? 1 : (FAM == F_SELL2 ? 2 : 4);
                dev::SellArgs a = md.sell;
                a.x = x;
                a.y = y;
                const int32_t u = t.z * 8 + warp;
                if (u < t.w) dev::sell_unit<R>(a, u, lane);
            } else {
                switch (t.y) {
                    case T_CSR_ZERO: {
                        dev::CsrArgs a = md.csr;
                        a.x = x;
                        a.y = y;
                        dev::csr_zero(a, (int64_t)t.z * 256 + threadIdx.x);
                        break;
                    }
                    case T_CSR_LANES: {  // the same arithmetic as the standalone lanes kernel
                        const dev::CsrArgs& c = md.csr;
                        const int64_t row0 = (int64_t)t.z * (256 / md.csr_lanes);
                        switch (md.csr_lanes) {
                            case 2: dev::csr_lanes_row<2>(c.ptr, c.idx, c.val, x, y, c.rows, row0 + threadIdx.x / 2, threadIdx.x & 1); break;
                            case 4: dev::csr_lanes_row<4>(c.ptr, c.idx, c.val, x, y, c.rows, row0 + threadIdx.x / 4, threadIdx.x & 3); break;
                            case 8: dev::csr_lanes_row<8>(c.ptr, c.idx, c.val, x, y, c.rows, row0 + threadIdx.x / 8, threadIdx.x & 7); break;
                            case 16: dev::csr_lanes_row<16>(c.ptr, c.idx, c.val, x, y, c.rows, row0 + threadIdx.x / 16, threadIdx.x & 15); break;
                            default: dev::csr_lanes_row<32>(c.ptr, c.idx, c.val, x, y, c.rows, row0 + threadIdx.x / 32, threadIdx.x & 31); break;
                        }
                        break;
                    }
                    case T_CSR5: {
                        dev::Csr5Args a = md.csr5;
                        a.x = x;
                        a.y = y;
                        const int64_t tile = (int64_t)t.z * 8 + warp;
                        if (tile < a.ntiles) dev::csr5_tile(a, tile, lane);
                        break;
                    }
                    case T_CSR5_ZERO: {
                        dev::Csr5Args a = md.csr5;
                        a.x = x;
                        a.y = y;
                        dev::csr5_zero_all(a, (int64_t)t.z * 256 + threadIdx.x);
                        break;
                    }
                    case T_ELL: {
                        dev::EllArgs a = md.ell;
                        a.x = x;
                        a.y = y;
                        dev::ell_rows2(a, t.z * 512 + threadIdx.x * 2);
                        break;
                    }
                    case T_ELL_LONG: {
                        dev::EllArgs a = md.ell;
                        a.x = x;
                        a.y = y;
                        dev::ell_long_row(a, md.long_rows[t.z], red);
                        break;
                    }
                    default: break;
                }
            }
        }
    }
}

constexpr int kBatchAllMinBlocks = 4;

// One launch for every task of the batch but the HYB tails (SPMV_BATCH_ONE_LAUNCH):
// blocks take tasks of 8 warp units (or 256 rows) from one counter, whatever
// their format; SELL tasks pick their slice height at run time, CSR tile tasks
// stage their nonzeros in the dynamic shared memory the launch then reserves.
// The register budget is the largest family's (C = 128 SELL), MINB blocks per SM.
template <int MINB>
__global__ void __launch_bounds__(256, MINB) k_batch_all(BatchDev B) {
    extern __shared__ __align__(16) unsigned char batch_smem[];
    dev::CsrWarpSmem* S = reinterpret_cast<dev::CsrWarpSmem*>(batch_smem);
    __shared__ double red[8];
    __shared__ int task_sh;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) task_sh = (int)atomicAdd(B.counter, 1u);
        __syncthreads();
        const int ti = task_sh;
        __syncthreads();
        if (ti >= B.n_tasks) break;
        const int4 t = B.tasks[ti];
        const MatDesc& md = B.mats[t.x];
        const double* x = B.xs[t.x];
        double* y = B.ys[t.x];
        switch (t.y) {
            case T_SELL: {
                dev::SellArgs a = md.sell;
                a.x = x;
                a.y = y;
                const int32_t u = t.z * 8 + warp;
                if (u < t.w) {
                    if (md.sell_r == 1) dev::sell_unit<1>(a, u, lane);
                    else if (md.sell_r == 2) dev::sell_unit<2>(a, u, lane);
                    else dev::sell_unit<4>(a, u, lane);
                }
                break;
            }
            case T_CSR: {
                dev::CsrArgs a = md.csr;
                const int32_t u = t.z * 8 + warp;
                if (u < a.ntiles) {
                    a.x = x;
                    a.y = y;
                    dev::csr_tile<false>(a, u, S[warp], lane);
                }
                break;
            }
            case T_CSR_ZERO: {
                dev::CsrArgs a = md.csr;
                a.x = x;
                a.y = y;
                dev::csr_zero(a, (int64_t)t.z * 256 + threadIdx.x);
                break;
            }
            case T_CSR_LANES: {
                const dev::CsrArgs& c = md.csr;
                const int64_t row0 = (int64_t)t.z * (256 / md.csr_lanes);
                switch (md.csr_lanes) {
                    case 2: dev::csr_lanes_row<2>(c.ptr, c.idx, c.val, x, y, c.rows, row0 + threadIdx.x / 2, threadIdx.x & 1); break;
                    case 4: dev::csr_lanes_row<4>(c.ptr, c.idx, c.val, x, y, c.rows, row0 + threadIdx.x / 4, threadIdx.x & 3); break;
                    case 8: dev::csr_lanes_row<8>(c.ptr, c.idx, c.val, x, y, c.rows, row0 + threadIdx.x / 8, threadIdx.x & 7); break;
                    case 16: dev::csr_lanes_row<16>(c.ptr, c.idx, c.val, x, y, c.rows, row0 + threadIdx.x / 16, threadIdx.x & 15); break;
                    default: dev::csr_lanes_row<32>(c.ptr, c.idx, c.val, x, y, c.rows, row0 + threadIdx.x / 32, threadIdx.x & 31); break;
                }
                break;
            }
            case T_CSR5: {
                dev::Csr5Args a = md.csr5;
                a.x = x;
                a.y = y;
                const int64_t tile = (int64_t)t.z * 8 + warp;
                if (tile < a.ntiles) dev::csr5_tile(a, tile, lane);
                break;
            }
            case T_CSR5_ZERO: {
                dev::Csr5Args a = md.csr5;
                a.x = x;
                a.y = y;
                dev::csr5_zero_all(a, (int64_t)t.z * 256 + threadIdx.x);
                break;
            }
            case T_ELL: {
                dev::EllArgs a = md.ell;
                a.x = x;
                a.y = y;
                dev::ell_rows2(a, t.z * 512 + threadIdx.x * 2);
                break;
            }
            case T_ELL_LONG: {
                dev::EllArgs a = md.ell;
                a.x = x;
                a.y = y;
                dev::ell_long_row(a, md.long_rows[t.z], red);
                break;
            }
            default: break;
        }
    }
}

}  // namespace spmv

struct spmv_batch {
    int32_t count = 0;
    int32_t flags = 0;
    bool csr_smem = false;  // one launch: CSR tile tasks present, the launch reserves their shared memory
    std::vector<spmv_handle*> handles;
    spmv::MatDesc* d_mats = nullptr;
    int4* d_tasks[spmv::F_COUNT] = {};  // one work list per task family
    int32_t n_tasks[spmv::F_COUNT] = {};
    int grid[spmv::F_COUNT] = {};
    unsigned* d_counters = nullptr;  // F_COUNT
    const double** d_xs = nullptr;
    double** d_ys = nullptr;
    std::vector<const double*> xs;
    std::vector<double*> ys;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphExec_t exec_sep = nullptr;
    std::vector<const double*> sep_xs;
    std::vector<double*> sep_ys;
    ~spmv_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (exec_sep) cudaGraphExecDestroy(exec_sep);
        if (cap) cudaStreamDestroy(cap);
        spmv::dev_free(d_mats);
        for (int i = 0; i < spmv::F_COUNT; ++i) spmv::dev_free(d_tasks[i]);
        spmv::dev_free(d_counters);
        spmv::dev_free(d_xs);
        spmv::dev_free(d_ys);
    }
};

namespace spmv {

dev::Csr5Args csr5_args(const spmv_handle* h, const double* x, double* y);

// Appends matrix b's tasks to the lists of their families.
static void fill_desc(const spmv_handle* h, MatDesc& d, std::vector<int4>* L, int32_t b) {
    std::vector<int4>& t1 = L[F_OTHER];
    std::vector<int4>& tc = L[F_CSR];
    std::vector<int4>& t2 = L[F_TAIL];
    memset(&d, 0, sizeof d);
    d.fmt = h->fmt;
    switch (h->fmt) {
        case SPMV_CSR:
            d.csr = csr_tile_args(h->cu, h->ptr, h->idx, h->val, nullptr, nullptr, nullptr);
            d.csr_lanes = h->csr_lanes;
            if (h->csr_lanes > 0) {  // the handle's own path, so the batch gives the same bits
                for (int64_t g = 0; g < ceil_div(h->m, 256 / h->csr_lanes); ++g)
                    t1.push_back(make_int4(b, T_CSR_LANES, (int32_t)g, 0));
                break;
            }
            for (int64_t g = 0; g < ceil_div(h->cu.n, 8); ++g) tc.push_back(make_int4(b, T_CSR, (int32_t)g, 0));
            if (h->cu.n == 0)
                for (int64_t g = 0; g < ceil_div(h->m, 256); ++g) t1.push_back(make_int4(b, T_CSR_ZERO, (int32_t)g, 0));
            break;
        case SPMV_CSR5: {
            d.csr5 = csr5_args(h, nullptr, nullptr);
            const int64_t g1 = ceil_div(h->ntiles, 8);
            for (int64_t g = 0; g < g1; ++g) t1.push_back(make_int4(b, T_CSR5, (int32_t)g, 0));
            if (h->ntiles == 0)
                for (int64_t g = 0; g < ceil_div(h->n_zero_rows, 256); ++g)
                    t1.push_back(make_int4(b, T_CSR5_ZERO, (int32_t)g, 0));
            break;
        }
        case SPMV_ELL:
        case SPMV_HYB: {
            const int32_t long_len = h->fmt == SPMV_ELL ? (int32_t)h->aux[2] : 0x7fffffff;
            d.ell = dev::EllArgs{h->ell.row_len, h->ell.col, h->ell.val, h->ell.ld, h->m, long_len, nullptr, nullptr};
            d.long_rows = h->ell.long_rows;
            d.ell_nb = (int32_t)ceil_div(h->m, 512);
            for (int32_t g = 0; g < d.ell_nb; ++g) t1.push_back(make_int4(b, T_ELL, g, 0));
            if (h->fmt == SPMV_ELL)
                for (int32_t j = 0; j < h->ell.n_long; ++j) t1.push_back(make_int4(b, T_ELL_LONG, j, 0));
            if (h->fmt == SPMV_HYB && h->n_tail_rows > 0) {
                d.csr = csr_tile_args(h->tail_units, h->tail_ptr, h->tail_col, h->tail_val, h->tail_rows, nullptr,
                                      nullptr);
                for (int64_t g = 0; g < ceil_div(h->tail_units.n, 8); ++g)
                    t2.push_back(make_int4(b, T_HYB_TAIL, (int32_t)g, 0));
            }
            break;
        }
        case SPMV_SELL:
            d.sell = dev::SellArgs{h->sell_units, h->slice_ptr, h->sell_len, h->perm, h->sell_col, h->sell_val,
                                   h->sell_partial, h->sell_counters, h->m, kSellUnitWidth, nullptr, nullptr};
            d.sell_r = h->sell_C / 32;
            for (int64_t g = 0; g < ceil_div(h->n_sell_units, 8); ++g)
                L[d.sell_r == 1 ? F_SELL1 : (d.sell_r == 2 ? F_SELL2 : F_SELL4)].push_back(
                    make_int4(b, T_SELL, (int32_t)g, h->n_sell_units));
            break;
    }
}

static int capture_batch(spmv_batch* bt) {
    cudaGraph_t g = nullptr;
    SPMV_CUDA(cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(bt->d_counters, 0, F_COUNT * sizeof(unsigned), bt->cap);
    for (int i = 0; i < F_COUNT; ++i) {
        if (bt->n_tasks[i] == 0) continue;
        BatchDev a{bt->d_mats, bt->d_tasks[i], bt->n_tasks[i], bt->d_counters + i, bt->d_xs, bt->d_ys};
        const int grid = bt->grid[i];
        switch (i) {
            case F_OTHER:
                if (bt->flags & SPMV_BATCH_ONE_LAUNCH)
                    k_batch_all<kBatchAllMinBlocks><<<grid, 256, bt->csr_smem ? dev::kCsrSmemBytes : 0, bt->cap>>>(a);
                else
                    k_batch<F_OTHER><<<grid, 256, 0, bt->cap>>>(a);
                break;
            case F_SELL1: k_batch<F_SELL1><<<grid, 256, 0, bt->cap>>>(a); break;
            case F_SELL2: k_batch<F_SELL2><<<grid, 256, 0, bt->cap>>>(a); break;
            case F_SELL4: k_batch<F_SELL4><<<grid, 256, 0, bt->cap>>>(a); break;
            case F_CSR: k_batch<F_CSR><<<grid, 256, dev::kCsrSmemBytes, bt->cap>>>(a); break;
            default: k_batch<F_TAIL><<<grid, 256, dev::kCsrSmemBytes, bt->cap>>>(a); break;
        }
    }
    cudaError_t e = cudaStreamEndCapture(bt->cap, &g);
    if (e != cudaSuccess) return cuda_error(e, "batch graph capture");
    e = cudaGraphInstantiate(&bt->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_error(e, "batch graph instantiate");
    return SPMV_OK;
}

static int capture_separate(spmv_batch* bt) {
    if (bt->exec_sep) {
        cudaGraphExecDestroy(bt->exec_sep);
        bt->exec_sep = nullptr;
    }
    cudaGraph_t g = nullptr;
    SPMV_CUDA(cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal));
    int st = SPMV_OK;
    for (int32_t b = 0; b < bt->count && st == SPMV_OK; ++b)
        st = spmv_run(bt->handles[b], bt->sep_xs[b], bt->sep_ys[b], bt->cap);
    cudaError_t e = cudaStreamEndCapture(bt->cap, &g);
    if (st != SPMV_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_error(e, "separate graph capture");
    e = cudaGraphInstantiate(&bt->exec_sep, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_error(e, "separate graph instantiate");
    return SPMV_OK;
}

}  // namespace spmv

using namespace spmv;

extern "C" {

int spmv_batch_build(spmv_handle* const* handles, int32_t count, cudaStream_t stream, spmv_batch** out) {
    return spmv_batch_build_ex(handles, count, 0, stream, out);
}

int spmv_batch_build_ex(spmv_handle* const* handles, int32_t count, int32_t flags, cudaStream_t stream,
                        spmv_batch** out) {
    if (!handles || count <= 0 || !out) return set_error(SPMV_ERR_INVALID_ARG, "bad argument");
    if (flags & ~SPMV_BATCH_ONE_LAUNCH) return set_error(SPMV_ERR_INVALID_ARG, "unknown batch flags 0x%x", flags);
    *out = nullptr;
    for (int32_t b = 0; b < count; ++b) {
        if (!handles[b]) return set_error(SPMV_ERR_INVALID_ARG, "handle %d is NULL", b);
        if (!handles[b]->panels.empty())  // its panels must run one after another
            return set_error(SPMV_ERR_INVALID_ARG, "handle %d is a SELL matrix in column panels; batches take "
                             "single-panel handles (sell_panel_cols = SPMV_SELL_PANELS_NONE)", b);
    }
    spmv_batch* bt = new spmv_batch();
    bt->count = count;
    bt->flags = flags;
    bt->handles.assign(handles, handles + count);
    std::vector<MatDesc> mats(count);
    std::vector<int4> lists[F_COUNT];
    for (int32_t b = 0; b < count; ++b) fill_desc(handles[b], mats[b], lists, b);
    if (flags & SPMV_BATCH_ONE_LAUNCH) {
        // every list but the HYB tails goes to the one launch (its list: F_OTHER);
        // CSR tile items become tasks of 8 tiles, one per warp (their index is
        // already the group of 8)
        bt->csr_smem = !lists[F_CSR].empty();
        for (int i : {F_SELL1, F_SELL2, F_SELL4, F_CSR}) {
            lists[F_OTHER].insert(lists[F_OTHER].end(), lists[i].begin(), lists[i].end());
            lists[i].clear();
        }
    }
    int st = dev_malloc((void**)&bt->d_mats, sizeof(MatDesc) * count);
    for (int i = 0; i < F_COUNT; ++i) {
        bt->n_tasks[i] = (int32_t)lists[i].size();
        if (st == SPMV_OK) st = dev_malloc((void**)&bt->d_tasks[i], sizeof(int4) * (lists[i].size() + 1));
    }
    if (st == SPMV_OK) st = dev_malloc((void**)&bt->d_counters, F_COUNT * sizeof(unsigned));
    if (st == SPMV_OK) st = dev_malloc((void**)&bt->d_xs, sizeof(double*) * count);
    if (st == SPMV_OK) st = dev_malloc((void**)&bt->d_ys, sizeof(double*) * count);
    if (st != SPMV_OK) {
        delete bt;
        return st;
    }
    cudaError_t e = cudaMemcpy(bt->d_mats, mats.data(), sizeof(MatDesc) * count, cudaMemcpyHostToDevice);
    for (int i = 0; i < F_COUNT; ++i)
        if (e == cudaSuccess && !lists[i].empty())
            e = cudaMemcpy(bt->d_tasks[i], lists[i].data(), sizeof(int4) * lists[i].size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(bt->d_xs, 0, sizeof(double*) * count);
    if (e == cudaSuccess) e = cudaMemset(bt->d_ys, 0, sizeof(double*) * count);
    int dev = 0, sms = 0;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch<F_CSR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dev::kCsrSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch<F_TAIL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dev::kCsrSmemBytes);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void* kernels[F_COUNT] = {(const void*)k_batch<F_OTHER>, (const void*)k_batch<F_SELL1>,
                                    (const void*)k_batch<F_SELL2>, (const void*)k_batch<F_SELL4>,
                                    (const void*)k_batch<F_CSR>, (const void*)k_batch<F_TAIL>};
    if (flags & SPMV_BATCH_ONE_LAUNCH) {
        kernels[F_OTHER] = (const void*)k_batch_all<kBatchAllMinBlocks>;
        if (e == cudaSuccess && bt->csr_smem)
            e = cudaFuncSetAttribute(k_batch_all<kBatchAllMinBlocks>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)dev::kCsrSmemBytes);
    }
    for (int i = 0; i < F_COUNT && e == cudaSuccess; ++i) {
        int per_sm = 0;
        const size_t smem = (i == F_CSR || i == F_TAIL || (i == F_OTHER && bt->csr_smem)) ? dev::kCsrSmemBytes : 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernels[i], 256, smem);
        // the counter-driven families fill the GPU once; the warp-striding CSR tiles take four waves
        bt->grid[i] = sms * (per_sm > 0 ? per_sm : 1) * ((i == F_CSR || i == F_TAIL) ? 4 : 1);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete bt;
        return cuda_error(e, "spmv_batch_build");
    }
    bt->xs.assign(count, nullptr);
    bt->ys.assign(count, nullptr);
    st = capture_batch(bt);
    if (st != SPMV_OK) {
        delete bt;
        return st;
    }
    (void)stream;
    *out = bt;
    return SPMV_OK;
}

static int upload_vectors(spmv_batch* bt, const double* const* xs, double* const* ys, cudaStream_t stream) {
    bool same = true;
    for (int32_t b = 0; b < bt->count && same; ++b) same = bt->xs[b] == xs[b] && bt->ys[b] == ys[b];
    if (same) return SPMV_OK;
    for (int32_t b = 0; b < bt->count; ++b)
        if (!xs[b] || !ys[b]) return set_error(SPMV_ERR_INVALID_ARG, "x or y of matrix %d is NULL", b);
    // The cached host tables describe what the device tables hold: forget them
    // until both copies have landed, so a failed upload is retried in full.
    std::fill(bt->xs.begin(), bt->xs.end(), nullptr);
    std::fill(bt->ys.begin(), bt->ys.end(), nullptr);
    std::vector<const double*> hx(xs, xs + bt->count);
    std::vector<double*> hy(ys, ys + bt->count);
    SPMV_CUDA(cudaMemcpyAsync(bt->d_xs, hx.data(), sizeof(double*) * bt->count, cudaMemcpyHostToDevice, stream));
    SPMV_CUDA(cudaMemcpyAsync(bt->d_ys, hy.data(), sizeof(double*) * bt->count, cudaMemcpyHostToDevice, stream));
    SPMV_CUDA(cudaStreamSynchronize(stream));  // the staging vectors go out of scope
    bt->xs.assign(hx.begin(), hx.end());
    bt->ys.assign(hy.begin(), hy.end());
    return SPMV_OK;
}

int spmv_batch_run(spmv_batch* bt, const double* const* xs, double* const* ys, cudaStream_t stream) {
    if (!bt || !xs || !ys) return set_error(SPMV_ERR_INVALID_ARG, "bad argument");
    SPMV_TRY(upload_vectors(bt, xs, ys, stream));
    SPMV_CUDA(cudaGraphLaunch(bt->exec, stream));
    return SPMV_OK;
}

int spmv_batch_run_separate(spmv_batch* bt, const double* const* xs, double* const* ys, cudaStream_t stream) {
    if (!bt || !xs || !ys) return set_error(SPMV_ERR_INVALID_ARG, "bad argument");
    bool same = bt->exec_sep != nullptr && (int32_t)bt->sep_xs.size() == bt->count;
    for (int32_t b = 0; b < bt->count && same; ++b) same = bt->sep_xs[b] == xs[b] && bt->sep_ys[b] == ys[b];
    if (!same) {
        bt->sep_xs.assign(xs, xs + bt->count);
        bt->sep_ys.assign(ys, ys + bt->count);
        const int st = capture_separate(bt);
        if (st != SPMV_OK) {  // no graph for these vectors: the next call captures again
            bt->sep_xs.clear();
            bt->sep_ys.clear();
            return st;
        }
    }
    SPMV_CUDA(cudaGraphLaunch(bt->exec_sep, stream));
    return SPMV_OK;
}

int spmv_batch_launches(const spmv_batch* bt, int32_t* out) {
    if (!bt || !out) return set_error(SPMV_ERR_INVALID_ARG, "bad argument");
    int32_t n = 0;
    for (int i = 0; i < F_COUNT; ++i) n += bt->n_tasks[i] > 0;
    *out = n;
    return SPMV_OK;
}

void spmv_batch_free(spmv_batch* bt) { delete bt; }

}  // extern "C"
