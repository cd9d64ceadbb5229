// SELL-C-sigma (Sec. II-B "SELL and SELL-C-sigma"): rows are sorted by
// length, descending and stably, inside windows of sigma rows; consecutive
// groups of C sorted rows form slices, each stored as a column-major ELL of
// its own width.  sigma = 1 is plain SELL.  The product writes y[perm[p]]
// for the row at sorted position p, or y[p] directly when the sort moved no
// row (sigma = 1, or rows already in order), so that perm is not read.
//
// Conversion on the device: a stable segmented LSD radix sort (one bit per
// pass, a scan and a scatter each) orders every window by (maxlen - length);
// slice widths and their prefix sum give slice_ptr; one thread per nonzero
// scatters into the slices.
#include <algorithm>

#include "internal.cuh"
#include "kernels.cuh"

namespace spmv {

using dev::row_of_nnz;

__global__ void k_iota_keys(const int32_t* __restrict__ len, int32_t m, int32_t maxlen, uint32_t* __restrict__ key,
                            int32_t* __restrict__ row) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) {
        key[i] = (uint32_t)(maxlen - len[i]);
        row[i] = (int32_t)i;
    }
}

// Group of row i in the shared order of column panels, as a descending key:
// rows longer than long_len first (group 0), then the other rows in windows
// of `window` consecutive rows (group 1 + i / window).  g[i] = gmax - group.
__global__ void k_panel_group(const int32_t* __restrict__ ptr, int32_t m, int32_t long_len, int64_t window,
                              int32_t gmax, int32_t* __restrict__ g) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) g[i] = gmax - (ptr[i + 1] - ptr[i] > long_len ? 0 : (int32_t)(1 + i / window));
}

__global__ void k_inverse_perm(const int32_t* __restrict__ perm, int32_t m, int32_t* __restrict__ ipos) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < m) ipos[perm[p]] = (int32_t)p;
}

// key[i] = maxlen - len[rows[i]]: the next key of a multi-key sort, in the
// order the previous keys left.
__global__ void k_gather_keys(const int32_t* __restrict__ len, const int32_t* __restrict__ rows, int32_t m,
                              int32_t maxlen, uint32_t* __restrict__ key) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) key[i] = (uint32_t)(maxlen - len[rows[i]]);
}

__global__ void k_bit_zero(const uint32_t* __restrict__ key, int32_t m, int bit, int32_t* __restrict__ z) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i <= m) z[i] = (i < m) ? (int32_t)(((key[i] >> bit) & 1u) ^ 1u) : 0;
}

// Stable partition of every window [w*sigma, min(w*sigma + sigma, m)) by one
// key bit: zeros keep their order and go first, ones follow in order.
__global__ void k_bit_scatter(const uint32_t* __restrict__ key, const int32_t* __restrict__ row, int32_t m,
                              int64_t sigma, int bit, const int32_t* __restrict__ Z, uint32_t* __restrict__ key2,
                              int32_t* __restrict__ row2) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t ws = (i / sigma) * sigma;
    const int64_t we = ws + sigma < m ? ws + sigma : m;
    const int32_t zb = Z[i] - Z[ws];
    const int32_t zt = Z[we] - Z[ws];
    const uint32_t k = key[i];
    const int64_t pos = ((k >> bit) & 1u) ? ws + zt + (i - ws - zb) : ws + zb;
    key2[pos] = k;
    row2[pos] = row[i];
}

// moved: set to 1 (by every writer alike) when some row left its place
__global__ void k_sorted_len(const int32_t* __restrict__ len, const int32_t* __restrict__ perm, int32_t m,
                             int64_t mp, int32_t* __restrict__ sl, int32_t* __restrict__ ipos,
                             int32_t* __restrict__ moved) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < m) {
        const int32_t r = perm[p];
        sl[p] = len[r];
        ipos[r] = (int32_t)p;
        if (r != p) *moved = 1;
    } else if (p < mp) {
        sl[p] = 0;
    }
}

__global__ void k_slice_width(const int32_t* __restrict__ sl, int64_t ns, int32_t C, int64_t* __restrict__ cw,
                              int32_t* __restrict__ nunit, int32_t W) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s > ns) return;
    if (s == ns) {
        cw[ns] = 0;
        nunit[ns] = 0;
        return;
    }
    int32_t w = 0;
    for (int32_t l = 0; l < C; ++l) w = max(w, sl[s * C + l]);
    cw[s] = (int64_t)C * w;
    nunit[s] = w > W ? (w + W - 1) / W : 1;
}

__global__ void k_sell_units(const int64_t* __restrict__ sp, int64_t ns, int32_t C, int32_t W,
                             const int32_t* __restrict__ uoff, int2* __restrict__ units) {
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s > ns) return;
    if (s == ns) {
        units[uoff[ns]] = make_int2((int32_t)ns, -1);
        return;
    }
    const int32_t w = (int32_t)((sp[s + 1] - sp[s]) / C);
    const int32_t n = uoff[s + 1] - uoff[s];
    for (int32_t c = 0; c < n; ++c) units[uoff[s] + c] = make_int2((int32_t)s, w > W ? c : -1);
}

__global__ void k_sell_scatter(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                               const double* __restrict__ val, int32_t m, int64_t nnz, const int32_t* __restrict__ ipos,
                               const int64_t* __restrict__ sp, int32_t C, int32_t* __restrict__ col,
                               double* __restrict__ sv) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = row_of_nnz(ptr, m, k);
        const int64_t j = k - ptr[r];
        const int32_t p = ipos[r];
        const int64_t dst = sp[p / C] + j * C + (p % C);
        col[dst] = idx[k];
        sv[dst] = val[k];
    }
}

// Sorts rows stably, descending, within windows of sigma rows by the keys
// lens[0..nk) taken lexicographically (lens[0] first): one-bit LSD passes
// (a scan and a scatter each), least significant key first.  perm[pos] = row.
static int sort_rows(const int32_t* const* lens, const int32_t* maxlens, int nk, int32_t m, int64_t sigma,
                     int32_t* perm, cudaStream_t s, Scratch& tmp) {
    uint32_t *key = nullptr, *key2 = nullptr;
    int32_t *row2 = nullptr, *Z = nullptr;
    SPMV_TRY(tmp.get(&key, (size_t)m));
    SPMV_TRY(tmp.get(&key2, (size_t)m));
    SPMV_TRY(tmp.get(&row2, (size_t)m));
    SPMV_TRY(tmp.get(&Z, (size_t)m + 2));
    k_iota_keys<<<grid_for(m, 256), 256, 0, s>>>(lens[nk - 1], m, maxlens[nk - 1], key, perm);
    SPMV_CUDA(cudaGetLastError());
    if (sigma <= 1) return SPMV_OK;
    int32_t* rows_a = perm;
    uint32_t* keys_a = key;
    for (int q = nk - 1; q >= 0; --q) {
        if (q != nk - 1) k_gather_keys<<<grid_for(m, 256), 256, 0, s>>>(lens[q], rows_a, m, maxlens[q], keys_a);
        int bits = 0;
        while (bits < 32 && (maxlens[q] >> bits) != 0) ++bits;
        for (int b = 0; b < bits; ++b) {
            k_bit_zero<<<grid_for((int64_t)m + 1, 256), 256, 0, s>>>(keys_a, m, b, Z);
            SPMV_TRY(exclusive_scan<int32_t>(Z, Z, (int64_t)m + 1, s, tmp));
            k_bit_scatter<<<grid_for(m, 256), 256, 0, s>>>(keys_a, rows_a, m, sigma, b, Z, key2, row2);
            SPMV_CUDA(cudaGetLastError());
            std::swap(keys_a, key2);
            std::swap(rows_a, row2);
        }
    }
    if (rows_a != perm)
        SPMV_CUDA(cudaMemcpyAsync(perm, rows_a, sizeof(int32_t) * (size_t)m, cudaMemcpyDeviceToDevice, s));
    return SPMV_OK;
}

// Builds h's SELL layout from CSR c.  perm_in, when given, is the row order
// to use instead of sorting c's rows (the order column panels share, owned by
// the caller).
static int sell_build(spmv_handle* h, const spmv_csr* c, cudaStream_t s, int32_t* perm_in = nullptr) {
    const int32_t m = c->m;
    int32_t C = h->params.sell_C ? h->params.sell_C : 32;
    if (C != 32 && C != 64 && C != 128) return set_error(SPMV_ERR_INVALID_ARG, "sell_C must be 32, 64 or 128 (got %d)", C);
    int64_t sigma = h->params.sell_sigma ? h->params.sell_sigma : (int64_t)m;
    if (sigma == SPMV_SELL_SIGMA_ALL || sigma > m) sigma = m;
    if (sigma < 1 || (sigma != 1 && sigma != m && sigma % C != 0))
        return set_error(SPMV_ERR_INVALID_ARG, "sell_sigma must be 1, a multiple of sell_C, or -1 (got %lld)",
                         (long long)h->params.sell_sigma);
    h->params.sell_C = C;
    h->params.sell_sigma = (int32_t)sigma;
    h->sell_C = C;
    h->sell_sigma = (int32_t)sigma;
    Scratch tmp;
    int32_t *len = nullptr, *ipos = nullptr;
    SPMV_TRY(tmp.get(&len, (size_t)m + 1));
    SPMV_TRY(row_lengths(c->ptr, m, len, s));
    int32_t maxlen = 0;
    SPMV_TRY(max_i32(len, m, &maxlen, s, tmp));
    SPMV_TRY(tmp.get(&ipos, (size_t)m));
    if (perm_in) {
        h->perm = perm_in;
    } else {
        SPMV_TRY(h->alloc(&h->perm, (size_t)m, "perm"));
        const int32_t* lens[1] = {len};
        SPMV_TRY(sort_rows(lens, &maxlen, 1, m, sigma, h->perm, s, tmp));
    }
    const int64_t ns = ceil_div(m, C);
    const int64_t mp = ns * C;
    h->n_slices = ns;
    SPMV_TRY(h->alloc(&h->sell_len, (size_t)mp, "row_len"));
    int32_t* moved = nullptr;
    SPMV_TRY(tmp.get(&moved, 1));
    SPMV_CUDA(cudaMemsetAsync(moved, 0, sizeof(int32_t), s));
    k_sorted_len<<<grid_for(mp, 256), 256, 0, s>>>(len, h->perm, m, mp, h->sell_len, ipos, moved);
    int64_t* cw = nullptr;
    int32_t *nunit = nullptr, *uoff = nullptr;
    SPMV_TRY(tmp.get(&cw, (size_t)ns + 1));
    SPMV_TRY(tmp.get(&nunit, (size_t)ns + 1));
    SPMV_TRY(tmp.get(&uoff, (size_t)ns + 2));
    k_slice_width<<<grid_for(ns + 1, 256), 256, 0, s>>>(h->sell_len, ns, C, cw, nunit, kSellUnitWidth);
    SPMV_CUDA(cudaGetLastError());
    SPMV_TRY(h->alloc(&h->slice_ptr, (size_t)ns + 1, "slice_ptr"));
    SPMV_TRY(exclusive_scan<int64_t>(cw, h->slice_ptr, ns, s, tmp));
    SPMV_TRY(exclusive_scan<int32_t>(nunit, uoff, ns + 1, s, tmp));
    int64_t total = 0;
    int32_t nu = 0, moved_h = 1;
    SPMV_CUDA(cudaMemcpyAsync(&total, h->slice_ptr + ns, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA(cudaMemcpyAsync(&nu, uoff + ns, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA(cudaMemcpyAsync(&moved_h, moved, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SPMV_CUDA(cudaStreamSynchronize(s));
    // a sort that moved no row (sigma = 1, or rows already in order): the
    // product writes y at the sorted positions and never reads perm
    h->sell_ident = perm_in == nullptr && moved_h == 0;
    const int64_t bytes = total * 12 + mp * 8 + (int64_t)nu * (C * 8 + 12);
    const int64_t cap = resolve_cap(h->params);
    if (bytes > cap)
        return set_error(SPMV_ERR_TOO_LARGE, "SELL needs %lld bytes, cap %lld", (long long)bytes, (long long)cap);
    SPMV_TRY(h->alloc(&h->sell_col, (size_t)total, "col"));
    SPMV_TRY(h->alloc(&h->sell_val, (size_t)total, "val"));
    if (total > 0) {
        SPMV_CUDA(cudaMemsetAsync(h->sell_col, 0, sizeof(int32_t) * (size_t)total, s));
        SPMV_CUDA(cudaMemsetAsync(h->sell_val, 0, sizeof(double) * (size_t)total, s));
    }
    if (c->nnz > 0) {
        int g = grid_capped(c->nnz, 256, 64);
        k_sell_scatter<<<g, 256, 0, s>>>(c->ptr, c->idx, c->val, m, c->nnz, ipos, h->slice_ptr, C, h->sell_col,
                                         h->sell_val);
    }
    h->n_sell_units = nu;
    SPMV_TRY(h->alloc(&h->sell_units, (size_t)nu + 1, "units"));
    SPMV_TRY(h->alloc(&h->sell_partial, (size_t)nu * C, nullptr));
    SPMV_TRY(h->alloc(&h->sell_counters, (size_t)nu + 1, nullptr));
    SPMV_CUDA(cudaMemsetAsync(h->sell_counters, 0, sizeof(unsigned) * ((size_t)nu + 1), s));
    k_sell_units<<<grid_for(ns + 1, 256), 256, 0, s>>>(h->slice_ptr, ns, C, kSellUnitWidth, uoff, h->sell_units);
    SPMV_CUDA(cudaGetLastError());
    SPMV_CUDA(cudaStreamSynchronize(s));
    h->stored_slots = total;
    h->aux[0] = ns;
    h->aux[1] = nu;
    h->aux[2] = maxlen;
    h->aux[3] = h->sell_ident ? -1 : 0;
    return SPMV_OK;
}

// ------------------------------------------------------------- column panels
//
// x larger than about three quarters of L2 is not kept there by random
// gathers.  Splitting the matrix by columns into panels whose part of x fits
// (at most 64 MiB each) and accumulating y = sum_p A_p x_p in panel order
// trades one more read and write of y per panel for gathers that hit L2
// (the 2e7-row power-law graph: 2.8 -> about 1.8 ms).
constexpr int64_t kPanelAutoBytes = 96ll << 20;
constexpr int64_t kPanelBytes = 64ll << 20;
constexpr int32_t kPanelLongRow = 32;         // longer rows are sorted over the whole matrix
constexpr int64_t kPanelWindow = 1ll << 16;   // the other rows, in windows of this many rows (512 KiB of y)
constexpr int kPanelMax = 256;                // panels are sort keys of the shared order: a bounded number

// Entries of row i with column in [c0, c1).
__global__ void k_panel_count(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx, int32_t m, int32_t c0,
                              int32_t c1, int32_t* __restrict__ cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > m) return;
    if (i == m) {
        cnt[m] = 0;
        return;
    }
    int32_t c = 0;
    for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) c += (idx[k] >= c0 && idx[k] < c1);
    cnt[i] = c;
}

// Row i's entries of the panel, in CSR order, with local columns and their CSR positions.
__global__ void k_panel_scatter(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                const double* __restrict__ val, int32_t m, int32_t c0, int32_t c1,
                                const int32_t* __restrict__ sub_ptr, int32_t* __restrict__ sub_idx,
                                double* __restrict__ sub_val, int32_t* __restrict__ pos) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    int32_t o = sub_ptr[i];
    for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) {
        const int32_t c = idx[k];
        if (c >= c0 && c < c1) {
            sub_idx[o] = c - c0;
            sub_val[o] = val[k];
            pos[o] = k;
            ++o;
        }
    }
}

// The way back: entry j of a panel returns to CSR position pos[j].
__global__ void k_panel_unscatter(const int32_t* __restrict__ sub_idx, const double* __restrict__ sub_val,
                                  const int32_t* __restrict__ pos, int64_t nnz_p, int32_t c0, int32_t* __restrict__ idx,
                                  double* __restrict__ val) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz_p; j += (int64_t)gridDim.x * blockDim.x) {
        idx[pos[j]] = sub_idx[j] + c0;
        val[pos[j]] = sub_val[j];
    }
}

int sell_convert(spmv_handle* h, const spmv_csr* c, cudaStream_t s) {
    const int32_t n = c->n, m = c->m;
    int64_t pc = h->params.sell_panel_cols;
    if (pc < SPMV_SELL_PANELS_NONE)
        return set_error(SPMV_ERR_INVALID_ARG, "sell_panel_cols must be > 0, 0 (rule) or SPMV_SELL_PANELS_NONE (got %lld)",
                         (long long)pc);
    if (pc == 0) {
        const int64_t xb = (int64_t)n * 8;
        pc = xb > kPanelAutoBytes ? ceil_div(n, ceil_div(xb, kPanelBytes)) : n;
    } else if (pc == SPMV_SELL_PANELS_NONE || pc > n) {
        pc = n;
    }
    h->params.sell_panel_cols = (int32_t)pc;
    h->panel_cols = (int32_t)pc;
    if (pc >= n) return sell_build(h, c, s);

    // column panels: one SELL matrix per band of pc columns, all in one row
    // order, so that the partial sums stay in sorted order between panels.
    // The order: rows longer than kPanelLongRow first, then the other rows in
    // windows of kPanelWindow consecutive rows; inside each group, rows sorted
    // by their panel lengths taken lexicographically (panel 0's first), which
    // keeps every panel's slices nearly full.  The last pass writes y with
    // the rows in order (whole sectors) and reads the sums through the order;
    // the windows keep those reads within half a MiB of ys at a time, where L2
    // serves the neighbouring entries.
    const int64_t np64 = ceil_div(n, pc);
    if (np64 > kPanelMax)
        return set_error(SPMV_ERR_INVALID_ARG, "%lld column panels requested; at most %d (sell_panel_cols >= %lld)",
                         (long long)np64, kPanelMax, (long long)ceil_div(n, kPanelMax));
    const int32_t np = (int32_t)np64;
    SPMV_TRY(h->alloc(&h->ptr, (size_t)m + 1, "ptr"));
    SPMV_CUDA(cudaMemcpyAsync(h->ptr, c->ptr, sizeof(int32_t) * ((size_t)m + 1), cudaMemcpyDeviceToDevice, s));
    Scratch keep;  // per panel: its row lengths and row pointers
    std::vector<int32_t*> cnts(np), sub_ptrs(np);
    std::vector<int32_t> maxl(np), nnzs(np);
    for (int32_t p = 0; p < np; ++p) {
        const int32_t c0 = (int32_t)(p * pc), c1 = (int32_t)std::min<int64_t>(n, (int64_t)(p + 1) * pc);
        SPMV_TRY(keep.get(&cnts[p], (size_t)m + 1));
        SPMV_TRY(keep.get(&sub_ptrs[p], (size_t)m + 1));
        k_panel_count<<<grid_for((int64_t)m + 1, 256), 256, 0, s>>>(c->ptr, c->idx, m, c0, c1, cnts[p]);
        SPMV_CUDA(cudaGetLastError());
        Scratch tmp;
        SPMV_TRY(exclusive_scan<int32_t>(cnts[p], sub_ptrs[p], m, s, tmp));
        SPMV_TRY(max_i32(cnts[p], m, &maxl[p], s, tmp));
        SPMV_CUDA(cudaMemcpyAsync(&nnzs[p], sub_ptrs[p] + m, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SPMV_CUDA(cudaStreamSynchronize(s));
    }
    int64_t sigma = h->params.sell_sigma ? h->params.sell_sigma : (int64_t)m;
    if (sigma == SPMV_SELL_SIGMA_ALL || sigma > m) sigma = m;
    {
        SPMV_TRY(h->alloc(&h->perm, (size_t)m, "perm"));
        Scratch tmp;
        int32_t* grp = nullptr;
        SPMV_TRY(tmp.get(&grp, (size_t)m));
        const int64_t window = std::min<int64_t>(sigma, kPanelWindow);
        const int32_t gmax = (int32_t)(1 + (m - 1) / window);
        k_panel_group<<<grid_for(m, 256), 256, 0, s>>>(c->ptr, m, kPanelLongRow, window, gmax, grp);
        SPMV_CUDA(cudaGetLastError());
        std::vector<const int32_t*> lens{grp};
        lens.insert(lens.end(), cnts.begin(), cnts.end());
        std::vector<int32_t> maxk{gmax};
        maxk.insert(maxk.end(), maxl.begin(), maxl.end());
        // sigma = 1 (plain SELL) keeps the rows in order; otherwise one global sort by (group, panel lengths)
        SPMV_TRY(sort_rows(lens.data(), maxk.data(), np + 1, m, sigma > 1 ? m : 1, h->perm, s, tmp));
        SPMV_CUDA(cudaStreamSynchronize(s));
    }
    SPMV_TRY(h->alloc(&h->sell_ys, (size_t)m, nullptr));
    SPMV_TRY(h->alloc(&h->sell_ipos, (size_t)m, nullptr));
    k_inverse_perm<<<grid_for(m, 256), 256, 0, s>>>(h->perm, m, h->sell_ipos);
    SPMV_CUDA(cudaGetLastError());
    int64_t slots = 0, ns = 0, nu = 0, maxlen = 0;
    for (int32_t p = 0; p < np; ++p) {
        const int32_t c0 = (int32_t)(p * pc), c1 = (int32_t)std::min<int64_t>(n, (int64_t)(p + 1) * pc);
        const int32_t nnz_p = nnzs[p];
        Scratch tmp;
        int32_t *sub_idx = nullptr, *pos = nullptr;
        double* sub_val = nullptr;
        SPMV_TRY(tmp.get(&sub_idx, (size_t)nnz_p + 1));
        SPMV_TRY(tmp.get(&sub_val, (size_t)nnz_p + 1));
        SPMV_TRY(h->alloc(&pos, (size_t)nnz_p + 1, nullptr));
        k_panel_scatter<<<grid_for(m, 256), 256, 0, s>>>(c->ptr, c->idx, c->val, m, c0, c1, sub_ptrs[p], sub_idx,
                                                         sub_val, pos);
        SPMV_CUDA(cudaGetLastError());
        spmv_handle* child = new spmv_handle();
        h->panels.push_back(child);  // owned by h from here on
        h->panel_pos.push_back(pos);
        child->fmt = h->fmt;
        child->m = m;
        child->n = c1 - c0;
        child->nnz = nnz_p;
        child->device = h->device;
        child->params = h->params;
        child->params.sell_panel_cols = SPMV_SELL_PANELS_NONE;
        const spmv_csr sub{m, c1 - c0, (int64_t)nnz_p, sub_ptrs[p], sub_idx, sub_val};
        SPMV_TRY(sell_build(child, &sub, s, h->perm));  // the shared order; the child does not own it
        child->sell_ys = h->sell_ys;
        SPMV_CUDA(cudaStreamSynchronize(s));
        h->device_bytes += child->device_bytes;
        slots += child->stored_slots;
        ns += child->aux[0];
        nu += child->aux[1];
        maxlen = std::max<int64_t>(maxlen, child->aux[2]);
    }
    h->sell_C = h->panels[0]->sell_C;
    h->sell_sigma = h->panels[0]->sell_sigma;
    h->params.sell_C = h->panels[0]->params.sell_C;
    h->params.sell_sigma = h->panels[0]->params.sell_sigma;
    h->stored_slots = slots;
    h->aux[0] = ns;
    h->aux[1] = nu;
    h->aux[2] = maxlen;
    h->aux[3] = np;
    return SPMV_OK;
}

// Warp w takes units w, w + warps, ... (the sort puts the widest slices,
// split into chunks, first, so the static split is balanced).  Register
// budgets keep 8 / 5 / 4 blocks resident for C = 32 / 64 / 128 (measured:
// C = 32 on the power-law matrix 77.6 us at 40 registers, 74.8 at 32).
template <int R, int MODE>
__global__ void __launch_bounds__(256, R == 1 ? 8 : (R == 2 ? 5 : 4)) k_sell(dev::SellArgs a, int32_t nu) {
    dev::pdl_wait();  // launched early (launch_pdl): wait for the kernel ahead
    const int32_t stride = (int32_t)gridDim.x * 8;
    for (int32_t u = (int32_t)(blockIdx.x * 8 + (threadIdx.x >> 5)); u < nu; u += stride)
        dev::sell_unit<R, MODE>(a, u, threadIdx.x & 31);
}

// Blocks of the SELL kernel: four waves of resident blocks, each warp taking
// every (grid x 8)-th unit.  Measured on the 2e6-row power-law matrix: one
// unit per warp 81.6 us, one wave 89.5 (imbalance), two 78.9, four 77.6,
// eight 78.7.
template <int R>
static int32_t sell_grid() {
    static int32_t g = 0;  // the same GPU model on every device of a box
    if (g == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sell<R, dev::kSellPlain>, 256, 0);
        g = sms * (per_sm > 0 ? per_sm : 1) * 4;
    }
    return g;
}

template <int MODE>
static void sell_launch(const spmv_handle* h, const double* x, double* y, cudaStream_t s) {
    dev::SellArgs a{h->sell_units, h->slice_ptr, h->sell_len, h->perm, h->sell_col, h->sell_val,
                    h->sell_partial, h->sell_counters, h->m, kSellUnitWidth, x, y, h->sell_ys};
    if (h->n_sell_units <= 0) return;
    const int64_t need = grid_for(h->n_sell_units, 8);
    switch (h->sell_C) {
        case 32:
            launch_pdl(k_sell<1, MODE>, dim3((unsigned)std::min<int64_t>(need, sell_grid<1>())), dim3(256), 0, s, a,
                       h->n_sell_units);
            break;
        case 64:
            launch_pdl(k_sell<2, MODE>, dim3((unsigned)std::min<int64_t>(need, sell_grid<2>())), dim3(256), 0, s, a,
                       h->n_sell_units);
            break;
        default:
            launch_pdl(k_sell<4, MODE>, dim3((unsigned)std::min<int64_t>(need, sell_grid<4>())), dim3(256), 0, s, a,
                       h->n_sell_units);
            break;
    }
}

// y[i] = ys[ipos[i]]: the panels' sums back in row order.  Rows in order
// write whole sectors of y; the reads of ys stay inside a window of the
// shared order at a time (or in the small region of the long rows), where
// L2 serves the neighbouring entries.
__global__ void __launch_bounds__(256) k_sell_unpermute(const int32_t* __restrict__ ipos, const double* __restrict__ ys,
                                                        double* __restrict__ y, int32_t m) {
    dev::pdl_wait();  // launched early (launch_pdl): wait for the last panel
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += stride)
        __stcs(y + i, ys[__ldcs(ipos + i)]);
}

int sell_run(const spmv_handle* h, const double* x, double* y, cudaStream_t s) {
    if (h->panels.empty()) {
        if (h->sell_ident) sell_launch<dev::kSellIdent>(h, x, y, s);
        else sell_launch<dev::kSellPlain>(h, x, y, s);
    } else {  // ys = A_0 x_0, ys += A_p x_p (p = 1 .. last), then y = ys through the shared row order
        const size_t np = h->panels.size();
        for (size_t p = 0; p < np; ++p) {
            const double* xp = x + (int64_t)p * h->panel_cols;
            if (p == 0) sell_launch<dev::kSellFirst>(h->panels[p], xp, y, s);
            else sell_launch<dev::kSellMid>(h->panels[p], xp, y, s);
        }
        launch_pdl(k_sell_unpermute, dim3((unsigned)grid_capped(h->m, 256, 8)), dim3(256), 0, s,
                   (const int32_t*)h->sell_ipos, (const double*)h->sell_ys, y, h->m);
    }
    SPMV_CUDA(cudaGetLastError());
    return SPMV_OK;
}

__global__ void k_unsort_len(const int32_t* __restrict__ sl, const int32_t* __restrict__ perm, int32_t m,
                             int32_t* __restrict__ len, int32_t* __restrict__ ipos) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < m) {
        len[perm[p]] = sl[p];
        ipos[perm[p]] = (int32_t)p;
    }
}

__global__ void k_sell_gather(const int32_t* __restrict__ ptr, int32_t m, int64_t nnz, const int32_t* __restrict__ ipos,
                              const int64_t* __restrict__ sp, int32_t C, const int32_t* __restrict__ col,
                              const double* __restrict__ sv, int32_t* __restrict__ idx, double* __restrict__ val) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = row_of_nnz(ptr, m, k);
        const int64_t j = k - ptr[r];
        const int32_t p = ipos[r];
        const int64_t src = sp[p / C] + j * C + (p % C);
        idx[k] = col[src];
        val[k] = sv[src];
    }
}

static int sell_to_csr_one(const spmv_handle* h, int32_t* ptr, int32_t* idx, double* val, cudaStream_t s);

int sell_to_csr(const spmv_handle* h, int32_t* ptr, int32_t* idx, double* val, cudaStream_t s) {
    if (h->panels.empty()) return sell_to_csr_one(h, ptr, idx, val, s);
    SPMV_CUDA(cudaMemcpyAsync(ptr, h->ptr, sizeof(int32_t) * ((size_t)h->m + 1), cudaMemcpyDeviceToDevice, s));
    for (size_t p = 0; p < h->panels.size(); ++p) {
        const spmv_handle* c = h->panels[p];
        Scratch tmp;
        int32_t *sp = nullptr, *si = nullptr;
        double* sv = nullptr;
        SPMV_TRY(tmp.get(&sp, (size_t)h->m + 1));
        SPMV_TRY(tmp.get(&si, (size_t)c->nnz + 1));
        SPMV_TRY(tmp.get(&sv, (size_t)c->nnz + 1));
        SPMV_TRY(sell_to_csr_one(c, sp, si, sv, s));
        if (c->nnz > 0) {
            int g = grid_capped(c->nnz, 256, 64);
            k_panel_unscatter<<<g, 256, 0, s>>>(si, sv, h->panel_pos[p], c->nnz, (int32_t)(p * h->panel_cols), idx, val);
            SPMV_CUDA(cudaGetLastError());
        }
        SPMV_CUDA(cudaStreamSynchronize(s));
    }
    return SPMV_OK;
}

static int sell_to_csr_one(const spmv_handle* h, int32_t* ptr, int32_t* idx, double* val, cudaStream_t s) {
    Scratch tmp;
    int32_t *len = nullptr, *ipos = nullptr;
    SPMV_TRY(tmp.get(&len, (size_t)h->m));
    SPMV_TRY(tmp.get(&ipos, (size_t)h->m));
    k_unsort_len<<<grid_for(h->m, 256), 256, 0, s>>>(h->sell_len, h->perm, h->m, len, ipos);
    SPMV_CUDA(cudaGetLastError());
    SPMV_TRY(exclusive_scan<int32_t>(len, ptr, h->m, s, tmp));
    if (h->nnz > 0) {
        int g = grid_capped(h->nnz, 256, 64);
        k_sell_gather<<<g, 256, 0, s>>>(ptr, h->m, h->nnz, ipos, h->slice_ptr, h->sell_C, h->sell_col, h->sell_val, idx,
                                        val);
    }
    SPMV_CUDA(cudaGetLastError());
    SPMV_CUDA(cudaStreamSynchronize(s));
    return SPMV_OK;
}

}  // namespace spmv
