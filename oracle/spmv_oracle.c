/*
 * CPU ORACLE -- test infrastructure only.
 *
 * Plain, single-threaded (one optional row-split threaded copy), obviously
 * correct C for what the library computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load this file's library;
 * the product path never does, and this file shares no code with it.
 *
 * Build: gcc -O2 -ffp-contract=off (multiply and add stay separate, so every
 * row sum is the plain left-to-right recursive sum in CSR order).
 *
 * Citations are to arXiv:1805.11938 ("Optimizing Sparse Matrix-Vector
 * Multiplication on Emerging Many-Core Architectures"):
 *   Sec. II-A     y = A x, A sparse M x N, x and y dense.
 *   Sec. II-B     COO, CSR, CSR5, ELL, SELL / SELL-C-sigma and HYB layouts;
 *   Table I       the worked 4 x 4, nnz = 8 example of every layout.
 * Readings where the paper is silent are stated at each function.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------ SpMV, Sec. II-A */

/* y_i = sum over k in [ptr[i], ptr[i+1]) of val[k] * x[idx[k]], summed left to
 * right in CSR order (Sec. II-A definition over the Sec. II-B CSR arrays).
 * An empty row gives +0.0. */
void oracle_csr_spmv(int32_t m, const int32_t* ptr, const int32_t* idx, const double* val,
                     const double* x, double* y) {
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
            double p = val[k] * x[idx[k]];
            s = s + p;
        }
        y[i] = s;
    }
}

/* The same per-row code on contiguous row ranges, one range per thread.  Each
 * y_i is computed by exactly the loop above, so the result is bit-identical to
 * the single-threaded call. */
typedef struct {
    int32_t lo, hi;
    const int32_t* ptr; const int32_t* idx; const double* val; const double* x; double* y;
} oracle_rows_job;

static void* oracle_rows_worker(void* p) {
    oracle_rows_job* j = (oracle_rows_job*)p;
    oracle_csr_spmv(j->hi - j->lo, j->ptr + j->lo, j->idx, j->val, j->x, j->y + j->lo);
    return NULL;
}

void oracle_csr_spmv_threads(int32_t m, const int32_t* ptr, const int32_t* idx, const double* val,
                             const double* x, double* y, int nthreads) {
    if (nthreads <= 1 || m < 1024) { oracle_csr_spmv(m, ptr, idx, val, x, y); return; }
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    oracle_rows_job jobs[256];
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].lo = (int32_t)((int64_t)m * t / nthreads);
        jobs[t].hi = (int32_t)((int64_t)m * (t + 1) / nthreads);
        jobs[t].ptr = ptr; jobs[t].idx = idx; jobs[t].val = val; jobs[t].x = x; jobs[t].y = y;
        if (pthread_create(&th[t], NULL, oracle_rows_worker, &jobs[t]) == 0) started = t + 1;
        else oracle_rows_worker(&jobs[t]);
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
}

/* s_i = sum_j |a_ij * x_j|, the scale of the floating-point error bound
 * |y_i - y_ref,i| <= 4 * nnz_i * 2^-53 * s_i. */
void oracle_row_abs_sum(int32_t m, const int32_t* ptr, const int32_t* idx, const double* val,
                        const double* x, double* s) {
    for (int64_t i = 0; i < m; ++i) {
        double a = 0.0;
        for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) a = a + fabs(val[k] * x[idx[k]]);
        s[i] = a;
    }
}

/* Dense y = A x for tiny inputs, A row-major m x n, summed over j in order. */
void oracle_dense_matvec(int32_t m, int32_t n, const double* a, const double* x, double* y) {
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double p = a[i * (int64_t)n + j] * x[j];
            s = s + p;
        }
        y[i] = s;
    }
}

/* ------------------------------------------------------ COO -> CSR, Sec. II-B */

/* CSR from COO: ptr[i] = number of entries in rows < i; entries keep their
 * COO order within a row (stable). */
void oracle_coo_to_csr(int32_t m, int64_t nnz, const int32_t* row, const int32_t* col, const double* v,
                       int32_t* ptr, int32_t* idx, double* val) {
    for (int64_t i = 0; i <= m; ++i) ptr[i] = 0;
    for (int64_t k = 0; k < nnz; ++k) ptr[row[k] + 1] += 1;
    for (int64_t i = 0; i < m; ++i) ptr[i + 1] += ptr[i];
    int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t i = 0; i < m; ++i) fill[i] = ptr[i];
    for (int64_t k = 0; k < nnz; ++k) {
        int32_t p = fill[row[k]]++;
        idx[p] = col[k];
        val[p] = v[k];
    }
    free(fill);
}

/* --------------------------------------------------------------- ELL, Sec. II-B */

int32_t oracle_max_row_len(int32_t m, const int32_t* ptr) {
    int32_t mx = 0;
    for (int64_t i = 0; i < m; ++i)
        if (ptr[i + 1] - ptr[i] > mx) mx = ptr[i + 1] - ptr[i];
    return mx;
}

/* ELL with K slots per row (K >= the longest row), stored column-major: slot s
 * of row i at s*m + i.  row_len[i] counts the real entries of row i.
 * Reading: padding holds col 0 and value +0.0 (Sec. II-B pads with zeros,
 * Table I draws them as '*'); kernels never read it. */
void oracle_csr_to_ell(int32_t m, const int32_t* ptr, const int32_t* idx, const double* val, int32_t K,
                       int32_t* row_len, int32_t* ell_col, double* ell_val) {
    for (int64_t s = 0; s < K; ++s)
        for (int64_t i = 0; i < m; ++i) { ell_col[s * m + i] = 0; ell_val[s * m + i] = 0.0; }
    for (int64_t i = 0; i < m; ++i) {
        row_len[i] = ptr[i + 1] - ptr[i];
        for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
            int64_t s = k - ptr[i];
            ell_col[s * m + i] = idx[k];
            ell_val[s * m + i] = val[k];
        }
    }
}

void oracle_ell_to_csr(int32_t m, int32_t K, const int32_t* row_len, const int32_t* ell_col, const double* ell_val,
                       int32_t* ptr, int32_t* idx, double* val) {
    (void)K;
    ptr[0] = 0;
    for (int64_t i = 0; i < m; ++i) ptr[i + 1] = ptr[i] + row_len[i];
    for (int64_t i = 0; i < m; ++i)
        for (int64_t s = 0; s < row_len[i]; ++s) {
            idx[ptr[i] + s] = ell_col[s * m + i];
            val[ptr[i] + s] = ell_val[s * m + i];
        }
}

/* ------------------------------------------------- SELL-C-sigma, Sec. II-B */

typedef struct { int32_t len, row; } len_row;

/* Longer rows first; equal lengths keep their original order (stable), the
 * tie-break Table I shows for SELL-C-sigma (row 0 before row 3). */
static int cmp_len_desc(const void* a, const void* b) {
    const len_row* p = (const len_row*)a;
    const len_row* q = (const len_row*)b;
    if (p->len != q->len) return p->len > q->len ? -1 : 1;
    return (p->row > q->row) - (p->row < q->row);
}

/* Row order and slice sizes of SELL-C-sigma.  Rows are sorted by length,
 * descending and stably, within windows of sigma rows aligned at multiples of
 * sigma (the last window may be short); sigma = 1 is plain SELL.  Sorted
 * position p holds row perm[p]; row_len[p] is that row's length.  Slice s
 * covers positions [s*C, s*C + C) (the last slice may hold fewer real rows)
 * and its width w_s is the longest row in it.  slice_ptr[s] = sum over s' < s
 * of C * w_s'.  Returns the total number of slots, slice_ptr[nslices]. */
int64_t oracle_sell_layout(int32_t m, const int32_t* ptr, int32_t C, int32_t sigma,
                           int32_t* perm, int32_t* row_len, int64_t* slice_ptr) {
    len_row* w = (len_row*)malloc(sizeof(len_row) * (size_t)(sigma > 0 ? sigma : 1));
    for (int64_t b = 0; b < m; b += sigma) {
        int64_t e = b + sigma < m ? b + sigma : m;
        for (int64_t i = b; i < e; ++i) { w[i - b].len = ptr[i + 1] - ptr[i]; w[i - b].row = (int32_t)i; }
        qsort(w, (size_t)(e - b), sizeof(len_row), cmp_len_desc);
        for (int64_t i = b; i < e; ++i) { perm[i] = w[i - b].row; row_len[i] = w[i - b].len; }
    }
    free(w);
    int64_t nslices = ((int64_t)m + C - 1) / C;
    slice_ptr[0] = 0;
    for (int64_t s = 0; s < nslices; ++s) {
        int32_t width = 0;
        for (int64_t p = s * C; p < s * C + C && p < m; ++p)
            if (row_len[p] > width) width = row_len[p];
        slice_ptr[s + 1] = slice_ptr[s] + (int64_t)C * width;
    }
    return slice_ptr[nslices];
}

/* Slot j of lane l (sorted position s*C + l) of slice s lives at
 * slice_ptr[s] + j*C + l (column-major inside the slice).  Padding: col 0,
 * value +0.0. */
void oracle_csr_to_sell(int32_t m, const int32_t* ptr, const int32_t* idx, const double* val, int32_t C,
                        const int32_t* perm, const int64_t* slice_ptr, int32_t* col, double* v) {
    int64_t nslices = ((int64_t)m + C - 1) / C;
    for (int64_t t = 0; t < slice_ptr[nslices]; ++t) { col[t] = 0; v[t] = 0.0; }
    for (int64_t p = 0; p < m; ++p) {
        int64_t s = p / C, l = p % C;
        int32_t r = perm[p];
        for (int64_t j = 0; j < ptr[r + 1] - ptr[r]; ++j) {
            col[slice_ptr[s] + j * C + l] = idx[ptr[r] + j];
            v[slice_ptr[s] + j * C + l] = val[ptr[r] + j];
        }
    }
}

void oracle_sell_to_csr(int32_t m, int32_t C, const int32_t* perm, const int32_t* row_len, const int64_t* slice_ptr,
                        const int32_t* col, const double* v, int32_t* ptr, int32_t* idx, double* val) {
    int32_t* len = (int32_t*)calloc((size_t)(m > 0 ? m : 1), sizeof(int32_t));
    for (int64_t p = 0; p < m; ++p) len[perm[p]] = row_len[p];
    ptr[0] = 0;
    for (int64_t i = 0; i < m; ++i) ptr[i + 1] = ptr[i] + len[i];
    for (int64_t p = 0; p < m; ++p) {
        int64_t s = p / C, l = p % C;
        int32_t r = perm[p];
        for (int64_t j = 0; j < row_len[p]; ++j) {
            idx[ptr[r] + j] = col[slice_ptr[s] + j * C + l];
            val[ptr[r] + j] = v[slice_ptr[s] + j * C + l];
        }
    }
    free(len);
}

/* --------------------------------------------------------------- HYB, Sec. II-B */

/* The "typical" row length K of HYB.  Reading of Sec. II-B (K "can be
 * calculated directly"): K is the largest k such that at least ceil(m/3) rows
 * hold k or more entries, 0 if there is none.  Table I's K = 2 follows: three
 * of four rows have >= 2 entries, one has >= 3. */
int32_t oracle_hyb_k(int32_t m, const int32_t* ptr) {
    if (m <= 0) return 0;
    int64_t need = ((int64_t)m + 2) / 3;
    int32_t mx = oracle_max_row_len(m, ptr);
    int64_t* cnt = (int64_t*)calloc((size_t)mx + 2, sizeof(int64_t));
    for (int64_t i = 0; i < m; ++i) cnt[ptr[i + 1] - ptr[i]] += 1;
    int64_t atleast = 0; /* rows with length >= k, for k from mx down */
    int32_t K = 0;
    for (int64_t k = mx; k >= 1; --k) {
        atleast += cnt[k];
        if (atleast >= need) { K = (int32_t)k; break; }
    }
    free(cnt);
    return K;
}

/* Entries past the first K of each row. */
int64_t oracle_hyb_tail_count(int32_t m, const int32_t* ptr, int32_t K) {
    int64_t t = 0;
    for (int64_t i = 0; i < m; ++i)
        if (ptr[i + 1] - ptr[i] > K) t += ptr[i + 1] - ptr[i] - K;
    return t;
}

/* HYB = ELL holding the first min(len_i, K) entries of every row (column-major,
 * as oracle_csr_to_ell) + COO holding the rest, rows ascending and CSR order
 * within a row (Table I: row 1's third entry (1, 3, 3) goes to COO). */
void oracle_csr_to_hyb(int32_t m, const int32_t* ptr, const int32_t* idx, const double* val, int32_t K,
                       int32_t* row_len_ell, int32_t* ell_col, double* ell_val,
                       int32_t* coo_row, int32_t* coo_col, double* coo_val) {
    for (int64_t s = 0; s < K; ++s)
        for (int64_t i = 0; i < m; ++i) { ell_col[s * m + i] = 0; ell_val[s * m + i] = 0.0; }
    int64_t t = 0;
    for (int64_t i = 0; i < m; ++i) {
        int64_t len = ptr[i + 1] - ptr[i];
        row_len_ell[i] = (int32_t)(len < K ? len : K);
        for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
            int64_t s = k - ptr[i];
            if (s < K) { ell_col[s * m + i] = idx[k]; ell_val[s * m + i] = val[k]; }
            else { coo_row[t] = (int32_t)i; coo_col[t] = idx[k]; coo_val[t] = val[k]; ++t; }
        }
    }
}

void oracle_hyb_to_csr(int32_t m, int32_t K, const int32_t* row_len_ell, const int32_t* ell_col, const double* ell_val,
                       int64_t ntail, const int32_t* coo_row, const int32_t* coo_col, const double* coo_val,
                       int32_t* ptr, int32_t* idx, double* val) {
    (void)K;
    int32_t* len = (int32_t*)calloc((size_t)(m > 0 ? m : 1), sizeof(int32_t));
    for (int64_t i = 0; i < m; ++i) len[i] = row_len_ell[i];
    for (int64_t t = 0; t < ntail; ++t) len[coo_row[t]] += 1;
    ptr[0] = 0;
    for (int64_t i = 0; i < m; ++i) ptr[i + 1] = ptr[i] + len[i];
    for (int64_t i = 0; i < m; ++i)
        for (int64_t s = 0; s < row_len_ell[i]; ++s) {
            idx[ptr[i] + s] = ell_col[s * m + i];
            val[ptr[i] + s] = ell_val[s * m + i];
        }
    int32_t* fill = (int32_t*)calloc((size_t)(m > 0 ? m : 1), sizeof(int32_t));
    for (int64_t i = 0; i < m; ++i) fill[i] = ptr[i] + row_len_ell[i];
    for (int64_t t = 0; t < ntail; ++t) {
        int32_t p = fill[coo_row[t]]++;
        idx[p] = coo_col[t];
        val[p] = coo_val[t];
    }
    free(fill);
    free(len);
}

/* -------------------------------------------------------------- CSR5, Sec. II-B */

/* Row holding nonzero k: the i with ptr[i] <= k < ptr[i+1] (empty rows skipped). */
static int32_t row_of_nnz(int32_t m, const int32_t* ptr, int64_t k) {
    int32_t lo = 0, hi = m - 1;
    while (lo < hi) { /* largest i with ptr[i] <= k */
        int32_t mid = lo + (hi - lo + 1) / 2;
        if (ptr[mid] <= k) lo = mid; else hi = mid - 1;
    }
    return lo;
}

int64_t oracle_csr5_ntiles(int64_t nnz, int32_t omega, int32_t sigma) {
    int64_t S = (int64_t)omega * sigma;
    return (nnz + S - 1) / S;
}

/* CSR5 layout (Sec. II-B and Table I, omega = tile width, sigma = tile height).
 * Nonzeros are cut into tiles of S = omega*sigma consecutive entries.  Reading
 * of Table I: column c of tile t holds nonzeros t*S + c*sigma + r for
 * r = 0..sigma-1, and slot (r, c) is stored at t*S + r*omega + c (the tile is
 * stored transposed, so one row of the tile is omega consecutive values).
 * The last tile is padded with col 0, value +0.0, flag 0.
 *   bit_flag[t*S + r*omega + c] = 1 if that nonzero starts a row, or if it is
 *     the tile's first slot (Table I flags tile 1's first slot although row 1
 *     continues there).
 *   tile_ptr[t] = the row holding nonzero t*S; tile_ptr[ntiles] = m.
 *   y_off[t*omega + c] = flagged slots of tile t in columns before c.
 *   seg_off[t*omega + c] = 1 if column c of tile t has no flagged slot.
 * Reading for empty rows (the paper is silent): a tile whose row span
 * [tile_ptr[t], row of its last nonzero] contains an empty row lists, for
 * each flagged slot in nonzero order, the row it starts in
 * empty_rows[empty_ptr[t] .. empty_ptr[t+1]); other tiles list nothing and
 * their j-th flagged slot belongs to row tile_ptr[t] + j.
 * empty_rows may be NULL to size it: the return value is its length. */
int64_t oracle_csr_to_csr5(int32_t m, const int32_t* ptr, const int32_t* idx, const double* val,
                           int32_t omega, int32_t sigma,
                           int32_t* tile_ptr, uint8_t* bit_flag, int32_t* y_off, uint8_t* seg_off,
                           int32_t* tidx, double* tval, int32_t* empty_ptr, int32_t* empty_rows) {
    int64_t nnz = m > 0 ? ptr[m] : 0;
    int64_t S = (int64_t)omega * sigma;
    int64_t nt = oracle_csr5_ntiles(nnz, omega, sigma);
    int64_t ne = 0;
    for (int64_t t = 0; t < nt; ++t) {
        int64_t base = t * S;
        tile_ptr[t] = row_of_nnz(m, ptr, base);
        int64_t last = base + S - 1 < nnz - 1 ? base + S - 1 : nnz - 1;
        int32_t last_row = row_of_nnz(m, ptr, last);
        int has_empty = 0;
        for (int64_t i = tile_ptr[t]; i <= last_row; ++i)
            if (ptr[i + 1] == ptr[i]) has_empty = 1;
        empty_ptr[t] = (int32_t)ne;
        int32_t flagged_before = 0;
        for (int64_t c = 0; c < omega; ++c) {
            y_off[t * omega + c] = flagged_before;
            int32_t col_flags = 0;
            for (int64_t r = 0; r < sigma; ++r) {
                int64_t k = base + c * sigma + r;
                int64_t slot = base + r * omega + c;
                uint8_t f = 0;
                if (k < nnz) {
                    int32_t row = row_of_nnz(m, ptr, k);
                    f = (ptr[row] == k) || (c == 0 && r == 0);
                    tidx[slot] = idx[k];
                    tval[slot] = val[k];
                    if (f && has_empty) {
                        if (empty_rows) empty_rows[ne] = row;
                        ++ne;
                    }
                } else {
                    tidx[slot] = 0;
                    tval[slot] = 0.0;
                }
                bit_flag[slot] = f;
                col_flags += f;
            }
            seg_off[t * omega + c] = col_flags == 0;
            flagged_before += col_flags;
        }
    }
    tile_ptr[nt] = m;
    empty_ptr[nt] = (int32_t)ne;
    return ne;
}

/* Back to CSR: ptr is part of the CSR5 format (Table I lists it), and undoing
 * the tile transpose restores indices and values in CSR order. */
void oracle_csr5_to_csr(int32_t m, const int32_t* csr5_ptr, int64_t nnz, int32_t omega, int32_t sigma,
                        const int32_t* tidx, const double* tval, int32_t* ptr, int32_t* idx, double* val) {
    int64_t S = (int64_t)omega * sigma;
    for (int64_t i = 0; i <= m; ++i) ptr[i] = csr5_ptr[i];
    for (int64_t k = 0; k < nnz; ++k) {
        int64_t t = k / S, w = k % S, c = w / sigma, r = w % sigma;
        idx[k] = tidx[t * S + r * omega + c];
        val[k] = tval[t * S + r * omega + c];
    }
}
