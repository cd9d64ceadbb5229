/*
 * Seeded synthetic sparse-matrix generators.
 *
 * This module builds INPUTS only: row lengths, column patterns, values and
 * dense vectors for the workloads the library is measured on.  It holds none
 * of the sparse matrix-vector product's arithmetic and no format conversion;
 * both the CPU oracle and the CUDA path read the arrays it writes.
 *
 * Randomness is counter based: every draw is mix64(seed, stream, counter)
 * (a SplitMix64 finaliser applied twice), so the content of row i depends
 * only on (seed, i) and the result is the same for any thread count.
 * Normal deviates use the Box-Muller transform; power-law lengths use the
 * inverse CDF of a Pareto law truncated to [xmin, xmax].
 *
 * Plain C99 + pthreads, no architecture-specific code.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ull

static inline uint64_t splitmix_fin(uint64_t z) {
    z += GOLDEN;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* The one counter-based generator: value number `ctr` of stream `stream`. */
static inline uint64_t draw_u64(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return splitmix_fin(splitmix_fin(seed ^ splitmix_fin(stream * GOLDEN + 0x632BE59BD9B4E019ull)) + ctr * GOLDEN);
}

/* Uniform in [0, 1) with 53 random bits. */
static inline double draw_u01(uint64_t seed, uint64_t stream, uint64_t ctr) {
    return (double)(draw_u64(seed, stream, ctr) >> 11) * 0x1.0p-53;
}

/* Uniform integer in [0, n) (n >= 1), by 64x64->128 multiply-shift. */
static inline uint64_t draw_below(uint64_t seed, uint64_t stream, uint64_t ctr, uint64_t n) {
    unsigned __int128 p = (unsigned __int128)draw_u64(seed, stream, ctr) * n;
    return (uint64_t)(p >> 64);
}

static inline double draw_normal(uint64_t seed, uint64_t stream, uint64_t ctr) {
    double u1 = draw_u01(seed, stream, 2 * ctr);
    double u2 = draw_u01(seed, stream, 2 * ctr + 1);
    if (u1 < 0x1.0p-60) u1 = 0x1.0p-60;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Stream tags keep the different draws of one row independent. */
enum { TAG_LEN = 1, TAG_COL = 2, TAG_VAL = 3, TAG_VEC = 4, TAG_INT = 5 };
static inline uint64_t stream_of(int tag, int64_t row) { return ((uint64_t)tag << 56) ^ (uint64_t)row; }

/* ---------------------------------------------------------------- threads */

typedef void (*range_fn)(void* ctx, int64_t lo, int64_t hi);
typedef struct { range_fn fn; void* ctx; int64_t lo, hi; } range_job;

static void* range_trampoline(void* p) {
    range_job* j = (range_job*)p;
    j->fn(j->ctx, j->lo, j->hi);
    return NULL;
}

static void parallel_for(int64_t n, int nthreads, range_fn fn, void* ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (n < 4096 || nthreads == 1) { fn(ctx, 0, n); return; }
    pthread_t th[256];
    range_job jobs[256];
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn; jobs[t].ctx = ctx;
        jobs[t].lo = n * t / nthreads; jobs[t].hi = n * (t + 1) / nthreads;
        if (pthread_create(&th[t], NULL, range_trampoline, &jobs[t]) == 0) started = t + 1;
        else { fn(ctx, jobs[t].lo, jobs[t].hi); }
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------------------ row lengths */

/* Truncated Pareto on [xmin, xmax] with density proportional to x^-alpha,
 * rounded up, then clipped to [lmin, lmax].  Returns the total. */
int64_t synth_powerlaw_lengths(int32_t m, double alpha, double xmin, double xmax,
                               int32_t lmin, int32_t lmax, uint64_t seed, int32_t* len) {
    double a = alpha - 1.0;
    double tail = pow(xmin / xmax, a); /* P(X > xmax) of the untruncated law */
    int64_t total = 0;
    for (int64_t i = 0; i < m; ++i) {
        double u = draw_u01(seed, stream_of(TAG_LEN, i), 0);
        double x = xmin * pow(1.0 - u * (1.0 - tail), -1.0 / a);
        double c = ceil(x);
        int64_t l = (c > (double)lmax) ? lmax : (int64_t)c;
        if (l < lmin) l = lmin;
        len[i] = (int32_t)l;
        total += l;
    }
    return total;
}

/* Uniform integer lengths in [lo, hi]. */
int64_t synth_uniform_lengths(int32_t m, int32_t lo, int32_t hi, uint64_t seed, int32_t* len) {
    int64_t total = 0;
    for (int64_t i = 0; i < m; ++i) {
        len[i] = lo + (int32_t)draw_below(seed, stream_of(TAG_LEN, i), 0, (uint64_t)(hi - lo + 1));
        total += len[i];
    }
    return total;
}

/* ptr[0] = 0, ptr[i+1] = ptr[i] + len[i]; returns -1 if the total needs more than int32. */
int64_t synth_lengths_to_ptr(int32_t m, const int32_t* len, int32_t* ptr) {
    int64_t acc = 0;
    ptr[0] = 0;
    for (int64_t i = 0; i < m; ++i) {
        acc += len[i];
        if (acc > 2147483647LL) return -1;
        ptr[i + 1] = (int32_t)acc;
    }
    return acc;
}

/* ----------------------------------------------------- random column sets */

typedef struct { int32_t n_cols; const int32_t* ptr; uint64_t seed; int32_t* idx; } cols_ctx;

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static void sort_small(int32_t* v, int64_t n) {
    if (n > 48) { qsort(v, (size_t)n, sizeof(int32_t), cmp_i32); return; }
    for (int64_t i = 1; i < n; ++i) {
        int32_t t = v[i]; int64_t j = i - 1;
        while (j >= 0 && v[j] > t) { v[j + 1] = v[j]; --j; }
        v[j + 1] = t;
    }
}

/* Each row gets len distinct columns drawn uniformly from [0, n_cols),
 * sorted ascending; a duplicate is replaced by a fresh draw (resampling). */
static void cols_range(void* p, int64_t lo, int64_t hi) {
    cols_ctx* c = (cols_ctx*)p;
    for (int64_t i = lo; i < hi; ++i) {
        int64_t b = c->ptr[i], l = c->ptr[i + 1] - c->ptr[i];
        int32_t* r = c->idx + b;
        uint64_t s = stream_of(TAG_COL, i), ctr = 0;
        if (l >= c->n_cols) { /* the full row */
            for (int64_t k = 0; k < l; ++k) r[k] = (int32_t)(k % c->n_cols);
            continue;
        }
        for (int64_t k = 0; k < l; ++k) r[k] = (int32_t)draw_below(c->seed, s, ctr++, (uint64_t)c->n_cols);
        for (;;) {
            sort_small(r, l);
            int64_t dups = 0;
            for (int64_t k = 1; k < l; ++k)
                if (r[k] == r[k - 1]) { r[k - 1] = (int32_t)draw_below(c->seed, s, ctr++, (uint64_t)c->n_cols); ++dups; }
            if (!dups) break;
        }
    }
}

void synth_fill_random_cols(int32_t m, int32_t n_cols, const int32_t* ptr, uint64_t seed,
                            int32_t* idx, int nthreads) {
    cols_ctx c = {n_cols, ptr, seed, idx};
    parallel_for(m, nthreads, cols_range, &c);
}

/* ------------------------------------------------------------------ values */

typedef struct { uint64_t seed; int kind; double lo, hi; double* out; } val_ctx;

static void val_range(void* p, int64_t lo, int64_t hi) {
    val_ctx* c = (val_ctx*)p;
    for (int64_t k = lo; k < hi; ++k) {
        if (c->kind == 0) c->out[k] = draw_normal(c->seed, stream_of(TAG_VAL, k >> 20), (uint64_t)(k & 0xFFFFF));
        else if (c->kind == 1) c->out[k] = c->lo + (c->hi - c->lo) * draw_u01(c->seed, stream_of(TAG_VEC, k >> 20), (uint64_t)(k & 0xFFFFF));
        else c->out[k] = c->lo + (double)draw_below(c->seed, stream_of(TAG_INT, k >> 20), (uint64_t)(k & 0xFFFFF), (uint64_t)(c->hi - c->lo + 1));
    }
}

/* N(0,1) values. */
void synth_fill_normal(int64_t n, uint64_t seed, double* out, int nthreads) {
    val_ctx c = {seed, 0, 0, 0, out};
    parallel_for(n, nthreads, val_range, &c);
}

/* Uniform values in [lo, hi). */
void synth_fill_uniform(int64_t n, uint64_t seed, double lo, double hi, double* out, int nthreads) {
    val_ctx c = {seed, 1, lo, hi, out};
    parallel_for(n, nthreads, val_range, &c);
}

/* Integer values drawn uniformly from {lo, ..., hi}, stored as doubles. */
void synth_fill_int(int64_t n, uint64_t seed, int64_t lo, int64_t hi, double* out, int nthreads) {
    val_ctx c = {seed, 2, (double)lo, (double)hi, out};
    parallel_for(n, nthreads, val_range, &c);
}

/* ------------------------------------------------------------ structured */

/* Stencil kinds: 0 = 2D 5-point, 1 = 2D 9-point, 2 = 3D 7-point, 3 = 3D 27-point.
 * Grid point (x, y, z) with x fastest is row x + nx*(y + ny*z); neighbours
 * outside the grid are dropped.  Columns come out ascending. */
static int stencil_offsets(int kind, int off[27][3]) {
    int n = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int nz_ = (dz != 0) + (dy != 0) + (dx != 0);
                int keep;
                if (kind == 0) keep = (dz == 0) && nz_ <= 1;
                else if (kind == 1) keep = (dz == 0);
                else if (kind == 2) keep = nz_ <= 1;
                else keep = 1;
                if (keep) { off[n][0] = dx; off[n][1] = dy; off[n][2] = dz; ++n; }
            }
    return n;
}

typedef struct { int kind, nx, ny, nz; int32_t* ptr; int32_t* idx; int count_only; } sten_ctx;

static void sten_range(void* p, int64_t lo, int64_t hi) {
    sten_ctx* c = (sten_ctx*)p;
    int off[27][3];
    int no = stencil_offsets(c->kind, off);
    for (int64_t r = lo; r < hi; ++r) {
        int64_t x = r % c->nx, y = (r / c->nx) % c->ny, z = r / ((int64_t)c->nx * c->ny);
        int64_t w = c->count_only ? 0 : c->ptr[r];
        int cnt = 0;
        for (int k = 0; k < no; ++k) {
            int64_t xx = x + off[k][0], yy = y + off[k][1], zz = z + off[k][2];
            if (xx < 0 || yy < 0 || zz < 0 || xx >= c->nx || yy >= c->ny || zz >= c->nz) continue;
            if (!c->count_only) c->idx[w + cnt] = (int32_t)(xx + c->nx * (yy + c->ny * zz));
            ++cnt;
        }
        if (c->count_only) c->ptr[r + 1] = cnt; /* lengths, prefix-summed by the caller */
    }
}

/* Writes row lengths into ptr[1..m]; the caller prefix-sums them. */
void synth_stencil_lengths(int kind, int nx, int ny, int nz, int32_t* ptr, int nthreads) {
    sten_ctx c = {kind, nx, ny, nz, ptr, NULL, 1};
    parallel_for((int64_t)nx * ny * nz, nthreads, sten_range, &c);
}

void synth_stencil_cols(int kind, int nx, int ny, int nz, const int32_t* ptr, int32_t* idx, int nthreads) {
    sten_ctx c = {kind, nx, ny, nz, (int32_t*)ptr, idx, 0};
    parallel_for((int64_t)nx * ny * nz, nthreads, sten_range, &c);
}

/* Makes every row's diagonal entry 1 + sum of |off-diagonal| (diagonal dominance). */
void synth_diag_dominant(int32_t m, const int32_t* ptr, const int32_t* idx, double* val) {
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        int64_t d = -1;
        for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
            if (idx[k] == i) d = k; else s += fabs(val[k]);
        }
        if (d >= 0) val[d] = 1.0 + s;
    }
}

/* Band: row i holds columns max(0, i-bw) .. min(n-1, i+bw). */
void synth_band_lengths(int32_t m, int32_t bw, int32_t* len) {
    for (int64_t i = 0; i < m; ++i) {
        int64_t lo = i - bw < 0 ? 0 : i - bw, hi = i + bw > m - 1 ? m - 1 : i + bw;
        len[i] = (int32_t)(hi - lo + 1);
    }
}

void synth_band_cols(int32_t m, int32_t bw, const int32_t* ptr, int32_t* idx) {
    for (int64_t i = 0; i < m; ++i) {
        int64_t lo = i - bw < 0 ? 0 : i - bw;
        for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) idx[k] = (int32_t)(lo + (k - ptr[i]));
    }
}

/* Block diagonal with dense b x b blocks (the last block may be smaller). */
void synth_blockdiag_lengths(int32_t m, int32_t b, int32_t* len) {
    for (int64_t i = 0; i < m; ++i) {
        int64_t s = (i / b) * b, e = s + b > m ? m : s + b;
        len[i] = (int32_t)(e - s);
    }
}

void synth_blockdiag_cols(int32_t m, int32_t b, const int32_t* ptr, int32_t* idx) {
    for (int64_t i = 0; i < m; ++i) {
        int64_t s = (i / b) * b;
        for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) idx[k] = (int32_t)(s + (k - ptr[i]));
    }
}

/* Scalar draws for workload parameters (matrix sizes, families). */
double synth_scalar_u01(uint64_t seed, uint64_t stream, uint64_t ctr) { return draw_u01(seed, stream, ctr); }
uint64_t synth_scalar_u64(uint64_t seed, uint64_t stream, uint64_t ctr) { return draw_u64(seed, stream, ctr); }
