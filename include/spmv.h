/*
 * spmv.h -- C ABI of the GB300 (sm_103a) FP64 sparse matrix-vector library.
 *
 * The library computes y = A x for a sparse M x N matrix A held in one of the
 * five representations compared in arXiv:1805.11938 (CSR, CSR5, ELL,
 * SELL-C-sigma and HYB = ELL + COO), converts between CSR and each of them,
 * extracts static matrix features, and picks a format per matrix with a small
 * learned classifier, as the paper's Sec. V proposes.
 *
 * Conventions for every call
 *  - Pointers named *_dev, x, y and the spmv_csr arrays are DEVICE pointers of
 *    the current CUDA device; *_host pointers are host memory.
 *  - Indices are int32, values FP64.  Row pointers (ptr) are int32 with
 *    ptr[0] = 0 and ptr[M] = nnz, so nnz < 2^31.
 *  - Every call returns SPMV_OK (0) or a negative spmv_status.  A call that
 *    fails writes nothing to its outputs (y, handles, ...).
 *    spmv_last_error() gives a one-line detail of the calling thread's last
 *    failure.
 *  - Work is enqueued on the caller's stream and runs asynchronously; only
 *    the calls documented as synchronising wait for the device.
 *  - Handles and models own their device memory; inputs, x and y stay owned
 *    by the caller.  x and y must not alias.
 */
#ifndef SPMV_GB300_H
#define SPMV_GB300_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#if defined(__GNUC__)
#define SPMV_API __attribute__((visibility("default")))
#else
#define SPMV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* The five representations of Sec. II-B (Table I), in the paper's order. */
typedef enum {
    SPMV_CSR = 0,
    SPMV_CSR5 = 1,
    SPMV_ELL = 2,
    SPMV_SELL = 3, /* SELL-C-sigma; sigma = 1 is plain SELL */
    SPMV_HYB = 4
} spmv_fmt;

#define SPMV_NUM_FORMATS 5
#define SPMV_NUM_FEATURES 16
#define SPMV_MLP_PARAMS 5573 /* 16x64 + 64 + 64x64 + 64 + 64x5 + 5 */

typedef enum {
    SPMV_OK = 0,
    SPMV_ERR_INVALID_ARG = -1,    /* null pointer, bad size, malformed CSR, bad parameter */
    SPMV_ERR_INDEX_OVERFLOW = -2, /* a count or padded size does not fit the index type */
    SPMV_ERR_TOO_LARGE = -3,      /* padded footprint above spmv_params.max_bytes */
    SPMV_ERR_CUDA = -4,           /* a CUDA runtime call failed (detail in spmv_last_error) */
    SPMV_ERR_NO_MODEL = -5,       /* spmv_select without a model */
    SPMV_ERR_ALLOC = -6,          /* device allocation failed */
    SPMV_ERR_WRONG_FORMAT = -7    /* call not valid for this handle's format */
} spmv_status;

/* A CSR matrix in device memory (Sec. II-B "CSR"): ptr[M+1], idx[nnz],
 * val[nnz].  Columns need not be sorted within a row; duplicates are kept and
 * summed by every product.  The caller keeps the arrays alive for the duration
 * of the call that receives them (convert copies what it needs). */
typedef struct {
    int32_t m, n;
    int64_t nnz;
    const int32_t* ptr;
    const int32_t* idx;
    const double* val;
} spmv_csr;

/* Tuning parameters.  A zero field means "choose automatically".  The
 * paper names them: CSR5 tile width omega and height sigma (Sec. II-B "CSR5"),
 * SELL slice height C and sorting scope sigma (Sec. II-B "SELL"), and the HYB
 * ELL width K (Sec. II-B "HYB"). */
typedef struct {
    int32_t sell_C;        /* SELL slice height: 32, 64 or 128 rows (0 -> 32) */
    int32_t sell_sigma;    /* SELL sorting window in rows: 1 (plain SELL), a multiple of sell_C,
                              or -1 for the whole matrix (0 -> the whole matrix) */
    int32_t csr5_omega;    /* CSR5 tile width: 32, the warp width, is the only value (0 -> 32) */
    int32_t csr5_sigma;    /* CSR5 tile height, 1..32 (0 -> 32) */
    int32_t csr_block_nnz; /* CSR product: 352 = warp tiles of 352 nonzeros (any mix of row lengths);
                              -V (V = 2, 4, 8, 16, 32) = V lanes per row (rows of similar length);
                              0 = automatic: V lanes when the longest row is at most twice the mean
                              plus 8, V the smallest power of two >= mean / 8 in [2, 16], else tiles */
    int32_t hyb_k;         /* HYB ELL width: > 0 explicit, 0 -> the typical-length rule,
                              SPMV_HYB_K_NONE -> every entry in the COO part */
    int32_t sell_panel_cols; /* SELL column panels (not in the paper): columns per panel.  The matrix
                              is split by columns into panels, each a SELL matrix of its own, and
                              y = sum over panels of A_p x_p (in panel order), so that each panel's
                              part of x stays in L2.  The panels share one row order (rows longer
                              than 32 entries first, then windows of min(sell_sigma, 2^16) rows,
                              each sorted by the rows' panel lengths), so the partial sums stay in
                              that order; a last pass writes y in row order.  > 0 explicit (at most
                              256 panels, else INVALID_ARG), SPMV_SELL_PANELS_NONE -> one panel,
                              0 -> panels of at most 64 MiB of x when x exceeds 96 MiB */
    int64_t max_bytes;     /* cap on the handle's device footprint (0 -> 90% of free memory) */
} spmv_params;

#define SPMV_HYB_K_NONE (-1)
#define SPMV_SELL_SIGMA_ALL (-1)
#define SPMV_SELL_PANELS_NONE (-1)

typedef struct spmv_handle spmv_handle;
typedef struct spmv_model spmv_model;
typedef struct spmv_batch spmv_batch;

/* What a handle holds, after automatic choices are resolved. */
typedef struct {
    int32_t fmt, m, n;
    int64_t nnz;
    int64_t device_bytes;   /* memory owned by the handle */
    int64_t stored_slots;   /* value slots stored, padding included */
    spmv_params params;     /* resolved tuning parameters (hyb_k: the K used) */
    int64_t aux[4];         /* format detail (see spmv_handle_array for the arrays):
                               CSR  {warp tiles, lanes per row (0: the tiles run), 0, 0}
                               CSR5 {tiles, tiles listing their rows, empty rows, 0}
                               ELL  {K, rows left to whole blocks, their length threshold, 0}
                               SELL {slices, warp units, longest row, column panels: 0 one
                                     panel; -1 one panel whose sort moved no row, so that
                                     the product writes y without reading perm}
                               HYB  {COO tail entries, tail rows, K, tail warp tiles} */
} spmv_info;

/* ---------------------------------------------------------------- basics */

SPMV_API int spmv_version(void);
SPMV_API const char* spmv_strerror(int status);
/* One-line detail of the calling thread's last failed call ("" if none). */
SPMV_API const char* spmv_last_error(void);

/* -------------------------------------------------------- conversion, run */

/* Build a handle holding A in format `fmt` (Sec. II-B layouts; Sec. III-D and
 * Algorithm 1 convert once and then multiply many times).  The CSR input is
 * validated on the device first (ptr[0] = 0, ptr non-decreasing, ptr[M] = nnz,
 * 0 <= idx < N); a violation returns SPMV_ERR_INVALID_ARG.  params may be
 * NULL (all automatic).  Synchronises `stream` (it reads sizes back).
 * The handle owns copies of everything it needs; free it with spmv_free.
 * Errors: INVALID_ARG, INDEX_OVERFLOW (nnz >= 2^31: the row pointers are
 * int32; checked on the host before the CSR is read; padded layouts use 64-bit
 * offsets), TOO_LARGE (footprint > max_bytes), ALLOC, CUDA. */
SPMV_API int spmv_convert(spmv_fmt fmt, const spmv_csr* csr, const spmv_params* params, cudaStream_t stream,
                 spmv_handle** out);

/* y = A x (Sec. II-A), y overwritten (beta = 0).  x holds N doubles and y M
 * doubles, both device memory.  Asynchronous on `stream`; no host sync, no
 * allocation (the call can be captured into a CUDA graph).  Launches the
 * format's kernels: one (CSR, CSR5, ELL, SELL), two (HYB with a COO tail),
 * or one per column panel, in panel order, and one putting y in row order
 * (SELL in panels).  They are
 * launched with programmatic stream serialization: their blocks may become
 * resident while the kernel ahead of them in `stream` finishes, and each
 * waits for that kernel to complete (its writes visible) before it touches
 * memory, so stream order holds as for an ordinary launch.  Runs of one
 * handle must not overlap on the GPU (they share the handle's small scratch
 * for rows split across warps); runs of different handles may. */
SPMV_API int spmv_run(const spmv_handle* h, const double* x, double* y, cudaStream_t stream);

/* Write A back as CSR (ptr[M+1], idx[nnz], val[nnz], device, caller-owned).
 * The round trip is exact: same ptr, same column order within each row, same
 * value bits (explicit zeros, -0.0 and duplicates included).  Asynchronous. */
SPMV_API int spmv_to_csr(const spmv_handle* h, int32_t* ptr, int32_t* idx, double* val, cudaStream_t stream);

SPMV_API int spmv_handle_info(const spmv_handle* h, spmv_info* out);

/* Device pointer and element count of one of the handle's arrays, by name,
 * for inspection (e.g. "tile_ptr", "flags", "y_off", "seg_off", "tile_idx",
 * "tile_val", "empty_ptr", "empty_rows", "row_len", "col", "val", "perm",
 * "slice_ptr", "tail_rows", "tail_ptr", "tail_col", "tail_val", "units",
 * "ptr", "idx").  The memory stays owned by the handle.  Returns
 * INVALID_ARG for a name the format does not have. */
SPMV_API int spmv_handle_array(const spmv_handle* h, const char* name, const void** dev_ptr, int64_t* count,
                      int32_t* elem_bytes);

SPMV_API void spmv_free(spmv_handle* h);

/* ------------------------------------------------- features and selection */

/* The 16 static features of Sec. V-B (Table IV's eight plus eight more) as
 * float32 into feat_dev[16] (device memory): 0 n_rows, 1 n_cols, 2 nnz/(M*N),
 * 3 min, 4 max, 5 mean, 6 std of the row length, 7 std/mean, 8 log2 nnz,
 * 9 mean/max, 10 HYB tail fraction, 11 mean and 12 max |col - row| over each
 * row's first 16 entries, 13 empty-row fraction, 14 fraction of rows of length
 * >= 32, 15 SELL-32 fill.  Features 3-7, 9, 13 and 14 are exact over all M
 * rows (one pass over ptr); 10, 11, 12 and 15 come from rows floor(k*M/8192),
 * k < 8192, when M > 8192 (all rows otherwise), so their cost does not grow
 * with M.  csr->idx holds csr->nnz entries and needs no particular alignment.
 * The CSR must be well formed (ptr[0] = 0, non-decreasing, ptr[M] = nnz, as
 * spmv_convert checks); this call does not check it.  Two kernel launches
 * (the pass over ptr, then a thread-block cluster), asynchronous.  The pass
 * over ptr reduces into one slot of a small static device array of the
 * library (64 slots per device, taken in turn by the calls): at most 64
 * features or selection calls may be in flight on one device at once, and a
 * CUDA graph that captured such a call replays its slot, so replays of that
 * graph must not overlap each other on the GPU.  The first call on a device
 * looks up the array's address; make it before any stream capture. */
SPMV_API int spmv_features(const spmv_csr* csr, float* feat_dev, cudaStream_t stream);

/* A trained selector: network parameters (SPMV_MLP_PARAMS floats, W1, b1, W2,
 * b2, W3, b3 row-major) and the per-feature minimum and maximum of the
 * transformed training features (Sec. V-B "Feature Scaling"), host arrays
 * copied to the device.  The model's footprint cap for selection (see
 * spmv_select_async) starts at 90% of the device memory free at creation. */
SPMV_API int spmv_model_create(const float* params_host, const float* lo_host, const float* hi_host, spmv_model** out);
SPMV_API void spmv_model_free(spmv_model* m);

/* Sets the model's footprint cap for selection, in bytes (> 0). */
SPMV_API int spmv_model_set_max_bytes(spmv_model* m, int64_t max_bytes);

/* Features + scaling + network + argmax (Sec. V-A deployment: features in,
 * representation label out), the launches of spmv_features.  Writes the
 * format id to fmt_dev[0] and, if logits_dev is not NULL, the 5 logits.
 * The argmax never names ELL when ELL's padded layout (ceil(M/4)*4 rows of
 * max-row-length slots of 12 bytes, plus 4 bytes per row; exact, from the
 * longest row) exceeds the model's cap: it is then taken over the other
 * four formats, whose layouts stay within a small multiple of the CSR's.
 * Asynchronous. */
SPMV_API int spmv_select_async(const spmv_csr* csr, const spmv_model* model, int32_t* fmt_dev, float* logits_dev,
                      cudaStream_t stream);

/* As spmv_select_async, then waits for `stream` and returns the id in *out. */
SPMV_API int spmv_select(const spmv_csr* csr, const spmv_model* model, cudaStream_t stream, spmv_fmt* out);

/* --------------------------------------------------- selector training */

/* Sec. V-B "Feature Scaling" on the device: X[b][j] = clamp((t_j - lo_j) /
 * (hi_j - lo_j), 0, 1), t the transformed feature (log2(1+f) for sizes and
 * counts, -log2(max(f, 2^-60)) for nnz_frac), 0 where hi_j == lo_j.
 * feat_dev and X_dev are B x 16 row-major; lo/hi are device float[16]. */
SPMV_API int spmv_mlp_scale(const float* feat_dev, const float* lo_dev, const float* hi_dev, int32_t B, float* X_dev,
                   cudaStream_t stream);

/* Mean cross-entropy over B samples and its gradient with respect to all
 * SPMV_MLP_PARAMS parameters (one CTA, deterministic).  X_dev is B x 16,
 * labels_dev B ints in [0, 5).  loss_dev may be NULL. */
SPMV_API int spmv_mlp_loss_grad(const float* theta_dev, const float* X_dev, const int32_t* labels_dev, int32_t B,
                       float* grad_dev, float* loss_dev, cudaStream_t stream);

/* One Adam step (step number t >= 1) on n parameters, in place. */
SPMV_API int spmv_mlp_adam(float* theta_dev, const float* grad_dev, float* m_dev, float* v_dev, int32_t n, int32_t t,
                  float lr, float beta1, float beta2, float eps, cudaStream_t stream);

/* `steps` full-batch Adam steps (numbered t0+1 ... t0+steps) in one launch;
 * loss_hist_dev (may be NULL) receives each step's loss. */
SPMV_API int spmv_mlp_train(float* theta_dev, float* m_dev, float* v_dev, const float* X_dev, const int32_t* labels_dev,
                   int32_t B, int32_t steps, int32_t t0, float lr, float beta1, float beta2, float eps,
                   float* loss_hist_dev, cudaStream_t stream);

/* Logits (B x 5, may be NULL) and argmax labels (may be NULL). */
SPMV_API int spmv_mlp_forward(const float* theta_dev, const float* X_dev, int32_t B, float* logits_dev,
                     int32_t* pred_dev, cudaStream_t stream);

/* ------------------------------------------------- x and y in host memory */

/* Products whose x and y live in host memory (Sec. II-A's y = A x with the
 * copies in and out included).  An spmv_host_io holds, for one handle, two
 * device staging pairs (x: N doubles, y: M doubles) and two copy streams of
 * its own (in and out).  create allocates them on the handle's device (so it
 * is not for stream capture); the handle must outlive the io.  Errors:
 * INVALID_ARG, ALLOC, CUDA. */
typedef struct spmv_host_io spmv_host_io;
SPMV_API int spmv_host_io_create(const spmv_handle* h, spmv_host_io** out);

/* y_host = A x_host.  Copies x_host (N doubles) into a staging buffer on the
 * copy-in stream, runs spmv_run on `stream` once that copy is done, and
 * copies y to y_host (M doubles) on the copy-out stream once the product is
 * done.  Calls alternate between the two staging pairs, so one call's copies
 * overlap the products of the calls before and after it; a call waits on the
 * device (never on the host) for the call two before it to release its pair.
 * Returns at once.  `done` (may be NULL): an event recorded after the copy
 * out; once it has completed, y_host holds y and x_host may be rewritten.
 * With pinned host memory the copies are asynchronous; pageable memory works,
 * with copies that CUDA may stage.  Calls on one io must come from one host
 * thread at a time; products of one handle run in call order.  Errors:
 * INVALID_ARG (NULL io or buffers), CUDA. */
SPMV_API int spmv_run_host(spmv_host_io* io, const double* x_host, double* y_host, cudaStream_t stream,
                           cudaEvent_t done);

/* Blocks the host until every copy out issued through `io` has completed. */
SPMV_API int spmv_host_io_sync(spmv_host_io* io);

/* Waits for the io's copies, then releases its buffers and streams. */
SPMV_API void spmv_host_io_free(spmv_host_io* io);

/* ------------------------------------------------------------- batching */

/* Many independent products y_b = A_b x_b in one CUDA graph of persistent
 * launches, one per task family present: CSR5, ELL, the ELL part of HYB, CSR
 * on the lanes-per-row path and CSR without nonzeros; SELL with C = 32; with
 * C = 64; with C = 128; CSR tiles; HYB tails.  Every matrix's y equals its own
 * spmv_run bit for bit (the same arithmetic in the same order).  build lays
 * out the work lists over all handles (each keeps its own format) and
 * captures the launches on a stream of its own; the handles must outlive the
 * batch.  A SELL handle in column panels is refused
 * (INVALID_ARG): its panels must run one after another.  Synchronises. */
SPMV_API int spmv_batch_build(spmv_handle* const* handles, int32_t count, cudaStream_t stream, spmv_batch** out);

/* spmv_batch_build with options.  flags: 0 (the kernels per task family
 * above) or SPMV_BATCH_ONE_LAUNCH: one persistent kernel for every task but
 * the HYB tails (which still follow in a launch of their own when present),
 * with the largest family's register budget; SELL tasks pick their slice
 * height at run time and CSR tile tasks share the launch's shared memory.
 * The same products, bit for bit.  Unknown flags: INVALID_ARG. */
#define SPMV_BATCH_ONE_LAUNCH 1
SPMV_API int spmv_batch_build_ex(spmv_handle* const* handles, int32_t count, int32_t flags, cudaStream_t stream,
                                 spmv_batch** out);

/* Kernels one spmv_batch_run replays (the task families present, or one
 * plus the HYB tails' under SPMV_BATCH_ONE_LAUNCH). */
SPMV_API int spmv_batch_launches(const spmv_batch* b, int32_t* out);

/* xs_host[b] / ys_host[b]: device pointers of x_b and y_b (host arrays of
 * `count` pointers).  Uploads them when they differ from the previous call,
 * then replays the graph.  Asynchronous. */
SPMV_API int spmv_batch_run(spmv_batch* b, const double* const* xs_host, double* const* ys_host, cudaStream_t stream);

/* The same products as `count` ordinary per-matrix spmv_run launches,
 * captured once in their own CUDA graph and replayed (the comparison point). */
SPMV_API int spmv_batch_run_separate(spmv_batch* b, const double* const* xs_host, double* const* ys_host,
                            cudaStream_t stream);

SPMV_API void spmv_batch_free(spmv_batch* b);

/* ------------------------------------------------ allocation-free product */

/* y = A x straight from a caller's device CSR (no handle), allocating no
 * device memory at all.  For callers that cannot call cudaMalloc when they
 * need the product: code running under a memory manager that has already
 * reserved every device byte (a framework's caching allocator, an
 * application's own pool), and latency-critical paths that must not enter
 * the CUDA allocator, whose calls can synchronise the whole device.  The
 * paper has no counterpart: it is an interface of this library, computing
 * the same y as spmv_run on a CSR handle (within the FP64 tolerance; bit for
 * bit on integer-valued inputs).
 *  - csr, x, y: device arrays owned by the caller, layout as for spmv_convert;
 *    the CSR is not validated (pass one that spmv_convert accepts).
 *  - Scratch: a static device array of this library (6 MiB, held by every
 *    GPU that loads the library until the process exits); at most
 *    536,870,912 nonzeros, SPMV_ERR_TOO_LARGE beyond.
 *  - The first call on each device looks up that array's device address;
 *    make the first call on a device before any stream capture.
 *  - All calls share the one array and keep nothing between calls; calls
 *    whose kernels overlap on the GPU (different streams, no ordering) race.
 *  - Asynchronous on `stream`; two kernel launches. */
SPMV_API int spmv_csr_run_noalloc(const spmv_csr* csr, const double* x, double* y, cudaStream_t stream);

/* --------------------------------------------------------- fault testing */

/* Make the k-th device allocation from now fail with SPMV_ERR_ALLOC
 * (k >= 1; 0 disables).  For testing error paths; process-wide. */
SPMV_API void spmv_debug_fail_alloc(int32_t k);

/* Force the cluster size of the features kernel: 8 or 16 CTAs (0 restores the
 * automatic choice: 16 where the device can place such a cluster, else 8).
 * Both sizes compute the same features bit for bit; this lets a test run
 * each.  Process-wide.  A forced size the device cannot place makes the
 * features calls return SPMV_ERR_CUDA. */
SPMV_API void spmv_debug_features_cluster(int32_t ctas);

#ifdef __cplusplus
}
#endif

#endif /* SPMV_GB300_H */
