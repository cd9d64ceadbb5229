// The C ABI: argument checks, dispatch to the per-format code, handle
// bookkeeping.  Every entry point returns an spmv_status.
#include <cstring>
#include <memory>

#include "internal.cuh"

namespace spmv {
const char* last_error();
void clear_error();
void debug_fail_alloc(int k);
void debug_features_cluster(int ctas);
}  // namespace spmv

using namespace spmv;

extern "C" {

int spmv_version(void) { return 100; }

const char* spmv_strerror(int status) {
    switch (status) {
        case SPMV_OK: return "ok";
        case SPMV_ERR_INVALID_ARG: return "invalid argument";
        case SPMV_ERR_INDEX_OVERFLOW: return "index overflow";
        case SPMV_ERR_TOO_LARGE: return "footprint above the cap";
        case SPMV_ERR_CUDA: return "CUDA error";
        case SPMV_ERR_NO_MODEL: return "no model";
        case SPMV_ERR_ALLOC: return "device allocation failed";
        case SPMV_ERR_WRONG_FORMAT: return "wrong format for this call";
        default: return "unknown status";
    }
}

const char* spmv_last_error(void) { return last_error(); }

void spmv_debug_fail_alloc(int32_t k) { debug_fail_alloc(k); }

void spmv_debug_features_cluster(int32_t ctas) { debug_features_cluster(ctas); }

int spmv_convert(spmv_fmt fmt, const spmv_csr* csr, const spmv_params* params, cudaStream_t stream,
                 spmv_handle** out) {
    clear_error();
    if (!out) return set_error(SPMV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if ((int)fmt < 0 || (int)fmt >= SPMV_NUM_FORMATS) return set_error(SPMV_ERR_INVALID_ARG, "unknown format %d", (int)fmt);
    if (!csr) return set_error(SPMV_ERR_INVALID_ARG, "csr is NULL");
    if (csr->m <= 0 || csr->n <= 0) return set_error(SPMV_ERR_INVALID_ARG, "m and n must be positive (m=%d n=%d)", csr->m, csr->n);
    SPMV_TRY(validate_csr(csr, stream));
    std::unique_ptr<spmv_handle> h(new spmv_handle());
    h->fmt = (int32_t)fmt;
    h->m = csr->m;
    h->n = csr->n;
    h->nnz = csr->nnz;
    if (params) h->params = *params;
    SPMV_CUDA(cudaGetDevice(&h->device));
    int st = SPMV_OK;
    switch (fmt) {
        case SPMV_CSR: st = csr_convert(h.get(), csr, stream); break;
        case SPMV_CSR5: st = csr5_convert(h.get(), csr, stream); break;
        case SPMV_ELL: st = ell_convert(h.get(), csr, stream); break;
        case SPMV_SELL: st = sell_convert(h.get(), csr, stream); break;
        case SPMV_HYB: st = hyb_convert(h.get(), csr, stream); break;
    }
    if (st != SPMV_OK) {
        cudaStreamSynchronize(stream);
        return st;
    }
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_error(e, "spmv_convert");
    if (h->params.max_bytes <= 0) h->params.max_bytes = resolve_cap(h->params);
    *out = h.release();
    return SPMV_OK;
}

int spmv_run(const spmv_handle* h, const double* x, double* y, cudaStream_t stream) {
    if (!h) return set_error(SPMV_ERR_INVALID_ARG, "handle is NULL");
    if (!x || !y) return set_error(SPMV_ERR_INVALID_ARG, "x or y is NULL");
    if ((const void*)x == (const void*)y) return set_error(SPMV_ERR_INVALID_ARG, "x and y must not alias");
    switch (h->fmt) {
        case SPMV_CSR: return csr_run(h, x, y, stream);
        case SPMV_CSR5: return csr5_run(h, x, y, stream);
        case SPMV_ELL: return ell_run(h, x, y, stream);
        case SPMV_SELL: return sell_run(h, x, y, stream);
        case SPMV_HYB: return hyb_run(h, x, y, stream);
    }
    return set_error(SPMV_ERR_INVALID_ARG, "corrupt handle");
}

int spmv_to_csr(const spmv_handle* h, int32_t* ptr, int32_t* idx, double* val, cudaStream_t stream) {
    if (!h) return set_error(SPMV_ERR_INVALID_ARG, "handle is NULL");
    if (!ptr || (h->nnz > 0 && (!idx || !val))) return set_error(SPMV_ERR_INVALID_ARG, "output array is NULL");
    switch (h->fmt) {
        case SPMV_CSR:
            SPMV_CUDA(cudaMemcpyAsync(ptr, h->ptr, sizeof(int32_t) * ((size_t)h->m + 1), cudaMemcpyDeviceToDevice, stream));
            if (h->nnz > 0) {
                SPMV_CUDA(cudaMemcpyAsync(idx, h->idx, sizeof(int32_t) * (size_t)h->nnz, cudaMemcpyDeviceToDevice, stream));
                SPMV_CUDA(cudaMemcpyAsync(val, h->val, sizeof(double) * (size_t)h->nnz, cudaMemcpyDeviceToDevice, stream));
            }
            return SPMV_OK;
        case SPMV_CSR5: return csr5_to_csr(h, ptr, idx, val, stream);
        case SPMV_ELL: return ell_to_csr(h, ptr, idx, val, stream);
        case SPMV_SELL: return sell_to_csr(h, ptr, idx, val, stream);
        case SPMV_HYB: return hyb_to_csr(h, ptr, idx, val, stream);
    }
    return set_error(SPMV_ERR_INVALID_ARG, "corrupt handle");
}

int spmv_handle_info(const spmv_handle* h, spmv_info* out) {
    if (!h || !out) return set_error(SPMV_ERR_INVALID_ARG, "NULL argument");
    out->fmt = h->fmt;
    out->m = h->m;
    out->n = h->n;
    out->nnz = h->nnz;
    out->device_bytes = h->device_bytes;
    out->stored_slots = h->stored_slots;
    out->params = h->params;
    for (int i = 0; i < 4; ++i) out->aux[i] = h->aux[i];
    return SPMV_OK;
}

int spmv_handle_array(const spmv_handle* h, const char* name, const void** dev_ptr, int64_t* count,
                      int32_t* elem_bytes) {
    if (!h || !name || !dev_ptr || !count || !elem_bytes) return set_error(SPMV_ERR_INVALID_ARG, "NULL argument");
    auto it = h->arrays.find(name);
    if (it == h->arrays.end()) return set_error(SPMV_ERR_INVALID_ARG, "format %d has no array '%s'", h->fmt, name);
    *dev_ptr = it->second.ptr;
    *count = it->second.count;
    *elem_bytes = it->second.elem_bytes;
    return SPMV_OK;
}

void spmv_free(spmv_handle* h) { delete h; }

}  // extern "C"
