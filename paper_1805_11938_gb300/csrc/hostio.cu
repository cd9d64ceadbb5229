// Products with x and y in host memory: two device staging pairs per io,
// used in turn, and two copy streams, so that the copies of one call overlap
// the products of the calls around it.  Ordering is carried by events only
// (no host synchronisation on the call path):
//   copy in  (call i, pair b): waits until product i-2 has read x[b]
//   product  (call i):         waits for its copy in and for copy out i-2 (y[b] free)
//   copy out (call i):         waits for product i
#include "internal.cuh"

using namespace spmv;

struct spmv_host_io {
    const spmv_handle* h = nullptr;
    int device = 0;
    double* x[2] = {nullptr, nullptr};
    double* y[2] = {nullptr, nullptr};
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t copied_in[2] = {nullptr, nullptr};
    cudaEvent_t computed[2] = {nullptr, nullptr};
    cudaEvent_t copied_out[2] = {nullptr, nullptr};
    int64_t calls = 0;

    ~spmv_host_io() {
        if (in) cudaStreamSynchronize(in);
        if (out) cudaStreamSynchronize(out);
        for (int b = 0; b < 2; ++b) {
            if (computed[b]) cudaEventSynchronize(computed[b]);
            if (copied_in[b]) cudaEventDestroy(copied_in[b]);
            if (computed[b]) cudaEventDestroy(computed[b]);
            if (copied_out[b]) cudaEventDestroy(copied_out[b]);
            dev_free(x[b]);
            dev_free(y[b]);
        }
        if (in) cudaStreamDestroy(in);
        if (out) cudaStreamDestroy(out);
    }
};

extern "C" {

int spmv_host_io_create(const spmv_handle* h, spmv_host_io** out) {
    if (!out) return set_error(SPMV_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!h) return set_error(SPMV_ERR_INVALID_ARG, "handle is NULL");
    int dev = 0;
    SPMV_CUDA(cudaGetDevice(&dev));
    if (dev != h->device)
        return set_error(SPMV_ERR_INVALID_ARG, "the current device (%d) is not the handle's (%d)", dev, h->device);
    spmv_host_io* io = new spmv_host_io();
    io->h = h;
    io->device = dev;
    int st = SPMV_OK;
    for (int b = 0; b < 2 && st == SPMV_OK; ++b) {
        st = dev_malloc(reinterpret_cast<void**>(&io->x[b]), sizeof(double) * (size_t)h->n);
        if (st == SPMV_OK) st = dev_malloc(reinterpret_cast<void**>(&io->y[b]), sizeof(double) * (size_t)h->m);
    }
    cudaError_t e = cudaSuccess;
    if (st == SPMV_OK) e = cudaStreamCreateWithFlags(&io->in, cudaStreamNonBlocking);
    if (st == SPMV_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&io->out, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && st == SPMV_OK && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&io->copied_in[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->computed[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->copied_out[b], cudaEventDisableTiming);
    }
    if (st == SPMV_OK && e != cudaSuccess) st = cuda_error(e, "spmv_host_io_create");
    if (st != SPMV_OK) {
        delete io;
        return st;
    }
    *out = io;
    return SPMV_OK;
}

int spmv_run_host(spmv_host_io* io, const double* x_host, double* y_host, cudaStream_t stream, cudaEvent_t done) {
    if (!io) return set_error(SPMV_ERR_INVALID_ARG, "io is NULL");
    if (!x_host || !y_host) return set_error(SPMV_ERR_INVALID_ARG, "x_host or y_host is NULL");
    const spmv_handle* h = io->h;
    const int b = (int)(io->calls & 1);
    // copy in: pair b's x is free once the product two calls back has run
    SPMV_CUDA(cudaStreamWaitEvent(io->in, io->computed[b], 0));
    SPMV_CUDA(cudaMemcpyAsync(io->x[b], x_host, sizeof(double) * (size_t)h->n, cudaMemcpyHostToDevice, io->in));
    SPMV_CUDA(cudaEventRecord(io->copied_in[b], io->in));
    // product: after its copy in, and after pair b's y has been copied out
    SPMV_CUDA(cudaStreamWaitEvent(stream, io->copied_in[b], 0));
    SPMV_CUDA(cudaStreamWaitEvent(stream, io->copied_out[b], 0));
    SPMV_TRY(spmv_run(h, io->x[b], io->y[b], stream));
    SPMV_CUDA(cudaEventRecord(io->computed[b], stream));
    // copy out
    SPMV_CUDA(cudaStreamWaitEvent(io->out, io->computed[b], 0));
    SPMV_CUDA(cudaMemcpyAsync(y_host, io->y[b], sizeof(double) * (size_t)h->m, cudaMemcpyDeviceToHost, io->out));
    SPMV_CUDA(cudaEventRecord(io->copied_out[b], io->out));
    if (done) SPMV_CUDA(cudaEventRecord(done, io->out));
    ++io->calls;
    return SPMV_OK;
}

int spmv_host_io_sync(spmv_host_io* io) {
    if (!io) return set_error(SPMV_ERR_INVALID_ARG, "io is NULL");
    SPMV_CUDA(cudaStreamSynchronize(io->out));
    return SPMV_OK;
}

void spmv_host_io_free(spmv_host_io* io) { delete io; }

}  // extern "C"
