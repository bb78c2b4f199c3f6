// md_io.cu -- asynchronous state download (md_state_stream_*, include/md.h).
//
// For trajectory output while a context keeps stepping: each push takes a
// snapshot of x and v (original atom order, FP64 AoS) into one of two device
// slots on the context's stream, in stream order, and queues the copy of that
// slot to the caller's host buffers on the object's own stream.  A slot is
// reused only after its previous copy has finished (an event the context's
// stream waits on), so at most two downloads are in flight and the context's
// stream never waits for a copy it does not have to.
#include <new>
#include <string>

#include "md_common.cuh"

namespace mdb {  // md_api.cu
bool is_device_pointer(const void *p);
}  // namespace mdb

using namespace mdb;

struct md_state_stream {
    md_ctx *ctx = nullptr;
    cudaStream_t side = nullptr;
    double *slot[2] = {nullptr, nullptr};   // each: x (3n) then v (3n)
    cudaEvent_t taken[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
    int next = 0;
    std::string err;
};

namespace {

thread_local std::string g_io_error;

md_status io_fail(md_state_stream *s, md_status st, const std::string &msg) {
    if (s) s->err = msg;
    else g_io_error = msg;
    return st;
}

md_status io_cuda(md_state_stream *s, cudaError_t e, const char *where) {
    return io_fail(s, e == cudaErrorMemoryAllocation ? MD_ERR_NOMEM : MD_ERR_CUDA,
                   std::string(where) + ": " + cudaGetErrorString(e));
}

#define ICK(call)                                              \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return io_cuda(s, e_, #call);   \
    } while (0)

void io_destroy(md_state_stream *s) {
    if (s->side) cudaStreamSynchronize(s->side);
    for (int b = 0; b < 2; ++b) {
        if (s->slot[b]) cudaFree(s->slot[b]);
        if (s->taken[b]) cudaEventDestroy(s->taken[b]);
        if (s->done[b]) cudaEventDestroy(s->done[b]);
    }
    if (s->side) cudaStreamDestroy(s->side);
    cudaGetLastError();
}

md_status io_init(md_state_stream *s, md_ctx *c) {
    s->ctx = c;
    const size_t n = (size_t)c->n_total;
    for (int b = 0; b < 2; ++b) {
        ICK(cudaMalloc(reinterpret_cast<void **>(&s->slot[b]), 6 * n * sizeof(double)));
        ICK(cudaEventCreateWithFlags(&s->taken[b], cudaEventDisableTiming));
        ICK(cudaEventCreateWithFlags(&s->done[b], cudaEventDisableTiming));
    }
    ICK(cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking));
    return MD_OK;
}

}  // namespace

extern "C" {

md_status md_state_stream_create(md_ctx *ctx, md_state_stream **out) {
    if (!out) return io_fail(nullptr, MD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!ctx) return io_fail(nullptr, MD_ERR_ARG, "ctx is NULL");
    md_state_stream *s = new (std::nothrow) md_state_stream();
    if (!s) return io_fail(nullptr, MD_ERR_NOMEM, "host allocation failed");
    md_status st = io_init(s, ctx);
    if (st != MD_OK) {
        g_io_error = s->err;
        io_destroy(s);   // also clears a failed allocation's pending error
        delete s;
        return st;
    }
    *out = s;
    return MD_OK;
}

md_status md_state_stream_push(md_state_stream *s, double *x, double *v) {
    if (!s) return io_fail(nullptr, MD_ERR_ARG, "NULL state stream");
    md_ctx *c = s->ctx;
    if (!c->ready) return io_fail(s, MD_ERR_ARG, "internal: state between half-steps");
    if (!x && !v) return MD_OK;
    const size_t n = (size_t)c->n_total, bytes = 3 * n * sizeof(double);
    const int b = s->next;
    s->next ^= 1;
    double *sx = s->slot[b], *sv = s->slot[b] + 3 * n;
    // the slot's previous copy must be done before the snapshot overwrites it
    ICK(cudaStreamWaitEvent(c->stream, s->done[b], 0));
    ICK(launch_get_state(c, x ? sx : nullptr, v ? sv : nullptr, nullptr, nullptr, nullptr,
                         nullptr));
    ICK(cudaEventRecord(s->taken[b], c->stream));
    ICK(cudaStreamWaitEvent(s->side, s->taken[b], 0));
    if (x) ICK(cudaMemcpyAsync(x, sx, bytes, is_device_pointer(x) ? cudaMemcpyDeviceToDevice
                                                                   : cudaMemcpyDeviceToHost,
                               s->side));
    if (v) ICK(cudaMemcpyAsync(v, sv, bytes, is_device_pointer(v) ? cudaMemcpyDeviceToDevice
                                                                   : cudaMemcpyDeviceToHost,
                               s->side));
    ICK(cudaEventRecord(s->done[b], s->side));
    return MD_OK;
}

md_status md_state_stream_wait(md_state_stream *s) {
    if (!s) return io_fail(nullptr, MD_ERR_ARG, "NULL state stream");
    ICK(cudaStreamSynchronize(s->side));
    return MD_OK;
}

const char *md_state_stream_last_error(const md_state_stream *s) {
    return s ? s->err.c_str() : g_io_error.c_str();
}

void md_state_stream_destroy(md_state_stream *s) {
    if (!s) return;
    io_destroy(s);
    delete s;
}

}  // extern "C"
