// grace_step on host buffers: the upload of the state and the time steps, the
// SSP-RK3 steps (eq. RK3) of grace_step, and the download of the result, in one
// call whose copies run on two copy streams owned by the batch.
//
// Device staging is double-buffered: call i steps slot i mod 2, so the upload of
// call i+1 and the download of call i-1 overlap the steps of call i when the host
// buffers are page-locked.  Slot s is reused only after its previous download has
// finished (event `freed`).  grace_step_host_wait joins both copy streams.
#include <new>

#include "grace_internal.h"

namespace grace {

namespace {

struct HostIo {
    size_t n_doubles = 0;          // coefficients of the whole batch
    double *d_g[2] = {nullptr, nullptr};
    double *d_dt[2] = {nullptr, nullptr};
    double *d_mass[2] = {nullptr, nullptr};
    unsigned char *d_flags[2] = {nullptr, nullptr};
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t uploaded[2] = {nullptr, nullptr}, stepped[2] = {nullptr, nullptr},
                freed[2] = {nullptr, nullptr};
    int next = 0;
    // the previous call's output: an input overlapping it must wait for its download
    const char *last_out = nullptr;
    size_t last_bytes = 0;
    int last_slot = -1;
};

bool overlaps(const void *a, size_t na, const char *b, size_t nb)
{
    const char *pa = static_cast<const char *>(a);
    return b && pa < b + nb && b < pa + na;
}

void destroy_io(HostIo *io)
{
    if (!io) return;
    if (io->up) cudaStreamSynchronize(io->up);
    if (io->down) cudaStreamSynchronize(io->down);
    for (int s = 0; s < 2; ++s) {
        cudaFree(io->d_g[s]);
        cudaFree(io->d_dt[s]);
        cudaFree(io->d_mass[s]);
        cudaFree(io->d_flags[s]);
        if (io->uploaded[s]) cudaEventDestroy(io->uploaded[s]);
        if (io->stepped[s]) cudaEventDestroy(io->stepped[s]);
        if (io->freed[s]) cudaEventDestroy(io->freed[s]);
    }
    if (io->up) cudaStreamDestroy(io->up);
    if (io->down) cudaStreamDestroy(io->down);
    delete io;
}

cudaError_t create_io(grace_batch *b, HostIo **out)
{
    HostIo *io = new (std::nothrow) HostIo;
    if (!io) return cudaErrorMemoryAllocation;
    const size_t n = (size_t)b->n_cells;
    io->n_doubles = (size_t)b->h_off[n];
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
        e = cudaMalloc(&io->d_g[s], io->n_doubles * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&io->d_dt[s], n * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&io->d_mass[s], n * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&io->d_flags[s], n);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->uploaded[s], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->stepped[s], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->freed[s], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&io->up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&io->down, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        destroy_io(io);
        return e;
    }
    *out = io;
    return cudaSuccess;
}

}  // namespace

void free_host_io(grace_batch *b)
{
    destroy_io(static_cast<HostIo *>(b->host_io));
    b->host_io = nullptr;
}

}  // namespace grace

using namespace grace;

extern "C" {

grace_status grace_step_host(grace_batch *b, const double *h_g, double *h_out, const double *h_dt, int n_steps,
                             int prec, double *h_mass, unsigned char *h_flags)
{
    if (!b || !h_g || !h_out || !h_dt || n_steps < 0) {
        set_error("grace_step_host: null argument or negative step count");
        return GRACE_ERR_ARG;
    }
    Guard guard(b->ctx->device);
    if (!b->host_io) {
        HostIo *io = nullptr;
        cudaError_t e = create_io(b, &io);
        if (e != cudaSuccess) return cuda_fail(e, "grace_step_host: staging buffers");
        b->host_io = io;
    }
    HostIo *io = static_cast<HostIo *>(b->host_io);
    // graph replay keys on the device pointers: keep one slot so the graph is reused
    const int s = b->use_graph ? 0 : io->next;
    io->next ^= 1;
    const size_t n = (size_t)b->n_cells;
    cudaStream_t st = b->ctx->stream;

    // upload into slot s once its previous result has left the device, and after the previous
    // call's download when this call reads what that one writes (in-place or chained calls)
    const size_t g_bytes = io->n_doubles * sizeof(double);
    cudaError_t e = cudaStreamWaitEvent(io->up, io->freed[s], 0);
    if (e == cudaSuccess && io->last_slot >= 0 && io->last_slot != s &&
        (overlaps(h_g, g_bytes, io->last_out, io->last_bytes) ||
         overlaps(h_dt, n * sizeof(double), io->last_out, io->last_bytes)))
        e = cudaStreamWaitEvent(io->up, io->freed[io->last_slot], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(io->d_g[s], h_g, io->n_doubles * sizeof(double), cudaMemcpyHostToDevice, io->up);
    if (e == cudaSuccess) e = cudaMemcpyAsync(io->d_dt[s], h_dt, n * sizeof(double), cudaMemcpyHostToDevice, io->up);
    if (e == cudaSuccess) e = cudaEventRecord(io->uploaded[s], io->up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, io->uploaded[s], 0);
    if (e != cudaSuccess) return cuda_fail(e, "grace_step_host: upload");

    grace_status r = grace_step(b, io->d_g[s], io->d_dt[s], n_steps, prec, h_mass ? io->d_mass[s] : nullptr,
                                h_flags ? io->d_flags[s] : nullptr);
    if (r != GRACE_OK) return r;

    e = cudaEventRecord(io->stepped[s], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(io->down, io->stepped[s], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_out, io->d_g[s], io->n_doubles * sizeof(double), cudaMemcpyDeviceToHost, io->down);
    if (e == cudaSuccess && h_mass)
        e = cudaMemcpyAsync(h_mass, io->d_mass[s], n * sizeof(double), cudaMemcpyDeviceToHost, io->down);
    if (e == cudaSuccess && h_flags) e = cudaMemcpyAsync(h_flags, io->d_flags[s], n, cudaMemcpyDeviceToHost, io->down);
    if (e == cudaSuccess) e = cudaEventRecord(io->freed[s], io->down);
    if (e != cudaSuccess) return cuda_fail(e, "grace_step_host: download");
    io->last_out = reinterpret_cast<const char *>(h_out);
    io->last_bytes = g_bytes;
    io->last_slot = s;
    return GRACE_OK;
}

grace_status grace_step_host_wait(grace_batch *b)
{
    if (!b) {
        set_error("grace_step_host_wait: null batch");
        return GRACE_ERR_ARG;
    }
    if (!b->host_io) return GRACE_OK;
    Guard guard(b->ctx->device);
    HostIo *io = static_cast<HostIo *>(b->host_io);
    cudaError_t e = cudaStreamSynchronize(io->up);
    cudaError_t e2 = cudaStreamSynchronize(io->down);
    if (e == cudaSuccess) e = e2;
    return e == cudaSuccess ? GRACE_OK : cuda_fail(e, "grace_step_host_wait");
}

}  // extern "C"
