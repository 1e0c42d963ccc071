// noalloc.cu - relative error ||A - W H||_F / ||A||_F with no device allocation.
//
// rnmf_rel_err takes its per-tile partial sums from the context's scratch
// arena, which grows with cudaMalloc (and frees the old block with cudaFree)
// whenever a larger problem arrives.  Some callers cannot let that happen: a
// process that has handed all free HBM to its own pool at start-up has nothing
// left for the library to take, and a loop that keeps kernels running on other
// streams cannot afford the implicit device-wide synchronisation of
// cudaMalloc/cudaFree.  rnmf_rel_err_noalloc serves them: the same tile kernel
// and fixed-order reduction as rnmf_rel_err, with the partials and the two
// final sums in a file-scope device array of fixed size.
//
// * Size: the array holds NOALLOC_MAX_TILES pairs of partial sums (4 MiB) plus
//   the two sums; one pair per 64 x 64 tile of A, so ceil(m/64) * ceil(n/64)
//   may not exceed NOALLOC_MAX_TILES (e.g. 50000 x 20000 fits, 50000 x 50000
//   does not).  Larger problems are rejected with RNMF_EINVAL before any launch.
// * Nothing in the array has to start at zero: every partial is written by its
//   tile before the reduction reads it, and the reduction writes both sums.
// * One array per device, shared by every context on it: two calls whose work
//   overlaps in time on one device (different streams, threads or contexts)
//   race on it.  Calls on one device must be serialised by the caller.
// * The first call on a device looks the array's address up with
//   cudaGetSymbolAddress (with that device current) and keeps it; make that
//   first call before any stream capture begins.
#include <atomic>
#include <cmath>
#include <mutex>

#include "rnmf_internal.cuh"

namespace {

constexpr int64_t NOALLOC_MAX_TILES = 262144;
constexpr int NOALLOC_MAX_DEVICES = 64;

// [0, 2 * NOALLOC_MAX_TILES): partial (||A - WH||^2, ||A||^2) per tile;
// [2 * NOALLOC_MAX_TILES, + 2): the two sums.
static __device__ __align__(256) double g_relerr_scratch[2 * NOALLOC_MAX_TILES + 32];

std::atomic<double*> g_scratch_ptr[NOALLOC_MAX_DEVICES];
std::mutex g_setup_mutex;

// Address of this device's array; the device must be current.
double* scratch_for(int device, cudaError_t* err) {
    *err = cudaSuccess;
    double* p = g_scratch_ptr[device].load(std::memory_order_acquire);
    if (p) return p;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    p = g_scratch_ptr[device].load(std::memory_order_relaxed);
    if (p) return p;
    void* addr = nullptr;
    *err = cudaGetSymbolAddress(&addr, g_relerr_scratch);
    if (*err != cudaSuccess || !addr) return nullptr;
    p = static_cast<double*>(addr);
    g_scratch_ptr[device].store(p, std::memory_order_release);
    return p;
}

rnmf_status noalloc_fail(rnmf_ctx* ctx, rnmf_status st, const char* msg, cudaError_t e = cudaSuccess) {
    ctx->last_error = msg;
    if (e != cudaSuccess) {
        ctx->last_error += ": ";
        ctx->last_error += cudaGetErrorString(e);
    }
    return st;
}

}  // namespace

extern "C" rnmf_status rnmf_rel_err_noalloc(rnmf_ctx* ctx, const float* A, int64_t m, int64_t n, int64_t lda,
                                            const float* W, const float* H, int k, double* out) {
    if (!ctx) return RNMF_EINVAL;
    if (m < 1 || n < 1 || lda < n || k < 1 || !A || !W || !H || !out)
        return noalloc_fail(ctx, RNMF_EINVAL, "rnmf_rel_err_noalloc: bad argument");
    if (relerr_scratch_bytes(ctx, m, n) > (size_t)NOALLOC_MAX_TILES * 2 * sizeof(double))
        return noalloc_fail(ctx, RNMF_EINVAL,
                            "rnmf_rel_err_noalloc: ceil(m/64) * ceil(n/64) exceeds its fixed scratch of 262144 tiles");
    if (ctx->prof_on)
        return noalloc_fail(ctx, RNMF_EINVAL, "rnmf_rel_err_noalloc: switch per-kernel profiling off (it creates events)");
    if (ctx->device < 0 || ctx->device >= NOALLOC_MAX_DEVICES)
        return noalloc_fail(ctx, RNMF_EINVAL, "rnmf_rel_err_noalloc: device ordinal out of range");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return noalloc_fail(ctx, RNMF_ECUDA, "rnmf_rel_err_noalloc: cudaSetDevice", e);
    double* scratch = scratch_for(ctx->device, &e);
    if (!scratch) {
        cudaGetLastError();
        return noalloc_fail(ctx, RNMF_ECUDA, "rnmf_rel_err_noalloc: cudaGetSymbolAddress", e);
    }
    double* sums = scratch + 2 * NOALLOC_MAX_TILES;
    if (!launch_relerr(ctx, A, lda, W, k, 1, H, m, n, k, sums, scratch))
        return noalloc_fail(ctx, RNMF_ECUDA, "rnmf_rel_err_noalloc: kernel launch failed");
    // the two sums come back on the context's own stream, so the call never
    // waits on work that other streams have queued
    double h[2];
    if ((e = cudaMemcpyAsync(h, sums, sizeof h, cudaMemcpyDeviceToHost, ctx->stream)) != cudaSuccess)
        return noalloc_fail(ctx, RNMF_ECUDA, "rnmf_rel_err_noalloc: copy", e);
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
        return noalloc_fail(ctx, RNMF_ECUDA, "rnmf_rel_err_noalloc: kernels", e);
    *out = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
    return RNMF_OK;
}
