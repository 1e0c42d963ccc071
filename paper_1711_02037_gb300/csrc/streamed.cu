// streamed.cu - randomized QB with A in host memory, read in column blocks
// (Algorithm 2, Appendix A), followed by the compressed sweeps on the GPU.
//
// A (m x n, row-major, host) is never resident on the device: each pass copies
// blocks of columns A(:, J) into one of two device staging buffers on a copy
// stream while the previous block is multiplied on the context's stream
// (events order the two).  Passes: 1 (sketch) + q (power) + 1 (B) = q + 2.
//   Y = sum_J A(:, J) Omega(J, :)
//   q times: Q = qr(Y); Y = sum_J A(:, J) (A(:, J)^T Q)
//   Q = qr(Y); B^T(J, :) = A(:, J)^T Q
// The sweeps need only Q (m x l) and B^T (n x l); both stay on the device.
#include <algorithm>

#include "rnmf_internal.cuh"
#include "tc_gemm.cuh"

namespace {

// Copy of an m x w block (source rows lda apart, in device-accessible pinned
// host memory) into dst (rows w apart), read by the GPU's own loads over the
// host link.  16-byte pieces when rows are 16-byte aligned, else 4-byte words;
// each thread issues PULL_U loads before its stores, so many requests are in
// flight per SM (the link's latency, not its width, limits one load at a time).
constexpr int PULL_U = 8;

template <typename T>
__device__ __forceinline__ void pull_elems(const T* __restrict__ src, int64_t lda_t, int64_t m, int64_t w_t,
                                           T* __restrict__ dst) {
    const int64_t total = m * w_t;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e0 < total; e0 += stride * PULL_U) {
        T v[PULL_U];
#pragma unroll
        for (int u = 0; u < PULL_U; ++u) {
            const int64_t e = e0 + u * stride;
            if (e < total) v[u] = src[lda_t == w_t ? e : (e / w_t) * lda_t + e % w_t];
        }
#pragma unroll
        for (int u = 0; u < PULL_U; ++u) {
            const int64_t e = e0 + u * stride;
            if (e < total) dst[e] = v[u];
        }
    }
}

__global__ void __launch_bounds__(256) pull_block_kernel(const float* __restrict__ src, int64_t lda, int64_t m,
                                                         int64_t w, float* __restrict__ dst, int vec) {
    if (vec)
        pull_elems(reinterpret_cast<const float4*>(src), lda >> 2, m, w >> 2, reinterpret_cast<float4*>(dst));
    else
        pull_elems(src, lda, m, w, dst);
}

rnmf_status scuda(rnmf_ctx* ctx, const char* where) {
    cudaError_t e = cudaGetLastError();
    ctx->last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return RNMF_ECUDA;
}

struct Streamer {
    rnmf_ctx* ctx;
    const float* A;   // host
    int64_t m, n, lda, bc;
    float* stage[2];
    cudaEvent_t copied[2], consumed[2];
    const float* Adev = nullptr;  // device view of A when it is pinned host memory

    // Copy block b (columns [b bc, ...)) into stage[b & 1] on the copy stream.
    bool issue(int64_t b) {
        const int s = (int)(b & 1);
        const int64_t c0 = b * bc, w = std::min(bc, n - c0);
        if (cudaStreamWaitEvent(ctx->copy_stream, consumed[s], 0) != cudaSuccess) return false;
        if (Adev) {
            // the GPU pulls the block itself: many loads in flight per SM instead of
            // one DMA descriptor per (short) row of the block
            if (!launch_pull_rows(ctx, ctx->copy_stream, Adev + c0, lda, m, w, stage[s])) return false;
        } else if (cudaMemcpy2DAsync(stage[s], (size_t)w * 4, A + c0, (size_t)lda * 4, (size_t)w * 4, (size_t)m,
                                     cudaMemcpyHostToDevice, ctx->copy_stream) != cudaSuccess) {
            return false;
        }
        return cudaEventRecord(copied[s], ctx->copy_stream) == cudaSuccess;
    }

    // One pass over A: body(block index, device block (m x w, ld w), c0, w) on the
    // context's stream for every block, with the next block's copy in flight.
    template <class F>
    bool pass(F&& body) {
        const int64_t nb = (n + bc - 1) / bc;
        for (int s = 0; s < 2; ++s)
            if (cudaEventRecord(consumed[s], ctx->stream) != cudaSuccess) return false;
        if (!issue(0)) return false;
        for (int64_t b = 0; b < nb; ++b) {
            if (b + 1 < nb && !issue(b + 1)) return false;
            const int s = (int)(b & 1);
            if (cudaStreamWaitEvent(ctx->stream, copied[s], 0) != cudaSuccess) return false;
            const int64_t c0 = b * bc, w = std::min(bc, n - c0);
            if (!body(b, (const float*)stage[s], c0, w)) return false;
            if (cudaEventRecord(consumed[s], ctx->stream) != cudaSuccess) return false;
        }
        return true;
    }
};

}  // namespace

bool launch_pull_rows(rnmf_ctx* ctx, cudaStream_t stream, const float* src_dev, int64_t lda, int64_t m, int64_t w,
                      float* dst) {
    const int vec = (lda % 4 == 0 && w % 4 == 0 && (reinterpret_cast<uintptr_t>(src_dev) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(dst) & 15) == 0);
    pull_block_kernel<<<ctx->num_sms * 4, 256, 0, stream>>>(src_dev, lda, m, w, dst, vec);
    if (cudaGetLastError() != cudaSuccess) return false;
    ++ctx->launches;
    return true;
}

const float* host_device_view(const float* host) {
    cudaPointerAttributes pa{};
    const float* dev = nullptr;
    if (cudaPointerGetAttributes(&pa, host) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
        dev = static_cast<const float*>(pa.devicePointer);
    cudaGetLastError();
    return dev;
}

int64_t streamed_block_cols(int64_t m, int64_t n, int64_t requested) {
    int64_t bc = requested;
    if (bc <= 0) bc = (int64_t)(((size_t)1 << 30) / ((size_t)m * 4));  // 1 GiB per staging buffer
    bc = bc >= 4 ? bc / 4 * 4 : bc;
    if (bc < 1) bc = 1;
    return bc > n ? n : bc;
}

// Split-K scratch of A(:, J)^T Q for the full and for the last (narrower) block.
size_t streamed_atx_bytes(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int64_t bc) {
    const int64_t last = n - (n - 1) / bc * bc;
    const size_t a = gemm_atx_scratch_bytes(ctx, bc, l, m), b = gemm_atx_scratch_bytes(ctx, last, l, m);
    return (a > b ? a : b) + 8;
}

size_t streamed_qb_bytes(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int64_t bc, int precision) {
    size_t b = 2 * arena_round((size_t)m * bc * 4) + arena_round((size_t)m * l * 4) + arena_round((size_t)bc * l * 4);
    const int64_t big = m > n ? m : n;
    b += arena_round(cholqr_scratch_bytes(ctx, big, l));
    b += arena_round(streamed_atx_bytes(ctx, m, n, l, bc));
    b += tc_scratch_bytes(ctx, m, bc, l, precision);
    return b;
}

// Q (m x l) and Bt (n x l) on the device from A in host memory.  Scratch from
// the arena (streamed_qb_bytes), taken here; the caller reserved it.
rnmf_status run_qb_streamed(rnmf_ctx* ctx, const float* A_host, int64_t m, int64_t n, int64_t lda, int l, int q,
                            uint64_t seed, int omega_dist, int64_t bc, int precision, float* Q, float* Bt) {
    if (!ctx->copy_stream) {
        if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
            return scuda(ctx, "copy stream");
        for (int s = 0; s < 4; ++s)
            if (cudaEventCreateWithFlags(&ctx->copy_events[s], cudaEventDisableTiming) != cudaSuccess)
                return scuda(ctx, "copy events");
    }
    Streamer st{ctx, A_host, m, n, lda, bc, {nullptr, nullptr}, {ctx->copy_events[0], ctx->copy_events[1]},
                {ctx->copy_events[2], ctx->copy_events[3]}};
    // pinned (page-locked, registered) host memory has a device address: the
    // copy kernel reads it directly; pageable memory goes through cudaMemcpy2DAsync
    st.Adev = host_device_view(A_host);
    st.stage[0] = (float*)arena_take(ctx, (size_t)m * bc * 4);
    st.stage[1] = (float*)arena_take(ctx, (size_t)m * bc * 4);
    float* Y = (float*)arena_take(ctx, (size_t)m * l * 4);
    float* Zb = (float*)arena_take(ctx, (size_t)bc * l * 4);
    const int64_t big = m > n ? m : n;
    char* cq = (char*)arena_take(ctx, cholqr_scratch_bytes(ctx, big, l));
    double* atx = (double*)arena_take(ctx, streamed_atx_bytes(ctx, m, n, l, bc));
    const TcScratch tc = tc_scratch_take(ctx, m, bc, l, precision);
    float* Omega = Bt;  // Omega (n x l) lives in Bt's storage until the last pass writes B^T
    // Block products: tensor cores for RNMF_PREC_BF16 / RNMF_PREC_SPLIT3 (a block whose
    // width is not a multiple of 4 floats - no 16-byte TMA rows - takes the CUDA cores).
    // As in the in-memory QB, the BF16 form runs the power passes' products in one bf16
    // term and the products that fix Q and B in the 3-term split.
    const bool split_all = precision == RNMF_PREC_SPLIT3;
    auto ax = [&](const float* Ab, int64_t w, const float* X, float* Yo, bool accurate) {
        if (precision != RNMF_PREC_FP32 && w % 4 == 0)
            return tc_gemm_ax(ctx, tc, Ab, w, X, Yo, m, w, l, accurate ? 3 : 1, true);
        return launch_gemm_ax(ctx, Ab, w, X, l, 1, Yo, l, 1, m, l, w, true);
    };
    auto atx_p = [&](const float* Ab, int64_t w, const float* X, float* Zo, bool accurate) {
        if (precision != RNMF_PREC_FP32 && w % 4 == 0) return tc_gemm_atx(ctx, tc, Ab, w, X, Zo, m, w, l, accurate ? 3 : 1);
        return launch_gemm_atx(ctx, Ab, w, X, l, 1, Zo, l, 1, w, l, m, atx);
    };

    if (!launch_omega(ctx, Omega, n, l, seed, omega_dist, l, 1)) return scuda(ctx, "omega");
    if (cudaMemsetAsync(Y, 0, (size_t)m * l * 4, ctx->stream) != cudaSuccess) return scuda(ctx, "memset");
    // Y = sum_J A(:, J) Omega(J, :)
    if (!st.pass([&](int64_t, const float* Ab, int64_t c0, int64_t w) {
            return ax(Ab, w, Omega + c0 * l, Y, split_all || q == 0);
        }))
        return scuda(ctx, "sketch pass");
    for (int it = 0; it < q; ++it) {
        if (cudaMemcpyAsync(Q, Y, (size_t)m * l * 4, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
            return scuda(ctx, "copy Y");
        if (!cholqr2(ctx, Q, m, l, cq)) return scuda(ctx, "cholqr(Y)");
        if (cudaMemsetAsync(Y, 0, (size_t)m * l * 4, ctx->stream) != cudaSuccess) return scuda(ctx, "memset");
        // Y = sum_J A(:, J) (A(:, J)^T Q)
        if (!st.pass([&](int64_t, const float* Ab, int64_t, int64_t w) {
                return atx_p(Ab, w, Q, Zb, split_all) && ax(Ab, w, Zb, Y, split_all || it == q - 1);
            }))
            return scuda(ctx, "power pass");
    }
    if (cudaMemcpyAsync(Q, Y, (size_t)m * l * 4, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
        return scuda(ctx, "copy Y");
    if (!cholqr2(ctx, Q, m, l, cq)) return scuda(ctx, "cholqr(Y)");
    // B^T(J, :) = A(:, J)^T Q
    if (!st.pass([&](int64_t, const float* Ab, int64_t c0, int64_t w) {
            return atx_p(Ab, w, Q, Bt + c0 * l, true);
        }))
        return scuda(ctx, "projection pass");
    return RNMF_OK;
}
