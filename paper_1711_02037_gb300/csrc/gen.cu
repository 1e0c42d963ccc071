// gen.cu - random test matrix Omega (Section 2.3, Algorithm 1) and the uniform
// initial factors (Algorithm 1 initialisation), plus small layout helpers.
#include "philox.cuh"
#include "rnmf_internal.cuh"

namespace {

constexpr uint32_t STREAM_OMEGA = 1;

// One thread per Box-Muller pair: logical row-major elements 2b and 2b+1 of the
// n x l matrix; stored at out[i*s_row + j*s_col].
__global__ void omega_gauss_kernel(float* __restrict__ out, int64_t n, int l, uint64_t seed,
                                   int64_t s_row, int64_t s_col) {
    int64_t total = n * (int64_t)l;
    int64_t npairs = (total + 1) >> 1;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < npairs;
         b += (int64_t)gridDim.x * blockDim.x) {
        float z0, z1;
        rnmf_rng::gauss_pair(seed, STREAM_OMEGA, 0, (uint64_t)b, &z0, &z1);
        int64_t e0 = 2 * b;
        out[(e0 / l) * s_row + (e0 % l) * s_col] = z0;
        int64_t e1 = e0 + 1;
        if (e1 < total) out[(e1 / l) * s_row + (e1 % l) * s_col] = z1;
    }
}

// One thread per Philox block of 4 uniform words.
__global__ void uniform_kernel(float* __restrict__ out, int64_t rows, int64_t cols, uint64_t seed,
                               uint32_t stream_id, int64_t s_row, int64_t s_col) {
    int64_t total = rows * cols;
    int64_t nblk = (total + 3) >> 2;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk;
         b += (int64_t)gridDim.x * blockDim.x) {
        uint32_t w[4];
        rnmf_rng::block(seed, stream_id, 0, (uint64_t)b, w);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            int64_t e = 4 * b + t;
            if (e < total) out[(e / cols) * s_row + (e % cols) * s_col] = (float)(w[t] >> 8) * 0x1p-24f;
        }
    }
}

__global__ void transpose_kernel(const float* __restrict__ in, int64_t rows, int64_t cols,
                                 float* __restrict__ out) {
    __shared__ float tile[32][33];
    int64_t c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        int64_t r = r0 + dy, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[dy][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        int64_t c = c0 + dy, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = tile[threadIdx.x][dy];
    }
}

__global__ void copy_kernel(const float* __restrict__ in, float* __restrict__ out, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

__global__ void pad_rows_kernel(const float* __restrict__ in, int64_t rows, int cols, int ld_out,
                                float* __restrict__ out) {
    const int64_t total = rows * ld_out;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / ld_out;
        const int c = (int)(e % ld_out);
        out[e] = c < cols ? in[r * cols + c] : 0.f;
    }
}

int grid_for(rnmf_ctx* ctx, int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    int64_t cap = (int64_t)ctx->num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

bool launch_omega(rnmf_ctx* ctx, float* out, int64_t n, int l, uint64_t seed, int dist, int64_t s_row,
                  int64_t s_col) {
    prof_begin(ctx);
    if (dist == 0) {
        int64_t npairs = (n * l + 1) / 2;
        omega_gauss_kernel<<<grid_for(ctx, npairs, 256), 256, 0, ctx->stream>>>(out, n, l, seed, s_row, s_col);
    } else {
        int64_t nblk = (n * l + 3) / 4;
        uniform_kernel<<<grid_for(ctx, nblk, 256), 256, 0, ctx->stream>>>(out, n, l, seed, STREAM_OMEGA, s_row,
                                                                           s_col);
    }
    return launch_done(ctx, K_OMEGA, (double)n * l * 4, 0);
}

bool launch_uniform_matrix(rnmf_ctx* ctx, float* out, int64_t rows, int64_t cols, uint64_t seed,
                           uint32_t stream_id, int64_t s_row, int64_t s_col) {
    int64_t nblk = (rows * cols + 3) / 4;
    prof_begin(ctx);
    uniform_kernel<<<grid_for(ctx, nblk, 256), 256, 0, ctx->stream>>>(out, rows, cols, seed, stream_id, s_row,
                                                                       s_col);
    return launch_done(ctx, K_UNIFORM, (double)rows * cols * 4, 0);
}

bool launch_transpose(rnmf_ctx* ctx, const float* in, int64_t rows, int64_t cols, float* out) {
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    prof_begin(ctx);
    transpose_kernel<<<grid, dim3(32, 8), 0, ctx->stream>>>(in, rows, cols, out);
    return launch_done(ctx, K_TRANSPOSE, (double)rows * cols * 8, 0);
}

bool launch_copy(rnmf_ctx* ctx, const float* in, float* out, int64_t count) {
    prof_begin(ctx);
    copy_kernel<<<grid_for(ctx, count, 256), 256, 0, ctx->stream>>>(in, out, count);
    return launch_done(ctx, K_TRANSPOSE, (double)count * 8, 0);
}

bool launch_pad_rows(rnmf_ctx* ctx, const float* in, int64_t rows, int cols, int ld_out, float* out) {
    prof_begin(ctx);
    pad_rows_kernel<<<grid_for(ctx, rows * ld_out, 256), 256, 0, ctx->stream>>>(in, rows, cols, ld_out, out);
    return launch_done(ctx, K_TRANSPOSE, (double)rows * (cols + ld_out) * 4, 0);
}
