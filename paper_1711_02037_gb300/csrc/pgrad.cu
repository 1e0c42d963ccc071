// pgrad.cu - projected gradient of ||A - W H||_F^2 on the compressed problem
// (Section 3.3 stopping measure, A replaced by Q B).
//
//   G_W = 2 (W V - Q T),  V = H H^T, T = B H^T       (m x k)
//   G_H = 2 (S H - R^T),  S = W^T W, R = B^T W~      (k x n)
//   grad^P = G where the variable is > 0, min(0, G) where it is 0;
//   measure = ||grad^P_W||_F^2 + ||grad^P_H||_F^2 (float64 sums, fixed order).
#include "rnmf_internal.cuh"

namespace {

constexpr int PG_NT = 256;
constexpr int PG_KM = 128;   // k <= l <= 128

__device__ __forceinline__ double proj_sq(float g, float x) {
    const float p = x > 0.f ? g : fminf(0.f, g);
    return (double)p * (double)p;
}

__device__ __forceinline__ void block_sum_to(double v, double* out) {
    __shared__ double red[PG_NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < PG_NT / 32; ++w) s += red[w];
        *out = s;
    }
}

// Rows of W: thread per row r (W stored transposed, Wc = W^T k x m; Q rows pitch lq).
__global__ void __launch_bounds__(PG_NT) pg_w_kernel(const float* __restrict__ Wc, const float* __restrict__ Q,
                                                     int64_t m, int l, int lq, int k, const float* __restrict__ V,
                                                     const float* __restrict__ T, double* __restrict__ part) {
    extern __shared__ float sm[];
    float* Vs = sm;              // k x k
    float* Ts = Vs + k * k;      // l x k
    for (int e = threadIdx.x; e < k * k; e += PG_NT) Vs[e] = V[e];
    for (int e = threadIdx.x; e < l * k; e += PG_NT) Ts[e] = T[e];
    __syncthreads();
    double acc = 0.0;
    const int64_t r = (int64_t)blockIdx.x * PG_NT + threadIdx.x;
    if (r < m) {
        for (int j = 0; j < k; ++j) {
            float g = 0.f;
            for (int i = 0; i < k; ++i) g = fmaf(Wc[(int64_t)i * m + r], Vs[i * k + j], g);
            for (int t = 0; t < l; ++t) g = fmaf(-Q[r * lq + t], Ts[t * k + j], g);
            acc += proj_sq(2.f * g, Wc[(int64_t)j * m + r]);
        }
    }
    block_sum_to(acc, part + blockIdx.x);
}

// Columns of H: thread per column c (Rt = R^T, k x n).
__global__ void __launch_bounds__(PG_NT) pg_h_kernel(const float* __restrict__ H, const float* __restrict__ Rt,
                                                     int64_t n, int k, const float* __restrict__ S,
                                                     double* __restrict__ part) {
    extern __shared__ float sm[];
    float* Ss = sm;  // k x k
    for (int e = threadIdx.x; e < k * k; e += PG_NT) Ss[e] = S[e];
    __syncthreads();
    double acc = 0.0;
    const int64_t c = (int64_t)blockIdx.x * PG_NT + threadIdx.x;
    if (c < n) {
        for (int j = 0; j < k; ++j) {
            float g = -Rt[(int64_t)j * n + c];
            for (int i = 0; i < k; ++i) g = fmaf(Ss[i * k + j], H[(int64_t)i * n + c], g);
            acc += proj_sq(2.f * g, H[(int64_t)j * n + c]);
        }
    }
    block_sum_to(acc, part + blockIdx.x);
}

__global__ void pg_sum_kernel(const double* __restrict__ part, int64_t count, double* __restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += 256) s += part[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

size_t pgrad_scratch_bytes(int64_t m, int64_t n) {
    return (size_t)((m + PG_NT - 1) / PG_NT + (n + PG_NT - 1) / PG_NT + 1) * sizeof(double);
}

bool launch_pgrad(rnmf_ctx* ctx, const float* Wc, const float* Q, int64_t m, int l, int lq, int k, const float* V,
                  const float* T, const float* H, const float* Rt, int64_t n, const float* S, double* scratch,
                  double* out) {
    if (k > PG_KM || l > PG_KM) return false;
    const int64_t gw = (m + PG_NT - 1) / PG_NT, gh = (n + PG_NT - 1) / PG_NT;
    prof_begin(ctx);
    pg_w_kernel<<<(unsigned)gw, PG_NT, (size_t)(k * k + l * k) * sizeof(float), ctx->stream>>>(Wc, Q, m, l, lq, k, V,
                                                                                               T, scratch);
    if (!launch_done(ctx, K_RELERR, 4.0 * ((double)m * k + (double)m * l), 2.0 * m * k * (k + l))) return false;
    prof_begin(ctx);
    pg_h_kernel<<<(unsigned)gh, PG_NT, (size_t)k * k * sizeof(float), ctx->stream>>>(H, Rt, n, k, S, scratch + gw);
    if (!launch_done(ctx, K_RELERR, 4.0 * (2.0 * n * k), 2.0 * n * k * k)) return false;
    prof_begin(ctx);
    pg_sum_kernel<<<1, 256, 0, ctx->stream>>>(scratch, gw + gh, out);
    return launch_done(ctx, K_RELERR, 8.0 * (gw + gh), 0);
}
