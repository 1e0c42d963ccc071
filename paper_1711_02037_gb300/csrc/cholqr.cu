// cholqr.cu - orthonormalisation [Q, ~] = qr(Y) of Section 2.3 / Algorithm 1
// by CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa, Yamamoto 2014):
//   G = Y^T Y (float64), R = chol(G), Q = Y R^{-1}, repeated once.
// When a Gram matrix is not numerically positive definite (Y ill conditioned,
// e.g. an exactly low-rank A with l > rank), the first pass adds the shift
// s = 11 (N c + c (c + 1)) u trace(G), u = 2^-53, to the diagonal (shifted
// CholeskyQR, Fukaya et al. 2020) and a third pass follows.
// The Householder QR of the paper and this factorisation give bases of the
// same column space; the randomized HALS result does not depend on the basis
// (W~ = Q^T W rotates with Q).
#include "rnmf_internal.cuh"

namespace {

constexpr int NT = 512;

// One block: Cholesky of G (c x c, float64) in shared memory, optional shift on
// breakdown, inverse of the upper factor R, written as float32 Rinv (c x c,
// row-major, zero below the diagonal).
//   flags[0]: set to 1 when the shift was used (pass 1).
//   mode 0: pass 1 (may shift); mode 1: pass 2 (no shift);
//   mode 2: conditional pass 3 - if flags[0] == 0 write the identity instead.
__global__ void __launch_bounds__(NT) chol_inv_kernel(const double* __restrict__ G, int c, int64_t N, int mode,
                                                      int* __restrict__ flags, float* __restrict__ Rinv,
                                                      int* __restrict__ status) {
    extern __shared__ double sh[];
    double* Gs = sh;              // c x c, pitch c
    double* diag = sh + c * c;    // c
    __shared__ int fail;
    __shared__ double shift;
    const int tid = threadIdx.x;

    if (mode == 2 && flags[0] == 0) {
        for (int e = tid; e < c * c; e += NT) Rinv[e] = (e / c == e % c) ? 1.f : 0.f;
        return;
    }
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (tid == 0) {
            fail = 0;
            shift = 0.0;
            if (attempt == 1) {
                double tr = 0.0;
                for (int i = 0; i < c; ++i) tr += G[i * c + i];
                shift = 11.0 * ((double)N * c + (double)c * (c + 1)) * 0x1p-53 * tr;
            }
        }
        __syncthreads();
        for (int e = tid; e < c * c; e += NT) Gs[e] = G[e] + ((e / c == e % c) ? shift : 0.0);
        __syncthreads();
        // right-looking Cholesky on the upper triangle: G = R^T R
        for (int j = 0; j < c; ++j) {
            if (tid == 0) {
                double d = Gs[j * c + j];
                if (!(d > 0.0) || !isfinite(d)) {
                    fail = 1;
                } else {
                    Gs[j * c + j] = sqrt(d);
                }
            }
            __syncthreads();
            if (fail) break;
            const double dinv = 1.0 / Gs[j * c + j];  // one division per column, then products
            for (int t = j + 1 + tid; t < c; t += NT) Gs[j * c + t] *= dinv;
            __syncthreads();
            {
                const int warp = tid / 32, lane = tid % 32;
                for (int ii = j + 1 + warp; ii < c; ii += NT / 32) {
                    const double rji = Gs[j * c + ii];
                    for (int tt = ii + lane; tt < c; tt += 32) Gs[ii * c + tt] -= rji * Gs[j * c + tt];
                }
            }
            __syncthreads();
        }
        __syncthreads();
        if (!fail) break;
        if (mode != 0 || attempt == 1) {
            if (tid == 0) *status = RNMF_DEV_NOTPD;
            for (int e = tid; e < c * c; e += NT) Rinv[e] = (e / c == e % c) ? 1.f : 0.f;
            return;
        }
        if (tid == 0) flags[0] = 1;
        __syncthreads();
    }
    // R (upper, in Gs) -> X = R^{-1} (upper), X[i][jc] stored in Gs[jc][i] (lower part)
    for (int i = tid; i < c; i += NT) diag[i] = Gs[i * c + i];
    __syncthreads();
    for (int i = tid; i < c; i += NT) {
        const double r = 1.0 / diag[i];
        Gs[i * c + i] = r;
        diag[i] = r;  // from here on diag holds 1 / R[i][i]
    }
    __syncthreads();
    {
        // row sweep from the bottom: X[i][jc] = -(sum_{t=i+1..jc} R[i][t] X[t][jc]) / R[i][i]
        const int warp = tid / 32, lane = tid % 32;
        for (int i = c - 2; i >= 0; --i) {
            for (int jc = i + 1 + warp; jc < c; jc += NT / 32) {
                double s = 0.0;
                for (int t = i + 1 + lane; t <= jc; t += 32) s = fma(Gs[i * c + t], Gs[jc * c + t], s);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) Gs[jc * c + i] = -s * diag[i];
            }
            __syncthreads();
        }
    }
    for (int e = tid; e < c * c; e += NT) {
        int i = e / c, j = e % c;
        Rinv[e] = (i <= j) ? (float)Gs[j * c + i] : 0.f;
    }
}

}  // namespace

size_t cholqr_scratch_bytes(rnmf_ctx* ctx, int64_t N, int c) {
    return arena_round(gram_scratch_bytes(ctx, N, c)) + arena_round((size_t)c * c * sizeof(double)) +
           arena_round((size_t)c * c * sizeof(float));
}

// Q = qr(Y) in place on Y (N x c, row-major).  Scratch: cholqr_scratch_bytes().
bool cholqr2(rnmf_ctx* ctx, float* Y, int64_t N, int c, char* scratch) {
    double* gpart = reinterpret_cast<double*>(scratch);
    char* p = scratch + arena_round(gram_scratch_bytes(ctx, N, c));
    double* G = reinterpret_cast<double*>(p);
    p += arena_round((size_t)c * c * sizeof(double));
    float* Rinv = reinterpret_cast<float*>(p);
    size_t smem = ((size_t)c * c + c) * sizeof(double);
    cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(((size_t)RNMF_MAX_L * RNMF_MAX_L + RNMF_MAX_L) * sizeof(double)));
    if (cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), ctx->stream) != cudaSuccess) return false;
    for (int pass = 0; pass < 3; ++pass) {
        if (!launch_gram(ctx, Y, c, 1, N, c, G, nullptr, gpart, pass == 2 ? ctx->d_flags : nullptr, true))
            return false;
        prof_begin(ctx);
        chol_inv_kernel<<<1, NT, smem, ctx->stream>>>(G, c, N, pass, ctx->d_flags, Rinv, ctx->d_status);
        if (!launch_done(ctx, K_CHOL, 12.0 * c * c, (double)c * c * c * 2.0 / 3.0)) return false;
        if (!launch_gemm_ax(ctx, Y, c, Rinv, c, 1, Y, c, 1, N, c, c)) return false;
    }
    return true;
}
