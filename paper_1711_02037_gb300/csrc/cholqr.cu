// cholqr.cu - orthonormalisation [Q, ~] = qr(Y) of Section 2.3 / Algorithm 1
// by CholeskyQR2 (Fukaya, Nakatsukasa, Yanagisawa, Yamamoto 2014):
//   G = Y^T Y (error-free products, float32-pair sums), R = chol(G), Q = Y R^{-1},
//   repeated once.
// The Cholesky factor and its inverse are computed in double-float arithmetic
// (df.cuh, about 48 significant bits) on the float32 pipe: float64 runs at a
// small fraction of the float32 rate on this GPU.
// When a Gram matrix is not numerically positive definite (Y ill conditioned,
// e.g. an exactly low-rank A with l > rank), the first pass adds the shift
// s = 11 (N c + c (c + 1)) u trace(G), u = 2^-48 (the double-float unit
// roundoff), to the diagonal (shifted CholeskyQR, Fukaya et al. 2020) and a
// third pass follows.
// The Householder QR of the paper and this factorisation give bases of the
// same column space; the randomized HALS result does not depend on the basis
// (W~ = Q^T W rotates with Q).
#include "df.cuh"
#include "rnmf_internal.cuh"

namespace {

constexpr int NT = 512;

__device__ __forceinline__ dfloat df_shfl_xor(dfloat x, int o) {
    return df_make(__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o));
}

// One block: Cholesky of G (c x c, float pairs hi + lo) in shared memory,
// optional shift on breakdown, inverse of the upper factor R, written as
// float32 Rinv (c x c, row-major, zero below the diagonal).
//   flags[0]: set to 1 when the shift was used (pass 1).
//   mode 0: pass 1 (may shift); mode 1: pass 2 (no shift);
//   mode 2: conditional pass 3 - if flags[0] == 0 write the identity instead.
__global__ void __launch_bounds__(NT) chol_inv_kernel(const float2* __restrict__ G, int c, int64_t N, int mode,
                                                      int* __restrict__ flags, float* __restrict__ Rinv,
                                                      int* __restrict__ status) {
    extern __shared__ __align__(16) dfloat sh[];
    dfloat* Gs = sh;              // c x c, pitch c
    dfloat* diag = sh + c * c;    // c
    __shared__ int fail;
    __shared__ float shift;
    __shared__ dfloat dinv_j;
    const int tid = threadIdx.x;

    if (mode == 2 && flags[0] == 0) {
        for (int e = tid; e < c * c; e += NT) Rinv[e] = (e / c == e % c) ? 1.f : 0.f;
        return;
    }
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (tid == 0) {
            fail = 0;
            shift = 0.f;
            if (attempt == 1) {
                float tr = 0.f;
                for (int i = 0; i < c; ++i) tr += G[i * c + i].x;
                shift = (float)(11.0 * ((double)N * c + (double)c * (c + 1)) * 0x1p-48) * tr;
            }
        }
        __syncthreads();
        for (int e = tid; e < c * c; e += NT) {
            const float2 g = G[e];
            Gs[e] = (e / c == e % c) ? df_add(df_make(g.x, g.y), df_make(shift, 0.f)) : df_make(g.x, g.y);
        }
        __syncthreads();
        // right-looking Cholesky on the upper triangle: G = R^T R
        for (int j = 0; j < c; ++j) {
            if (tid == 0) {
                const dfloat d = Gs[j * c + j];
                if (!(d.hi > 0.f) || !isfinite(d.hi)) {
                    fail = 1;
                } else {
                    const dfloat r = df_sqrt(d);
                    Gs[j * c + j] = r;
                    dinv_j = df_recip(r);  // one reciprocal per column, then products
                }
            }
            __syncthreads();
            if (fail) break;
            const dfloat dinv = dinv_j;
            for (int t = j + 1 + tid; t < c; t += NT) Gs[j * c + t] = df_mul(Gs[j * c + t], dinv);
            __syncthreads();
            {
                const int warp = tid / 32, lane = tid % 32;
                for (int ii = j + 1 + warp; ii < c; ii += NT / 32) {
                    const dfloat rji = Gs[j * c + ii];
                    for (int tt = ii + lane; tt < c; tt += 32)
                        Gs[ii * c + tt] = df_fms(Gs[ii * c + tt], rji, Gs[j * c + tt]);
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
    for (int i = tid; i < c; i += NT) {
        const dfloat r = df_recip(Gs[i * c + i]);
        Gs[i * c + i] = r;
        diag[i] = r;  // 1 / R[i][i]
    }
    __syncthreads();
    {
        // row sweep from the bottom: X[i][jc] = -(sum_{t=i+1..jc} R[i][t] X[t][jc]) / R[i][i]
        const int warp = tid / 32, lane = tid % 32;
        for (int i = c - 2; i >= 0; --i) {
            for (int jc = i + 1 + warp; jc < c; jc += NT / 32) {
                dfloat s = df_make(0.f, 0.f);
                for (int t = i + 1 + lane; t <= jc; t += 32) s = df_add(s, df_mul(Gs[i * c + t], Gs[jc * c + t]));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s = df_add(s, df_shfl_xor(s, o));
                if (lane == 0) Gs[jc * c + i] = df_neg(df_mul(s, diag[i]));
            }
            __syncthreads();
        }
    }
    for (int e = tid; e < c * c; e += NT) {
        int i = e / c, j = e % c;
        Rinv[e] = (i <= j) ? df_to_float(Gs[j * c + i]) : 0.f;
    }
}

}  // namespace

size_t cholqr_scratch_bytes(rnmf_ctx* ctx, int64_t N, int c) {
    return arena_round(gram_scratch_bytes(ctx, N, c)) + arena_round((size_t)c * c * sizeof(float2)) +
           arena_round((size_t)c * c * sizeof(float));
}

// Q = qr(Y) in place on Y (N x c, row-major).  Scratch: cholqr_scratch_bytes().
bool cholqr2(rnmf_ctx* ctx, float* Y, int64_t N, int c, char* scratch) {
    double* gpart = reinterpret_cast<double*>(scratch);
    char* p = scratch + arena_round(gram_scratch_bytes(ctx, N, c));
    float2* G = reinterpret_cast<float2*>(p);  // the Gram as float pairs hi + lo
    p += arena_round((size_t)c * c * sizeof(float2));
    float* Rinv = reinterpret_cast<float*>(p);
    size_t smem = ((size_t)c * c + c) * sizeof(dfloat);
    cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(((size_t)RNMF_MAX_L * RNMF_MAX_L + RNMF_MAX_L) * sizeof(dfloat)));
    if (cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), ctx->stream) != cudaSuccess) return false;
    for (int pass = 0; pass < 3; ++pass) {
        if (!launch_gram(ctx, Y, c, 1, N, c, nullptr, nullptr, gpart, pass == 2 ? ctx->d_flags : nullptr, true, G))
            return false;
        prof_begin(ctx);
        chol_inv_kernel<<<1, NT, smem, ctx->stream>>>(G, c, N, pass, ctx->d_flags, Rinv, ctx->d_status);
        if (!launch_done(ctx, K_CHOL, 12.0 * c * c, (double)c * c * c * 2.0 / 3.0)) return false;
        if (!launch_gemm_ax(ctx, Y, c, Rinv, c, 1, Y, c, 1, N, c, c)) return false;
    }
    return true;
}
