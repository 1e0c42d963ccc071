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

// One block: Cholesky factor of G (c x c, float pairs hi + lo) and the inverse
// of the factor, from one right-looking elimination in double-float.
// G = L L^T with L = R^T.  Step j takes pivot d_j = G_jj (after steps < j):
//   trailing block  G_it -= G_ji G_jt / d_j          (j < i <= t)
//   rows of M       M_iu -= (G_ji / d_j) M_ju         (i > j, u <= j)
// and row j of G and of M is then divided by r_j = sqrt(d_j).  The same row
// operations turn G into L^T = R (upper part) and the identity M into L^{-1} =
// (R^{-1})^T (lower part), so R^{-1} needs no separate substitution.  Every
// update of step j reads only the unscaled row j, so the division of row j is
// deferred to step j + 1 and each step takes one block barrier.  The thread
// that updates G_{j+1,j+1} in step j also forms the next pivot's 1 / d and
// 1 / r.  Storage: G's upper triangle (R when done) and M's strict lower
// triangle share one c x c array; M's diagonal is kept apart.
//   flags[0]: set to 1 when the shift was used (pass 1).
//   mode 0: pass 1 (may shift); mode 1: pass 2 (no shift);
//   mode 2: conditional pass 3 - if flags[0] == 0 write the identity instead.
// Output: float32 Rinv (c x c, row-major, zero below the diagonal).
__global__ void __launch_bounds__(NT) chol_inv_kernel(const float2* __restrict__ G, int c, int64_t N, int mode,
                                                      int* __restrict__ flags, float* __restrict__ Rinv,
                                                      int* __restrict__ status) {
    extern __shared__ __align__(16) dfloat sh[];
    dfloat* Gs = sh;               // c x c: upper part G / R, strict lower part M
    dfloat* mdiag = sh + c * c;    // c: diagonal of M
    dfloat* dinv = mdiag + c;      // c: 1 / d_j
    dfloat* rinv = dinv + c;       // c: 1 / r_j
    __shared__ int fail;
    __shared__ float shift;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    constexpr int NW = NT / 32;

    if (mode == 2 && flags[0] == 0) {
        for (int e = tid; e < c * c; e += NT) Rinv[e] = (e / c == e % c) ? 1.f : 0.f;
        return;
    }
    // 1 / d and 1 / r of pivot d (false: not positive definite)
    auto pivot = [&](int j, dfloat d) {
        if (!(d.hi > 0.f) || !isfinite(d.hi)) {
            fail = 1;
            return;
        }
        dinv[j] = df_recip(d);
        rinv[j] = df_recip(df_sqrt(d));
    };
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
            const int i = e / c, t = e % c;
            const float2 g = G[e];
            if (t > i) Gs[e] = df_make(g.x, g.y);
            else if (t == i) Gs[e] = df_add(df_make(g.x, g.y), df_make(shift, 0.f));
            else Gs[e] = df_make(0.f, 0.f);  // M starts as the identity: zero below the diagonal
        }
        for (int i = tid; i < c; i += NT) mdiag[i] = df_make(1.f, 0.f);
        __syncthreads();
        if (tid == 0) pivot(0, Gs[0]);
        __syncthreads();
        for (int j = 0; j < c && !fail; ++j) {
            // deferred division of row j - 1 of R and of M by r_{j-1}
            if (j > 0) {
                const dfloat rv = rinv[j - 1];
                const int jm = j - 1;
                for (int e = tid; e < c; e += NT) Gs[jm * c + e] = df_mul(Gs[jm * c + e], rv);  // R and M parts
                if (tid == 0) mdiag[jm] = df_mul(mdiag[jm], rv);
            }
            const dfloat di = dinv[j];
            const dfloat* rowj = Gs + j * c;
            for (int i = j + 1 + warp; i < c; i += NW) {
                const dfloat a = df_mul(rowj[i], di);  // G_ji / d_j
                dfloat* rowi = Gs + i * c;
                for (int t = i + lane; t < c; t += 32) {
                    const dfloat v = df_fms(rowi[t], a, rowj[t]);
                    rowi[t] = v;
                    if (t == i && i == j + 1) pivot(i, v);
                }
                // M_iu for u <= j: the strict lower row j of M, its diagonal for u = j
                for (int u = lane; u <= j; u += 32) {
                    const dfloat mju = u < j ? rowj[u] : mdiag[j];
                    rowi[u] = df_fms(rowi[u], a, mju);
                }
            }
            __syncthreads();
        }
        if (!fail) {
            // division of the last row
            const dfloat rv = rinv[c - 1];
            for (int e = tid; e < c; e += NT) Gs[(c - 1) * c + e] = df_mul(Gs[(c - 1) * c + e], rv);
            if (tid == 0) mdiag[c - 1] = df_mul(mdiag[c - 1], rv);
            __syncthreads();
            break;
        }
        if (mode != 0 || attempt == 1) {
            if (tid == 0) *status = RNMF_DEV_NOTPD;
            for (int e = tid; e < c * c; e += NT) Rinv[e] = (e / c == e % c) ? 1.f : 0.f;
            return;
        }
        if (tid == 0) flags[0] = 1;
        __syncthreads();
    }
    // R^{-1} = M^T: entry (i, j), i <= j, is M_ji
    for (int e = tid; e < c * c; e += NT) {
        const int i = e / c, j = e % c;
        Rinv[e] = i < j ? df_to_float(Gs[j * c + i]) : (i == j ? df_to_float(mdiag[i]) : 0.f);
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
    size_t smem = ((size_t)c * c + 3 * c) * sizeof(dfloat);
    cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(((size_t)RNMF_MAX_L * RNMF_MAX_L + 3 * RNMF_MAX_L) * sizeof(dfloat)));
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
