// gram.cu - G = X^T X (c x c, c <= 128) with float64 accumulation.
//
// Used for the Gram matrix of CholeskyQR (the orthonormalisation qr() of
// Section 2.3 / Algorithm 1), and for S = W^T W and V = H H^T of a sweep
// (Algorithm 1 loop body).  Products of two float32 values are exact in
// float64, so each partial sum carries only float64 accumulation error.
// Rows are split over blocks; block partials are summed in a fixed order.
#include "rnmf_internal.cuh"

namespace {

constexpr int NT = 256;
constexpr int RB = 32;  // rows per shared-memory stage

template <int CP>
__global__ void __launch_bounds__(NT) gram_partial_kernel(const float* __restrict__ X, int64_t s_r, int64_t s_c,
                                                          int64_t N, int c, int64_t rchunk,
                                                          double* __restrict__ partial,
                                                          const int* __restrict__ skip_if_zero) {
    if (skip_if_zero && *skip_if_zero == 0) return;
    constexpr int PMAX = CP * (CP + 1) / 2;
    constexpr int PPT = (PMAX + NT - 1) / NT;
    __shared__ double Xs[RB][CP + 1];
    const int npairs = c * (c + 1) / 2;
    // decode this thread's pairs (i <= j), row-major over the upper triangle
    int pi[PPT], pj[PPT];
    double acc[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        int p = threadIdx.x + q * NT;
        int i = 0, rem = p;
        while (i < c && rem >= c - i) {
            rem -= c - i;
            ++i;
        }
        pi[q] = i < c ? i : 0;
        pj[q] = i < c ? i + rem : 0;
        acc[q] = 0.0;
    }
    const int64_t rbeg = (int64_t)blockIdx.x * rchunk;
    const int64_t rend = rbeg + rchunk < N ? rbeg + rchunk : N;
    for (int64_t r0 = rbeg; r0 < rend; r0 += RB) {
        for (int e = threadIdx.x; e < RB * CP; e += NT) {
            int rr, j;
            if (s_c == 1) {
                rr = e / CP;
                j = e % CP;
            } else {
                j = e / RB;
                rr = e % RB;
            }
            int64_t r = r0 + rr;
            Xs[rr][j] = (j < c && r < rend) ? (double)X[r * s_r + (int64_t)j * s_c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            if (threadIdx.x + q * NT < npairs) {
                double a = acc[q];
                const int i = pi[q], j = pj[q];
#pragma unroll 8
                for (int rr = 0; rr < RB; ++rr) a = fma(Xs[rr][i], Xs[rr][j], a);
                acc[q] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        int p = threadIdx.x + q * NT;
        if (p < npairs) partial[(int64_t)blockIdx.x * npairs + p] = acc[q];
    }
}

__global__ void gram_reduce_kernel(const double* __restrict__ partial, int nblk, int c, double* __restrict__ G,
                                   float* __restrict__ G32, const int* __restrict__ skip_if_zero) {
    if (skip_if_zero && *skip_if_zero == 0) return;
    const int npairs = c * (c + 1) / 2;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * npairs + p];
        int i = 0, rem = p;
        while (rem >= c - i) {
            rem -= c - i;
            ++i;
        }
        int j = i + rem;
        G[i * c + j] = s;
        G[j * c + i] = s;
        if (G32) {
            G32[i * c + j] = (float)s;
            G32[j * c + i] = (float)s;
        }
    }
}

void gram_split(rnmf_ctx* ctx, int64_t N, int* nblk, int64_t* rchunk) {
    int64_t target = (int64_t)ctx->num_sms * 2;
    int64_t rc = (N + target - 1) / target;
    rc = (rc + RB - 1) / RB * RB;
    if (rc < RB) rc = RB;
    int64_t nb = (N + rc - 1) / rc;
    if (nb < 1) nb = 1;
    *nblk = (int)nb;
    *rchunk = rc;
}

}  // namespace

size_t gram_scratch_bytes(rnmf_ctx* ctx, int64_t N, int c) {
    int nb;
    int64_t rc;
    gram_split(ctx, N, &nb, &rc);
    return (size_t)nb * (c * (c + 1) / 2) * sizeof(double);
}

bool launch_gram(rnmf_ctx* ctx, const float* X, int64_t s_r, int64_t s_c, int64_t N, int c, double* G,
                 float* G32, double* scratch, const int* skip_if_zero) {
    int nb;
    int64_t rc;
    gram_split(ctx, N, &nb, &rc);
    int cp = c <= 16 ? 16 : c <= 32 ? 32 : c <= 64 ? 64 : 128;
    prof_begin(ctx);
    switch (cp) {
        case 16: gram_partial_kernel<16><<<nb, NT, 0, ctx->stream>>>(X, s_r, s_c, N, c, rc, scratch, skip_if_zero); break;
        case 32: gram_partial_kernel<32><<<nb, NT, 0, ctx->stream>>>(X, s_r, s_c, N, c, rc, scratch, skip_if_zero); break;
        case 64: gram_partial_kernel<64><<<nb, NT, 0, ctx->stream>>>(X, s_r, s_c, N, c, rc, scratch, skip_if_zero); break;
        default: gram_partial_kernel<128><<<nb, NT, 0, ctx->stream>>>(X, s_r, s_c, N, c, rc, scratch, skip_if_zero); break;
    }
    if (!launch_done(ctx, K_GRAM, 4.0 * N * c, (double)N * c * (c + 1))) return false;
    int npairs = c * (c + 1) / 2;
    prof_begin(ctx);
    gram_reduce_kernel<<<(npairs + 255) / 256, 256, 0, ctx->stream>>>(scratch, nb, c, G, G32, skip_if_zero);
    return launch_done(ctx, K_GRAM, 8.0 * nb * npairs + 12.0 * c * c, (double)nb * npairs);
}
