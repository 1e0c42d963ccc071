// gram.cu - G = X^T X (c x c, c <= 128).
//
// Used for the Gram matrix of CholeskyQR (the orthonormalisation qr() of
// Section 2.3 / Algorithm 1), and for S = W^T W and V = H H^T of a sweep
// (Algorithm 1 loop body).  Two arithmetic forms, both on CUDA cores (float64
// throughput is low on this GPU):
//   exact = true : every product x_i x_j is split exactly into p + e
//                  (p = x_i x_j, e = fma(x_i, x_j, -p)) and accumulated as a
//                  float32 pair (hi, lo) with TwoSum - a float64-class Gram for
//                  the ill-conditioned sketch Y of CholeskyQR;
//   exact = false: float32 products summed over 32-row stages, stage sums
//                  folded into a (sum, compensation) pair with TwoSum.
// Each thread owns 4 x 4 blocks of the upper triangle; rows are split over
// blocks of the grid and block partials are summed in float64 in a fixed order.
#include "rnmf_internal.cuh"

namespace {

constexpr int NT = 256;
constexpr int RB = 32;  // rows per shared-memory stage

__device__ __forceinline__ void two_sum(float& s, float& c, float v) {
    const float t = s + v;
    const float bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
}

template <int CP, bool EXACT>
__global__ void __launch_bounds__(NT) gram_partial_kernel(const float* __restrict__ X, int64_t s_r, int64_t s_c,
                                                          int64_t N, int c, int64_t rchunk,
                                                          double* __restrict__ partial,
                                                          const int* __restrict__ skip_if_zero) {
    if (skip_if_zero && *skip_if_zero == 0) return;
    constexpr int NB = CP / 4;                    // 4 x 4 blocks per side
    constexpr int NBLK = NB * (NB + 1) / 2;       // blocks of the upper triangle
    constexpr int BPT = (NBLK + NT - 1) / NT;     // blocks per thread
    __shared__ __align__(16) float Xs[RB][CP + 4];
    int bi[BPT], bj[BPT];
    float hi[BPT][16], lo[BPT][16];
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
        int b = threadIdx.x + q * NT, i = 0;
        while (i < NB && b >= NB - i) {
            b -= NB - i;
            ++i;
        }
        bi[q] = i < NB ? i : 0;
        bj[q] = i < NB ? i + b : 0;
#pragma unroll
        for (int e = 0; e < 16; ++e) hi[q][e] = lo[q][e] = 0.f;
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
            const int64_t r = r0 + rr;
            Xs[rr][j] = (j < c && r < rend) ? X[r * s_r + (int64_t)j * s_c] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < BPT; ++q) {
            if (threadIdx.x + q * NT >= NBLK) continue;
            if (EXACT) {
                for (int rr = 0; rr < RB; ++rr) {
                    const float4 a = *reinterpret_cast<const float4*>(&Xs[rr][4 * bi[q]]);
                    const float4 b = *reinterpret_cast<const float4*>(&Xs[rr][4 * bj[q]]);
                    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) {
                            const float p = av[x] * bv[y];
                            const float e = fmaf(av[x], bv[y], -p);
                            two_sum(hi[q][4 * x + y], lo[q][4 * x + y], p);
                            lo[q][4 * x + y] += e;
                        }
                }
            } else {
                float st[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) st[e] = 0.f;
#pragma unroll 4
                for (int rr = 0; rr < RB; ++rr) {
                    const float4 a = *reinterpret_cast<const float4*>(&Xs[rr][4 * bi[q]]);
                    const float4 b = *reinterpret_cast<const float4*>(&Xs[rr][4 * bj[q]]);
                    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) st[4 * x + y] = fmaf(av[x], bv[y], st[4 * x + y]);
                }
#pragma unroll
                for (int e = 0; e < 16; ++e) two_sum(hi[q][e], lo[q][e], st[e]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
        const int b = threadIdx.x + q * NT;
        if (b >= NBLK) continue;
#pragma unroll
        for (int e = 0; e < 16; ++e)
            partial[((int64_t)blockIdx.x * NBLK + b) * 16 + e] = (double)hi[q][e] + (double)lo[q][e];
    }
}

// Sum the block partials (fixed order, float64) and scatter the upper-triangle
// entries of the 4 x 4 blocks into the symmetric G (double) and G32 (float).
template <int CP>
__global__ void gram_reduce_kernel(const double* __restrict__ partial, int nblk, int c, double* __restrict__ G,
                                   float* __restrict__ G32, const int* __restrict__ skip_if_zero) {
    if (skip_if_zero && *skip_if_zero == 0) return;
    constexpr int NB = CP / 4;
    constexpr int NBLK = NB * (NB + 1) / 2;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < NBLK * 16; t += gridDim.x * blockDim.x) {
        int blk = t / 16, i = 0;
        const int e = t % 16;
        while (blk >= NB - i) {
            blk -= NB - i;
            ++i;
        }
        const int gi = 4 * i + e / 4, gj = 4 * (i + blk) + e % 4;
        if (gi >= c || gj >= c || gi > gj) continue;  // lower entries of diagonal blocks: mirrored from above
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * NBLK * 16 + t];
        G[gi * c + gj] = s;
        G[gj * c + gi] = s;
        if (G32) {
            G32[gi * c + gj] = (float)s;
            G32[gj * c + gi] = (float)s;
        }
    }
}

int cpad(int c) { return c <= 16 ? 16 : c <= 32 ? 32 : c <= 64 ? 64 : 128; }

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

template <int CP>
bool gram_launch(rnmf_ctx* ctx, const float* X, int64_t s_r, int64_t s_c, int64_t N, int c, double* G, float* G32,
                 double* scratch, const int* skip, bool exact) {
    int nb;
    int64_t rc;
    gram_split(ctx, N, &nb, &rc);
    prof_begin(ctx);
    if (exact)
        gram_partial_kernel<CP, true><<<nb, NT, 0, ctx->stream>>>(X, s_r, s_c, N, c, rc, scratch, skip);
    else
        gram_partial_kernel<CP, false><<<nb, NT, 0, ctx->stream>>>(X, s_r, s_c, N, c, rc, scratch, skip);
    if (!launch_done(ctx, K_GRAM, 4.0 * N * c, (double)N * c * (c + 1))) return false;
    constexpr int NBLK = (CP / 4) * (CP / 4 + 1) / 2;
    prof_begin(ctx);
    gram_reduce_kernel<CP><<<(NBLK * 16 + 255) / 256, 256, 0, ctx->stream>>>(scratch, nb, c, G, G32, skip);
    return launch_done(ctx, K_GRAM, 8.0 * nb * NBLK * 16 + 12.0 * c * c, (double)nb * NBLK * 16);
}

}  // namespace

size_t gram_scratch_bytes(rnmf_ctx* ctx, int64_t N, int c) {
    int nb;
    int64_t rc;
    gram_split(ctx, N, &nb, &rc);
    const int nbk = cpad(c) / 4;
    return (size_t)nb * (nbk * (nbk + 1) / 2) * 16 * sizeof(double);
}

bool launch_gram(rnmf_ctx* ctx, const float* X, int64_t s_r, int64_t s_c, int64_t N, int c, double* G, float* G32,
                 double* scratch, const int* skip_if_zero, bool exact) {
    switch (cpad(c)) {
        case 16: return gram_launch<16>(ctx, X, s_r, s_c, N, c, G, G32, scratch, skip_if_zero, exact);
        case 32: return gram_launch<32>(ctx, X, s_r, s_c, N, c, G, G32, scratch, skip_if_zero, exact);
        case 64: return gram_launch<64>(ctx, X, s_r, s_c, N, c, G, G32, scratch, skip_if_zero, exact);
        default: return gram_launch<128>(ctx, X, s_r, s_c, N, c, G, G32, scratch, skip_if_zero, exact);
    }
}
