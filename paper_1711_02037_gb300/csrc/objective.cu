// objective.cu - ||A - W H||_F^2 and ||A||_F^2 in float64.
//
// The relative error ||A - W H||_F / ||A||_F is the "Error" of the tables of
// Section 4; ||A - W H||_F^2 is the NMF objective of Section 2.2 (the stopping
// test of Section 3.3).  Each entry of W H is formed in float32 from k
// products, the difference with A is squared and accumulated in float64.
// Tiles of 64 x 64 entries; per-block partials are summed in a fixed order.
//
// The same kernel gives the compressed objective f~(W~, H) = ||B - W~ H||_F^2
// of Section 3.2 (launch_compobj): B^T (n x l) takes the place of A, H^T of W
// and W~^T of H.  It is evaluated as a residual, not by expanding the square
// into ||B||^2 - 2 <B H^T, W~> + <W~^T W~, H H^T>: near a good fit the three
// terms cancel to a few parts in 10^4 (or 10^5) of ||B||^2, so float32 rounding
// of B H^T alone would move the expanded value by ~1e-3 relative, while each
// float32 residual entry carries only its own rounding.
#include "rnmf_internal.cuh"

namespace {

constexpr int TILE = 64;
constexpr int NT = 256;

constexpr int KC = 32;  // k-slice per shared-memory stage

// Block b takes tile (b / nbx, b % nbx) of the ceil(m/64) x nbx tile grid (a 1-D
// grid, so m is not limited by the 65535 blocks of a grid's y extent).  H element
// (t, j) is at H[t sh_r + j sh_c].
__global__ void __launch_bounds__(NT) relerr_kernel(const float* __restrict__ A, int64_t lda,
                                                    const float* __restrict__ W, int64_t sw_r, int64_t sw_c,
                                                    const float* __restrict__ H, int64_t sh_r, int64_t sh_c,
                                                    int64_t m, int64_t n, int k, int64_t nbx,
                                                    double* __restrict__ part) {
    __shared__ __align__(16) float Ws[KC][TILE];  // Ws[t][i] = W(i0 + i, t0 + t)
    __shared__ __align__(16) float Hs[KC][TILE];  // Hs[t][j] = H(t0 + t, j0 + j)
    __shared__ double red[2][NT / 32];
    const int64_t blk = blockIdx.x;
    const int64_t i0 = (blk / nbx) * TILE, j0 = (blk % nbx) * TILE;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int t0 = 0; t0 < k; t0 += KC) {
        for (int e = threadIdx.x; e < KC * TILE; e += NT) {
            int t, i;
            if (sw_c == 1) {
                i = e / KC;
                t = e % KC;
            } else {
                t = e / TILE;
                i = e % TILE;
            }
            Ws[t][i] = (t0 + t < k && i0 + i < m) ? W[(i0 + i) * sw_r + (int64_t)(t0 + t) * sw_c] : 0.f;
        }
        for (int e = threadIdx.x; e < KC * TILE; e += NT) {
            int t = e / TILE, j = e % TILE;
            Hs[t][j] = (t0 + t < k && j0 + j < n) ? H[(int64_t)(t0 + t) * sh_r + (j0 + j) * sh_c] : 0.f;
        }
        __syncthreads();
        const int tend = k - t0 < KC ? k - t0 : KC;
        for (int t = 0; t < tend; ++t) {
            float4 w = *reinterpret_cast<const float4*>(&Ws[t][ty * 4]);
            float4 h = *reinterpret_cast<const float4*>(&Hs[t][tx * 4]);
            float wv[4] = {w.x, w.y, w.z, w.w}, hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(wv[a], hv[b], acc[a][b]);
        }
        __syncthreads();
    }
    double e2 = 0.0, a2 = 0.0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int64_t i = i0 + ty * 4 + a;
        if (i >= m) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int64_t j = j0 + tx * 4 + b;
            if (j >= n) continue;
            float av = A[i * lda + j];
            float d = av - acc[a][b];
            e2 = fma((double)d, (double)d, e2);
            a2 = fma((double)av, (double)av, a2);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (threadIdx.x % 32 == 0) {
        red[0][threadIdx.x / 32] = e2;
        red[1][threadIdx.x / 32] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < NT / 32; ++w) {
            s0 += red[0][w];
            s1 += red[1][w];
        }
        part[2 * blk] = s0;
        part[2 * blk + 1] = s1;
    }
}

__global__ void relerr_reduce_kernel(const double* __restrict__ part, int64_t nblk, double* __restrict__ out2) {
    __shared__ double red[2][32];
    double s0 = 0.0, s1 = 0.0;
    for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) {
        s0 += part[2 * b];
        s1 += part[2 * b + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (threadIdx.x % 32 == 0) {
        red[0][threadIdx.x / 32] = s0;
        red[1][threadIdx.x / 32] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
            t0 += red[0][w];
            t1 += red[1][w];
        }
        out2[0] = t0;
        out2[1] = t1;
    }
}

}  // namespace

size_t relerr_scratch_bytes(rnmf_ctx* ctx, int64_t m, int64_t n) {
    (void)ctx;
    int64_t nb = ((n + TILE - 1) / TILE) * ((m + TILE - 1) / TILE);
    return (size_t)nb * 2 * sizeof(double);
}

namespace {

bool relerr_tiles(rnmf_ctx* ctx, int cls, const float* A, int64_t lda, const float* W, int64_t sw_r, int64_t sw_c,
                  const float* H, int64_t sh_r, int64_t sh_c, int64_t m, int64_t n, int k, double* out2,
                  double* scratch) {
    const int64_t nbx = (n + TILE - 1) / TILE, nblk = nbx * ((m + TILE - 1) / TILE);
    if (nblk > 0x7fffffffLL) return false;
    prof_begin(ctx);
    relerr_kernel<<<(unsigned)nblk, NT, 0, ctx->stream>>>(A, lda, W, sw_r, sw_c, H, sh_r, sh_c, m, n, k, nbx, scratch);
    if (!launch_done(ctx, cls, 4.0 * ((double)m * n + (double)m * k + (double)k * n), 2.0 * m * n * k)) return false;
    prof_begin(ctx);
    relerr_reduce_kernel<<<1, 1024, 0, ctx->stream>>>(scratch, nblk, out2);
    return launch_done(ctx, cls, 16.0 * nblk, 0);
}

}  // namespace

bool launch_relerr(rnmf_ctx* ctx, const float* A, int64_t lda, const float* W, int64_t sw_r, int64_t sw_c,
                   const float* H, int64_t m, int64_t n, int k, double* out2, double* scratch) {
    return relerr_tiles(ctx, K_RELERR, A, lda, W, sw_r, sw_c, H, n, 1, m, n, k, out2, scratch);
}

size_t compobj_scratch_bytes(rnmf_ctx* ctx, int64_t n, int l) { return relerr_scratch_bytes(ctx, n, l); }

bool launch_compobj(rnmf_ctx* ctx, const float* Bt, int64_t n, int l, const float* Wt, int k, const float* H,
                    double* out2, double* scratch) {
    // rows c of B^T against (H^T W~^T)(c, :): W := H^T (element (c, j) at H[j n + c]),
    // H := W~^T (element (j, i) at Wt[i k + j])
    return relerr_tiles(ctx, K_COMPOBJ, Bt, l, H, 1, n, Wt, 1, k, n, l, k, out2, scratch);
}
