// tiles8.cu - the small dense products of a sweep on 8 x 8 register tiles.
//
//   xty8: out (cx x cy) = X^T Y, contraction over N (tens of thousands of rows):
//         T = B H^T (X = B^T stored n x l, Y = H^T) and W~ = Q^T W of
//         Algorithm 1's loop body; cx, cy <= 128.
//   ax8 : out (M x N) = A X, contraction over K <= 128, M large:
//         R^T = (B^T W~)^T of the H half (Algorithm 1's loop body).
//
// Both give each thread one 8 x 8 output tile and read operands as float4
// along the contraction from shared memory: 16 float4 reads feed 256 FMAs.
// Accuracy: xty8 sums a block's rows (at most ceil(N / (2 SMs)), a few hundred)
// in float32 and adds the block partials as two-sum pairs (pair_sum.cuh) in a
// fixed order; ax8 sums float32 products over at most 32 contraction steps and
// adds those (at most 4) sums in float32.  Results are deterministic; the rounding error is that of
// a float32 sum of a few hundred terms, relative to the sum of |terms|.
#include "async_copy.cuh"
#include "pair_sum.cuh"
#include "rnmf_internal.cuh"

namespace {

constexpr int NT = 256;
constexpr int RB = 32;     // contraction rows per stage
constexpr int CMAX = 128;  // output extent per side (both operands padded to it)

// swizzled position of stage row rr of operand row j: 16-byte chunks XOR (j / 8) mod 8
__device__ __forceinline__ int swz8(int j, int rr) { return (((rr >> 2) ^ ((j >> 3) & 7)) << 2) | (rr & 3); }

// One contraction step at a time over the whole tile: the 64 FMAs in a row are
// independent, so a warp can issue them back to back.
__device__ __forceinline__ void fma_tile(float (&acc)[8][8], const float4 (&a)[8], const float4 (&b)[8]) {
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(a[x].x, b[y].x, acc[x][y]);
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(a[x].y, b[y].y, acc[x][y]);
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(a[x].z, b[y].z, acc[x][y]);
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(a[x].w, b[y].w, acc[x][y]);
}

// ---------------------------------------------------------------- xty8
// Block b sums rows [b rchunk, (b + 1) rchunk).  Thread (tile, grp): tile
// (ti, tj) = (tile / tyc, tile % tyc) of the tx x ty tile grid, row group grp
// takes the 4-row chunks ch = grp (mod G) of every stage.  X (N x cx) has
// strides (sxr, sxc), Y (N x cy) strides (syr, syc); a column-major Y with
// 16-byte aligned columns (yvec) is copied in 16-byte pieces.  Stages are
// transposed into XsT[j][r] / YsT[j][r] and double-buffered.
__device__ __forceinline__ void stage_elems(float* dst, const float* __restrict__ src, int64_t sr, int64_t sc, int cnt,
                                            int cntp, int64_t r0, int64_t rend) {
    for (int e = threadIdx.x; e < cntp * RB; e += NT) {
        // consecutive threads take consecutive operand columns j when the rows are contiguous
        int j, rr;
        if (sc == 1) {
            j = e % cntp;
            rr = e / cntp;
        } else {
            j = e / RB;
            rr = e % RB;
        }
        const int64_t r = r0 + rr;
        const bool ok = j < cnt && r < rend;
        cp_async4(dst + j * RB + swz8(j, rr), ok ? src + r * sr + (int64_t)j * sc : src, ok);
    }
}

__global__ void __launch_bounds__(NT, 2) xty8_kernel(const float* __restrict__ X, int64_t sxr, int64_t sxc, int cx,
                                                    const float* __restrict__ Y, int64_t syr, int64_t syc, int cy,
                                                    int64_t N, int64_t rchunk, int tyc, int ntiles, int G, int yvec,
                                                    float* __restrict__ partial) {
    extern __shared__ __align__(16) float sm8[];
    float* XsT = sm8;                      // [2][CMAX][RB]
    float* YsT = sm8 + 2 * CMAX * RB;      // [2][CMAX][RB]
    const int tid = threadIdx.x;
    const int tile = tid % ntiles, grp = tid / ntiles;
    const bool active = grp < G;
    const int ti = tile / tyc, tj = tile % tyc;
    const int txc = ntiles / tyc;
    const int cxp = 8 * txc, cyp = 8 * tyc;
    const int64_t rbeg = (int64_t)blockIdx.x * rchunk;
    const int64_t rend = rbeg + rchunk < N ? rbeg + rchunk : N;
    auto load_stage = [&](int buf, int64_t r0) {
        float* xs = XsT + buf * CMAX * RB;
        float* ys = YsT + buf * CMAX * RB;
        stage_elems(xs, X, sxr, sxc, cx, cxp, r0, rend);
        if (yvec) {
            for (int e = tid; e < cyp * (RB / 4); e += NT) {
                const int j = e / (RB / 4), q = e % (RB / 4);
                const int64_t r = r0 + 4 * q;
                const int bytes = (j < cy && r < rend) ? (rend - r >= 4 ? 16 : (int)(rend - r) * 4) : 0;
                cp_async16_n(ys + j * RB + ((q ^ ((j >> 3) & 7)) << 2), bytes ? Y + (int64_t)j * syc + r : Y, bytes);
            }
        } else {
            stage_elems(ys, Y, syr, syc, cy, cyp, r0, rend);
        }
        cp_async_commit();
    };
    float hi[8][8];  // the block's float32 sums
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) hi[x][y] = 0.f;
    int buf = 0;
    if (rbeg < rend) load_stage(0, rbeg);
    for (int64_t r0 = rbeg; r0 < rend; r0 += RB) {
        if (r0 + RB < rend) {
            load_stage(buf ^ 1, r0 + RB);
            cp_async_wait_1();
        } else {
            cp_async_wait_0();
        }
        __syncthreads();
        if (active) {
            const float* xs = XsT + buf * CMAX * RB;
            const float* ys = YsT + buf * CMAX * RB;
            for (int ch = grp; ch < RB / 4; ch += G) {
                float4 b[8];
#pragma unroll
                for (int y = 0; y < 8; ++y)
                    b[y] = *reinterpret_cast<const float4*>(ys + (8 * tj + y) * RB + ((ch ^ (tj & 7)) << 2));
                // one operand row at a time keeps the live registers to 64 sums + 36
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    const float4 a = *reinterpret_cast<const float4*>(xs + (8 * ti + x) * RB + ((ch ^ (ti & 7)) << 2));
#pragma unroll
                    for (int y = 0; y < 8; ++y) hi[x][y] = fmaf(a.x, b[y].x, hi[x][y]);
#pragma unroll
                    for (int y = 0; y < 8; ++y) hi[x][y] = fmaf(a.y, b[y].y, hi[x][y]);
#pragma unroll
                    for (int y = 0; y < 8; ++y) hi[x][y] = fmaf(a.z, b[y].z, hi[x][y]);
#pragma unroll
                    for (int y = 0; y < 8; ++y) hi[x][y] = fmaf(a.w, b[y].w, hi[x][y]);
                }
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    // row groups added in group order (the stage buffers hold ntiles x 64 floats)
    for (int g = 1; g < G; ++g) {
        if (grp == g)
#pragma unroll
            for (int e = 0; e < 64; ++e) sm8[e * ntiles + tile] = hi[e / 8][e % 8];
        __syncthreads();
        if (grp == 0)
#pragma unroll
            for (int e = 0; e < 64; ++e) hi[e / 8][e % 8] += sm8[e * ntiles + tile];
        __syncthreads();
    }
    if (grp == 0)
#pragma unroll
        for (int e = 0; e < 64; ++e)
            partial[((int64_t)blockIdx.x * 64 + e) * ntiles + tile] = hi[e / 8][e % 8];
}

// Fixed-order sum of the block partials (group pg adds blocks pg, pg + 8, ...
// as a two-sum pair, the eight groups are added in order) and scatter into
// out(gi, gj) = out[gi so_r + gj so_c].
__global__ void __launch_bounds__(256) xty8_reduce_kernel(const float* __restrict__ partial, int nblk, int ntiles,
                                                          int tyc, int cx, int cy, float* __restrict__ out,
                                                          int64_t so_r, int64_t so_c, int accumulate) {
    __shared__ float2 red[8][32];
    const int E = ntiles * 64;
    const int el = threadIdx.x & 31, pg = threadIdx.x >> 5;
    const int t = blockIdx.x * 32 + el;
    float2 a = make_float2(0.f, 0.f);
    if (t < E) {
        for (int b0 = pg; b0 < nblk; b0 += 8 * 16) {
            float v[16];  // sixteen loads in flight; past the end adds +0
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = b0 + 8 * u < nblk ? partial[(int64_t)(b0 + 8 * u) * E + t] : 0.f;
#pragma unroll
            for (int u = 0; u < 16; ++u) two_sum_add(a, v[u]);
        }
    }
    red[pg][el] = a;
    __syncthreads();
    if (pg != 0 || t >= E) return;
    const int e = t / ntiles, tile = t % ntiles;
    const int gi = 8 * (tile / tyc) + e / 8, gj = 8 * (tile % tyc) + e % 8;
    if (gi >= cx || gj >= cy) return;
    float2 s = red[0][el];
#pragma unroll
    for (int q = 1; q < 8; ++q) s = pair_add(s, red[q][el]);
    float* o = out + gi * so_r + (int64_t)gj * so_c;
    if (accumulate) two_sum_add(s, *o);
    *o = pair_value(s);
}

void xty8_split(rnmf_ctx* ctx, int64_t N, int* nblk, int64_t* rchunk) {
    const int64_t target = (int64_t)ctx->num_sms * 2;  // two blocks per SM
    int64_t rc = (N + target - 1) / target;
    rc = (rc + RB - 1) / RB * RB;
    if (rc < RB) rc = RB;
    const int64_t nb = (N + rc - 1) / rc;
    *nblk = (int)(nb < 1 ? 1 : nb);
    *rchunk = rc;
}

// ---------------------------------------------------------------- ax8
// out (M x N) = A (M x K, row-major, lda) X (K x N, strides sx_r, sx_c), K <= 128,
// N <= 128.  Persistent blocks over 128-row tiles of A; X stays in shared
// memory (XsT[j][k], the whole contraction); A tiles are copied transposed,
// AsT[k][r], with cp.async into two buffers (the next tile loads while this
// one is multiplied).  Thread tile: rows 4 ti + {0..3} and 64 + 4 ti + {0..3}
// (ti fastest across threads, so 8 threads read 128 contiguous bytes of a
// stage row), columns 8 tj + {0..7}.
constexpr int AX_BM = 128;

__global__ void __launch_bounds__(NT, 1) ax8_kernel(const float* __restrict__ A, int64_t lda, const float* __restrict__ X,
                                                    int64_t sx_r, int64_t sx_c, float* __restrict__ out, int64_t so_r,
                                                    int64_t so_c, int64_t M, int N, int K, int accumulate) {
    extern __shared__ __align__(16) float sm8[];
    const int kp = (K + 31) / 32 * 32;  // contraction padded to whole 32-steps
    const int apitch = AX_BM + 4, xpitch = kp + 4;
    // two A buffers [kp][AX_BM + 4] at sm8 and sm8 + kp apitch, then XsT [8 tyc][kp + 4]
    float* XsT = sm8 + 2 * kp * apitch;
    const int tid = threadIdx.x;
    const int tyc = (N + 7) / 8;
    const int ntiles = (AX_BM / 8) * tyc;  // <= 16 x 16
    const bool active = tid < ntiles;
    const int ti = tid % (AX_BM / 8), tj = tid / (AX_BM / 8);
    // X^T once: XsT[j][k] = X(k, j), zero past K and N
    for (int e = tid; e < 8 * tyc * kp; e += NT) {
        const int j = e / kp, kk = e % kp;
        XsT[j * xpitch + kk] = (j < N && kk < K) ? X[(int64_t)kk * sx_r + (int64_t)j * sx_c] : 0.f;
    }
    auto load_tile = [&](float* dst, int64_t row0) {
        // consecutive threads copy consecutive k of one row of A
        for (int e = tid; e < AX_BM * kp; e += NT) {
            const int rr = e / kp, kk = e % kp;
            const int64_t r = row0 + rr;
            const bool ok = r < M && kk < K;
            cp_async4(dst + kk * apitch + rr, ok ? A + r * lda + kk : A, ok);
        }
        cp_async_commit();
    };
    const int64_t ntile_m = (M + AX_BM - 1) / AX_BM;
    int buf = 0;
    if ((int64_t)blockIdx.x < ntile_m) load_tile(sm8, (int64_t)blockIdx.x * AX_BM);
    for (int64_t bt = blockIdx.x; bt < ntile_m; bt += gridDim.x) {
        const int64_t nxt = bt + gridDim.x;
        if (nxt < ntile_m) {
            load_tile(sm8 + (buf ^ 1) * kp * apitch, nxt * AX_BM);
            cp_async_wait_1();
        } else {
            cp_async_wait_0();
        }
        __syncthreads();
        if (active) {
            const float* as = sm8 + buf * kp * apitch;
            float hi[8][8], acc[8][8];
#pragma unroll
            for (int x = 0; x < 8; ++x)
#pragma unroll
                for (int y = 0; y < 8; ++y) hi[x][y] = 0.f;
            for (int k0 = 0; k0 < kp; k0 += 32) {
#pragma unroll
                for (int x = 0; x < 8; ++x)
#pragma unroll
                    for (int y = 0; y < 8; ++y) acc[x][y] = 0.f;
#pragma unroll 2
                for (int kk = k0; kk < k0 + 32; kk += 4) {
                    float v[4][8];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 p0 = *reinterpret_cast<const float4*>(as + (kk + q) * apitch + 4 * ti);
                        const float4 p1 = *reinterpret_cast<const float4*>(as + (kk + q) * apitch + 64 + 4 * ti);
                        v[q][0] = p0.x; v[q][1] = p0.y; v[q][2] = p0.z; v[q][3] = p0.w;
                        v[q][4] = p1.x; v[q][5] = p1.y; v[q][6] = p1.z; v[q][7] = p1.w;
                    }
                    float4 a[8], b[8];
#pragma unroll
                    for (int x = 0; x < 8; ++x) a[x] = make_float4(v[0][x], v[1][x], v[2][x], v[3][x]);
#pragma unroll
                    for (int y = 0; y < 8; ++y)
                        b[y] = *reinterpret_cast<const float4*>(XsT + (8 * tj + y) * xpitch + kk);
                    fma_tile(acc, a, b);
                }
#pragma unroll
                for (int x = 0; x < 8; ++x)
#pragma unroll
                    for (int y = 0; y < 8; ++y) hi[x][y] += acc[x][y];
            }
            const int64_t row0 = bt * AX_BM;
#pragma unroll
            for (int y = 0; y < 8; ++y) {
                const int c = 8 * tj + y;
                if (c >= N) continue;
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    const int64_t r = row0 + (x < 4 ? 4 * ti + x : 64 + 4 * ti + x - 4);
                    if (r < M) {
                        float* o = out + r * so_r + (int64_t)c * so_c;
                        *o = accumulate ? *o + hi[x][y] : hi[x][y];
                    }
                }
            }
        }
        __syncthreads();  // buffer `buf` is refilled by the next iteration's prefetch
        buf ^= 1;
    }
}

}  // namespace

bool xty8_fits(int64_t M, int N) {
    return M >= 1 && N >= 1 && M <= CMAX && N <= CMAX && ((M + 7) / 8) * ((N + 7) / 8) <= NT;
}

size_t xty8_scratch_bytes(rnmf_ctx* ctx, int64_t M, int N, int64_t K) {
    if (!xty8_fits(M, N)) return 0;
    int nb;
    int64_t rc;
    xty8_split(ctx, K, &nb, &rc);
    return (size_t)nb * ((M + 7) / 8) * ((N + 7) / 8) * 64 * sizeof(float);
}

bool launch_xty8(rnmf_ctx* ctx, const float* Xr, int64_t sxr, int64_t sxc, int cx, const float* Y, int64_t syr,
                 int64_t syc, int cy, int64_t N, float* out, int64_t so_r, int64_t so_c, double* scratch,
                 bool accumulate) {
    const int tyc = (cy + 7) / 8, txc = (cx + 7) / 8, ntiles = txc * tyc;
    int G = NT / ntiles;
    if (G > 8) G = 8;
    int nb;
    int64_t rc;
    xty8_split(ctx, N, &nb, &rc);
    const int yvec = syr == 1 && (syc % 4 == 0) && ((reinterpret_cast<uintptr_t>(Y) & 15) == 0);
    const size_t smem = (size_t)4 * CMAX * RB * sizeof(float);
    cudaFuncSetAttribute(xty8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prof_begin(ctx);
    float* part = reinterpret_cast<float*>(scratch);  // [block][entry] float32 partials
    xty8_kernel<<<nb, NT, smem, ctx->stream>>>(Xr, sxr, sxc, cx, Y, syr, syc, cy, N, rc, tyc, ntiles, G, yvec,
                                               part);
    if (!launch_done(ctx, K_GEMM_ATX, 4.0 * ((double)N * cx + (double)N * cy), 2.0 * N * cx * cy)) return false;
    prof_begin(ctx);
    xty8_reduce_kernel<<<(ntiles * 64 + 31) / 32, 256, 0, ctx->stream>>>(part, nb, ntiles, tyc, cx, cy, out, so_r,
                                                                       so_c, accumulate ? 1 : 0);
    return launch_done(ctx, K_SPLITK, 4.0 * nb * ntiles * 64 + 4.0 * cx * cy, (double)nb * ntiles * 64);
}

bool ax8_fits(int N, int64_t K) { return N >= 1 && N <= CMAX && K >= 1 && K <= CMAX; }

bool launch_ax8(rnmf_ctx* ctx, const float* A, int64_t lda, const float* X, int64_t sx_r, int64_t sx_c, float* out,
                int64_t so_r, int64_t so_c, int64_t M, int N, int64_t K, bool accumulate) {
    const int kp = (int)((K + 31) / 32 * 32);
    const int tyc = (N + 7) / 8;
    const size_t smem = ((size_t)2 * kp * (AX_BM + 4) + (size_t)8 * tyc * (kp + 4)) * sizeof(float);
    cudaFuncSetAttribute(ax8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ax8_kernel, NT, smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    const int64_t tiles = (M + AX_BM - 1) / AX_BM;
    const int64_t slots = (int64_t)ctx->num_sms * occ;
    prof_begin(ctx);
    ax8_kernel<<<(unsigned)(tiles < slots ? tiles : slots), NT, smem, ctx->stream>>>(
        A, lda, X, sx_r, sx_c, out, so_r, so_c, M, N, (int)K, accumulate ? 1 : 0);
    return launch_done(ctx, K_GEMM_AX, 4.0 * ((double)M * K + (double)K * N + (double)M * N), 2.0 * M * N * K);
}
