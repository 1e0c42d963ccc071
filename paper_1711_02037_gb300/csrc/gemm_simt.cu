// gemm_simt.cu - skinny FP32 products on CUDA cores.
//
// Used for every product of the FP32 form of the randomized QB (Y = A Omega,
// Z = A^T Q, Y = A Q, B^T = A^T Q; Section 2.3 / Algorithm 1) and for the
// small dense products of a sweep (R = B^T W~, T = B H^T, W~ = Q^T W;
// Algorithm 1 loop body).  The output has at most 128 columns (l or k).
//
// Accuracy: each thread sums a 32-long slice of the contraction in float32,
// then folds the slice sum into a (sum, compensation) pair with Knuth's
// TwoSum, so the error does not grow with the contraction length (tens of
// thousands here).  Split-K partials are combined in float64 in a fixed order,
// so results are deterministic.
#include "async_copy.cuh"
#include "f32x2.cuh"
#include "rnmf_internal.cuh"

namespace {

constexpr int BM = 64;   // output rows per block
constexpr int BK = 32;   // contraction slice per shared-memory stage
constexpr int NT = 256;  // threads per block

__device__ __forceinline__ void two_sum_acc(float& s, float& c, float v) {
    float t = s + v;
    float bp = t - s;
    float e = (s - (t - bp)) + (v - bp);
    c += e;
    s = t;
}

// Shared tile compute: acc[4][TN] = sum_kk As[kk][ty*4+i] * Xs[kk][tx+16j].
template <int NP>
__device__ __forceinline__ void tile_fma(const float (*As)[BM + 4], const float (*Xs)[NP + 1], int tx, int ty,
                                         float acc[4][NP / 16]) {
    constexpr int TN = NP / 16;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
        float4 a4 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
        float a[4] = {a4.x, a4.y, a4.z, a4.w};
        float x[TN];
#pragma unroll
        for (int j = 0; j < TN; ++j) x[j] = Xs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], x[j], acc[i][j]);
    }
}

template <int NP>
__device__ __forceinline__ void load_x_tile(float (*Xs)[NP + 1], const float* __restrict__ X, int64_t sx_r,
                                            int64_t sx_c, int N, int64_t k0, int64_t kend) {
    for (int e = threadIdx.x; e < BK * NP; e += NT) {
        int kk, j;
        if (sx_c == 1) {
            kk = e / NP;
            j = e % NP;
        } else {
            j = e / BK;
            kk = e % BK;
        }
        const int64_t r = k0 + kk;
        const bool ok = j < N && r < kend;
        cp_async4(&Xs[kk][j], ok ? X + r * sx_r + (int64_t)j * sx_c : X, ok);
    }
}

// out (M x N) = A (M x K, row-major, lda) * X (K x N, strided).
template <int NP>
__global__ void __launch_bounds__(NT) gemm_ax_kernel(const float* __restrict__ A, int64_t lda,
                                                     const float* __restrict__ X, int64_t sx_r, int64_t sx_c,
                                                     float* __restrict__ out, int64_t so_r, int64_t so_c,
                                                     int64_t M, int N, int64_t K, int accumulate) {
    constexpr int TN = NP / 16;
    __shared__ __align__(16) float As[BK][BM + 4];
    __shared__ __align__(16) float Xs[BK][NP + 1];  // +1: conflict-free column-wise fills
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t row0 = (int64_t)blockIdx.x * BM;
    float sum[4][TN], comp[4][TN], acc[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) sum[i][j] = comp[i][j] = 0.f;

    // A-tile loader mapping: thread -> (row = t % 64, 8 consecutive k at (t / 64) * 8)
    const int lrow = threadIdx.x % BM;
    const int lk = (threadIdx.x / BM) * 8;
    const int64_t grow = row0 + lrow;
    const bool vec_ok = ((lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);

    for (int64_t k0 = 0; k0 < K; k0 += BK) {
        float v[8];
        if (grow < M) {
            const float* src = A + grow * lda + k0 + lk;
            if (vec_ok && k0 + lk + 8 <= K) {
                float4 p = *reinterpret_cast<const float4*>(src);
                float4 q = *reinterpret_cast<const float4*>(src + 4);
                v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w;
                v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = (k0 + lk + e < K) ? src[e] : 0.f;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = 0.f;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) As[lk + e][lrow] = v[e];
        load_x_tile<NP>(Xs, X, sx_r, sx_c, N, k0, K);
        cp_async_wait_all();
        __syncthreads();
        tile_fma<NP>(As, Xs, tx, ty, acc);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) two_sum_acc(sum[i][j], comp[i][j], acc[i][j]);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t r = row0 + ty * 4 + i;
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int c = tx + 16 * j;
            if (c < N) {
                float* o = out + r * so_r + (int64_t)c * so_c;
                *o = accumulate ? *o + (sum[i][j] + comp[i][j]) : sum[i][j] + comp[i][j];
            }
        }
    }
}

// out (M x N) = A^T X with A (K x M, row-major, lda), X (K x N, strided); the
// contraction is split over `gridDim.y` chunks of `kchunk` rows of A.
template <int NP>
__global__ void __launch_bounds__(NT) gemm_atx_kernel(const float* __restrict__ A, int64_t lda,
                                                      const float* __restrict__ X, int64_t sx_r, int64_t sx_c,
                                                      float* __restrict__ out, int64_t so_r, int64_t so_c,
                                                      int64_t M, int N, int64_t K, int64_t kchunk,
                                                      double* __restrict__ partial, int accumulate) {
    constexpr int TN = NP / 16;
    __shared__ __align__(16) float As[BK][BM + 4];
    __shared__ __align__(16) float Xs[BK][NP + 1];  // +1: conflict-free column-wise fills
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t col0 = (int64_t)blockIdx.x * BM;
    const int64_t kbeg = (int64_t)blockIdx.y * kchunk;
    const int64_t kend = kbeg + kchunk < K ? kbeg + kchunk : K;
    float sum[4][TN], comp[4][TN], acc[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) sum[i][j] = comp[i][j] = 0.f;

    // A-tile loader: thread -> (kk = t / 8, 8 consecutive columns at (t % 8) * 8)
    const int lkk = threadIdx.x / 8;
    const int li = (threadIdx.x % 8) * 8;
    const bool vec_ok = ((lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);

    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
        float v[8];
        int64_t r = k0 + lkk;
        int64_t c = col0 + li;
        if (r < kend) {
            const float* src = A + r * lda + c;
            if (vec_ok && c + 8 <= M) {
                float4 p = *reinterpret_cast<const float4*>(src);
                float4 q = *reinterpret_cast<const float4*>(src + 4);
                v[0] = p.x; v[1] = p.y; v[2] = p.z; v[3] = p.w;
                v[4] = q.x; v[5] = q.y; v[6] = q.z; v[7] = q.w;
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = (c + e < M) ? src[e] : 0.f;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = 0.f;
        }
        *reinterpret_cast<float4*>(&As[lkk][li]) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4*>(&As[lkk][li + 4]) = make_float4(v[4], v[5], v[6], v[7]);
        load_x_tile<NP>(Xs, X, sx_r, sx_c, N, k0, kend);
        cp_async_wait_all();
        __syncthreads();
        tile_fma<NP>(As, Xs, tx, ty, acc);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) two_sum_acc(sum[i][j], comp[i][j], acc[i][j]);
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t rr = col0 + ty * 4 + i;
        if (rr >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int cc = tx + 16 * j;
            if (cc >= N) continue;
            if (gridDim.y == 1) {
                float* o = out + rr * so_r + (int64_t)cc * so_c;
                *o = accumulate ? *o + (sum[i][j] + comp[i][j]) : sum[i][j] + comp[i][j];
            }
            else
                partial[((int64_t)blockIdx.y * M + rr) * N + cc] = (double)sum[i][j] + (double)comp[i][j];
        }
    }
}

// ---------------------------------------------------------------- 128-row kernels
// The QB's products over A (and deterministic HALS's A^T W, A H^T) on larger
// register tiles: a block owns 128 rows x NP <= 64 columns (wider outputs take
// several column blocks, adjacent in launch order so that the second reads A's
// tile from L2), each thread 8 rows x NP/16 columns, so one shared-memory read
// of A feeds NP/16 FMAs and one read of X feeds 8; two blocks per SM; stages are
// copied with cp.async into double buffers (the next stage's copy overlaps this
// stage's products); the FMAs run as packed pairs (f32x2.cuh).  Per 32-long
// slice of the contraction the float32 partial is folded into the (sum,
// compensation) pair as above, so the accuracy is that of the 64-row kernels.
constexpr int GM = 128;     // output rows per block
constexpr int GN = 64;      // output columns per block at most
constexpr int GP = GM + 4;  // pitch of a stage of A (floats): rows of 16-byte aligned float4s

template <int NP>
struct GShape {
    static constexpr int TN = NP / 16;      // columns per thread (tx + 16 j)
    static constexpr int XP = NP + 4;       // pitch of a stage of X
    static constexpr int AS = GM * (BK + 4) > BK * GP ? GM * (BK + 4) : BK * GP;  // floats of a stage of A
    static constexpr int STAGE = AS + BK * XP;
    static constexpr size_t SMEM = 2 * (size_t)STAGE * sizeof(float);
};

// A stage of the AX product, row-major: As[r][kk] = A[(row0 + r) lda + k0 + kk] (pitch
// GPA; eight consecutive threads copy one row's 32 floats, 16 bytes each where aligned).
constexpr int GPA = BK + 4;
__device__ __forceinline__ void g_stage_a_ax(float* As, const float* __restrict__ A, int64_t lda, int64_t row0,
                                             int64_t M, int64_t k0, int64_t kend, bool vec) {
#pragma unroll
    for (int t = 0; t < GM * BK / (4 * NT); ++t) {
        const int e = threadIdx.x + NT * t;
        const int r = e / (BK / 4), kk = (e % (BK / 4)) * 4;
        const int64_t gr = row0 + r, gk = k0 + kk;
        float* dst = As + r * GPA + kk;
        if (vec) {
            const int64_t left = gr < M ? kend - gk : 0;
            const int bytes = left >= 4 ? 16 : (left > 0 ? (int)left * 4 : 0);
            cp_async16_n(dst, bytes > 0 ? A + gr * lda + gk : A, bytes);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool ok = gr < M && gk + q < kend;
                cp_async4(dst + q, ok ? A + gr * lda + gk + q : A, ok);
            }
        }
    }
}
// A stage of the ATX product: As[kk][c] = A[(k0 + kk) lda + col0 + c] (rows of A
// are contiguous along c: 16-byte copies where aligned).
__device__ __forceinline__ void g_stage_a_atx(float* As, const float* __restrict__ A, int64_t lda, int64_t col0,
                                              int64_t M, int64_t k0, int64_t kend, bool vec) {
#pragma unroll
    for (int t = 0; t < GM * BK / (4 * NT); ++t) {
        const int e = threadIdx.x + NT * t;
        const int kk = e / (GM / 4), c = (e % (GM / 4)) * 4;
        const int64_t gk = k0 + kk, gc = col0 + c;
        float* dst = As + kk * GP + c;
        if (vec) {
            const int64_t left = gk < kend ? M - gc : 0;
            const int bytes = left >= 4 ? 16 : (left > 0 ? (int)left * 4 : 0);
            cp_async16_n(dst, bytes > 0 ? A + gk * lda + gc : A, bytes);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool ok = gk < kend && gc + q < M;
                cp_async4(dst + q, ok ? A + gk * lda + gc + q : A, ok);
            }
        }
    }
}
// A stage of X (K x N, strides sx_r, sx_c) into Xs[kk][j] (pitch XP), zero past N and kend.
template <int NP>
__device__ __forceinline__ void g_stage_x(float* Xs, const float* __restrict__ X, int64_t sx_r, int64_t sx_c, int N,
                                          int64_t k0, int64_t kend) {  // X and N: from the block's first column
    constexpr int XP = GShape<NP>::XP;
    for (int e = threadIdx.x; e < BK * NP; e += NT) {
        int kk, j;
        if (sx_c == 1) {
            kk = e / NP;
            j = e % NP;
        } else {
            j = e / BK;
            kk = e % BK;
        }
        const int64_t r = k0 + kk;
        const bool ok = j < N && r < kend;
        cp_async4(Xs + kk * XP + j, ok ? X + r * sx_r + (int64_t)j * sx_c : X, ok);
    }
}

// acc[i][j] += sum_kk As[kk][8 ty + i] Xs[kk][tx + 16 j] over one stage; pairs of
// columns (2 q, 2 q + 1) as packed FMAs, an odd last column as a scalar FMA.
template <int NP>
__device__ __forceinline__ void g_stage_fma(const float* As, const float* Xs, int tx, int ty,
                                            float (&acc)[8][GShape<NP>::TN]) {
    constexpr int TN = GShape<NP>::TN, XP = GShape<NP>::XP;
    const float* ap = As + 8 * ty;
    const float* xp = Xs + tx;
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(ap + kk * GP);
        const float4 a1 = *reinterpret_cast<const float4*>(ap + kk * GP + 4);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        float x[TN];
#pragma unroll
        for (int j = 0; j < TN; ++j) x[j] = xp[kk * XP + 16 * j];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float2 aa = make_float2(a[i], a[i]);
#pragma unroll
            for (int q = 0; q + 1 < TN; q += 2) {
                const float2 r = f2_fma(aa, make_float2(x[q], x[q + 1]), make_float2(acc[i][q], acc[i][q + 1]));
                acc[i][q] = r.x;
                acc[i][q + 1] = r.y;
            }
            if (TN & 1) acc[i][TN - 1] = fmaf(a[i], x[TN - 1], acc[i][TN - 1]);
        }
    }
}

// AX form of the stage products: A row-major (pitch GPA); thread ty owns rows
// 4 ty + i and 64 + 4 ty + i (i < 4), so the two row groups of a warp's lanes sit
// 16 banks apart; one 8-byte read gives a row's next two contraction values.
template <int NP>
__device__ __forceinline__ void g_stage_fma_ax(const float* As, const float* Xs, int tx, int ty,
                                               float (&acc)[8][GShape<NP>::TN]) {
    constexpr int TN = GShape<NP>::TN, XP = GShape<NP>::XP;
    const float* xp = Xs + tx;
#pragma unroll 1
    for (int kk = 0; kk < BK; kk += 2) {
        float2 ra[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            ra[i] = *reinterpret_cast<const float2*>(As + (4 * ty + (i & 3) + 64 * (i >> 2)) * GPA + kk);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            float x[TN];
#pragma unroll
            for (int j = 0; j < TN; ++j) x[j] = xp[(kk + u) * XP + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float ai = u ? ra[i].y : ra[i].x;
                const float2 aa = make_float2(ai, ai);
#pragma unroll
                for (int q = 0; q + 1 < TN; q += 2) {
                    const float2 r = f2_fma(aa, make_float2(x[q], x[q + 1]), make_float2(acc[i][q], acc[i][q + 1]));
                    acc[i][q] = r.x;
                    acc[i][q + 1] = r.y;
                }
                if (TN & 1) acc[i][TN - 1] = fmaf(ai, x[TN - 1], acc[i][TN - 1]);
            }
        }
    }
}

// mode 0 (AX): out (M x N) = A (M x K, lda) X (K x N);  mode 1 (ATX): out (M x N) =
// A^T X with A (K x M, lda); the contraction split over gridDim.y chunks of kchunk
// (more than one: float64 partials, added by splitk_reduce_kernel).
// Block x: row tile x / ncb, column block x % ncb (columns c0 .. c0 + NP - 1).
template <int NP, int MODE>
__global__ void __launch_bounds__(NT, 2) gemm_big_kernel(const float* __restrict__ A, int64_t lda,
                                                          const float* __restrict__ X, int64_t sx_r, int64_t sx_c,
                                                          float* __restrict__ out, int64_t so_r, int64_t so_c,
                                                          int64_t M, int N, int64_t K, int64_t kchunk,
                                                          double* __restrict__ partial, int accumulate, int ncb) {
    using Sh = GShape<NP>;
    constexpr int TN = Sh::TN;
    extern __shared__ __align__(16) float gsm[];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t row0 = (int64_t)(blockIdx.x / ncb) * GM;
    const int c0 = (int)(blockIdx.x % ncb) * NP;
    const int nb = N - c0 < NP ? N - c0 : NP;  // columns of this block
    const float* Xb = X + (int64_t)c0 * sx_c;
    const int64_t kbeg = (int64_t)blockIdx.y * kchunk;
    const int64_t kend = kbeg + kchunk < K ? kbeg + kchunk : K;
    const bool vec = ((lda & 3) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
    float sum[8][TN], comp[8][TN], acc[8][TN];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) sum[i][j] = comp[i][j] = 0.f;
    auto stage = [&](int b, int64_t k0) {
        float* As = gsm + b * Sh::STAGE;
        float* Xs = As + Sh::AS;
        if (MODE == 0) g_stage_a_ax(As, A, lda, row0, M, k0, kend, vec);
        else g_stage_a_atx(As, A, lda, row0, M, k0, kend, vec);
        g_stage_x<NP>(Xs, Xb, sx_r, sx_c, nb, k0, kend);
        cp_async_commit();
    };
    if (kbeg < kend) stage(0, kbeg);
    int b = 0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += BK, b ^= 1) {
        if (k0 + BK < kend) {
            stage(b ^ 1, k0 + BK);
            cp_async_wait_1();
        } else {
            cp_async_wait_0();
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
        const float* As = gsm + b * Sh::STAGE;
        if (MODE == 0) g_stage_fma_ax<NP>(As, As + Sh::AS, tx, ty, acc);
        else g_stage_fma<NP>(As, As + Sh::AS, tx, ty, acc);
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) two_sum_acc(sum[i][j], comp[i][j], acc[i][j]);
        __syncthreads();  // this buffer is refilled by the stage after next
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = row0 + (MODE == 0 ? 4 * ty + (i & 3) + 64 * (i >> 2) : ty * 8 + i);
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int c = c0 + tx + 16 * j;
            if (tx + 16 * j >= nb) continue;
            if (gridDim.y > 1) {
                partial[((int64_t)blockIdx.y * M + r) * N + c] = (double)sum[i][j] + (double)comp[i][j];
            } else {
                float* o = out + r * so_r + (int64_t)c * so_c;
                *o = accumulate ? *o + (sum[i][j] + comp[i][j]) : sum[i][j] + comp[i][j];
            }
        }
    }
}

// out = sum of the split-K partials.  A block handles 32 consecutive outputs with
// 8 groups of threads: group pg sums partials p = pg (mod 8) (loads batched), and
// the 8 group sums are added in group order - the same fixed order for every run.
__global__ void __launch_bounds__(256) splitk_reduce_kernel(const double* __restrict__ partial, int splits, int64_t M,
                                                            int N, float* __restrict__ out, int64_t so_r,
                                                            int64_t so_c, int accumulate) {
    __shared__ double red[8][32];
    const int64_t total = M * N;
    const int el = threadIdx.x & 31, pg = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * 32 + el;
    double a = 0.0;
    if (e < total) {
        int p = pg;
        for (; p + 24 < splits; p += 32) {
            const double v0 = partial[(int64_t)p * total + e], v1 = partial[(int64_t)(p + 8) * total + e];
            const double v2 = partial[(int64_t)(p + 16) * total + e], v3 = partial[(int64_t)(p + 24) * total + e];
            a += (v0 + v1) + (v2 + v3);
        }
        for (; p < splits; p += 8) a += partial[(int64_t)p * total + e];
    }
    red[pg][el] = a;
    __syncthreads();
    if (pg == 0 && e < total) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) s += red[q][el];
        const int64_t r = e / N;
        const int c = (int)(e % N);
        float* o = out + r * so_r + (int64_t)c * so_c;
        *o = accumulate ? (float)((double)*o + s) : (float)s;
    }
}

// Output width padded to a multiple of 16 (16 threads x TN columns).
int padded_n(int N) { return N <= 16 ? 16 : N >= 128 ? 128 : (N + 15) / 16 * 16; }

// The 128-row kernels take the products with many output rows (one block per
// SM: their register tiles hold 8 x NP/16 entries three times over).
constexpr int64_t BIG_M = 4096;
bool use_big(int64_t M) { return M >= BIG_M; }

int big_ncb(int N) { return (N + GN - 1) / GN; }
int big_np(int N) { return padded_n((N + big_ncb(N) - 1) / big_ncb(N)); }  // even column blocks

void atx_split(rnmf_ctx* ctx, int64_t M, int N, int64_t K, int* splits, int64_t* kchunk) {
    if (use_big(M) && K > 128) {
        // blocks = tiles x column blocks x splits, two resident per SM: the split count
        // (at least two waves, chunks of >= 512) that best fills the last wave
        const int64_t blocks = (M + GM - 1) / GM * big_ncb(N);
        const int64_t slots = 2 * (int64_t)ctx->num_sms;
        int64_t smax = (K + 511) / 512;
        if (smax < 1) smax = 1;
        int64_t s0 = (2 * slots + blocks - 1) / blocks;
        if (s0 > smax) s0 = smax;
        if (s0 < 1) s0 = 1;
        int64_t best = s0;
        double best_eff = -1.0;
        for (int64_t s2 = s0; s2 <= 2 * s0 + 4 && s2 <= smax; ++s2) {
            const double units = (double)blocks * s2;
            const double eff = units / (std::ceil(units / slots) * slots);
            if (eff > best_eff + 0.02) {
                best_eff = eff;
                best = s2;
            }
        }
        int64_t kc = (K + best - 1) / best;
        kc = (kc + BK - 1) / BK * BK;
        *kchunk = kc;
        *splits = (int)((K + kc - 1) / kc);
        return;
    }
    const bool big = false;
    int64_t tiles = (M + (big ? GM : BM) - 1) / (big ? GM : BM);
    int64_t target = (int64_t)ctx->num_sms * (big ? 2 : 4);
    int64_t s = (target + tiles - 1) / tiles;
    int64_t smax = (K + 511) / 512;
    if (s > smax) s = smax;
    if (s < 1) s = 1;
    int64_t kc = (K + s - 1) / s;
    kc = (kc + BK - 1) / BK * BK;
    if (kc < BK) kc = BK;
    s = (K + kc - 1) / kc;
    if (s < 1) s = 1;
    *splits = (int)s;
    *kchunk = kc;
}

}  // namespace

size_t gemm_ax_scratch_bytes(rnmf_ctx* ctx, int64_t M, int N, int64_t K) {
    if (ax8_fits(N, K) || !use_big(M)) return 0;
    int splits;
    int64_t kc;
    atx_split(ctx, M, N, K, &splits, &kc);
    return splits > 1 ? (size_t)splits * M * N * sizeof(double) : 0;
}

bool launch_gemm_ax(rnmf_ctx* ctx, const float* A, int64_t lda, const float* X, int64_t sx_r, int64_t sx_c,
                    float* out, int64_t so_r, int64_t so_c, int64_t M, int N, int64_t K, bool accumulate,
                    double* scratch) {
    if (M <= 0 || N <= 0) return true;
    if (ax8_fits(N, K)) return launch_ax8(ctx, A, lda, X, sx_r, sx_c, out, so_r, so_c, M, N, K, accumulate);
    if (use_big(M)) {
        const int ncb = big_ncb(N);
        int splits = 1;
        int64_t kc = K;
        if (scratch) atx_split(ctx, M, N, K, &splits, &kc);  // without scratch: one split
        dim3 g((unsigned)((M + GM - 1) / GM * ncb), (unsigned)splits);
        prof_begin(ctx);
        switch (big_np(N)) {
#define RNMF_BAX(NPV)                                                                                              \
    case NPV:                                                                                                      \
        cudaFuncSetAttribute(gemm_big_kernel<NPV, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,                 \
                             (int)GShape<NPV>::SMEM);                                                              \
        gemm_big_kernel<NPV, 0><<<g, NT, GShape<NPV>::SMEM, ctx->stream>>>(A, lda, X, sx_r, sx_c, out, so_r, so_c, \
                                                                           M, N, K, kc, scratch, accumulate ? 1 : 0, ncb); \
        break;
            RNMF_BAX(16) RNMF_BAX(32) RNMF_BAX(48)
            default: RNMF_BAX(64)
#undef RNMF_BAX
        }
        if (!launch_done(ctx, K_GEMM_AX, 4.0 * ((double)M * K + (double)K * N + (double)M * N), 2.0 * M * N * K))
            return false;
        if (splits > 1) {
            const int64_t total = M * N;
            prof_begin(ctx);
            splitk_reduce_kernel<<<(unsigned)((total + 31) / 32), 256, 0, ctx->stream>>>(scratch, splits, M, N, out,
                                                                                          so_r, so_c,
                                                                                          accumulate ? 1 : 0);
            return launch_done(ctx, K_SPLITK, 8.0 * splits * M * N + 4.0 * M * N, (double)splits * M * N);
        }
        return true;
    }
    dim3 grid((unsigned)((M + BM - 1) / BM));
    prof_begin(ctx);
    switch (padded_n(N)) {
#define RNMF_AX(NPV) \
    case NPV: gemm_ax_kernel<NPV><<<grid, NT, 0, ctx->stream>>>(A, lda, X, sx_r, sx_c, out, so_r, so_c, M, N, K, accumulate ? 1 : 0); break;
        RNMF_AX(16) RNMF_AX(32) RNMF_AX(48) RNMF_AX(64) RNMF_AX(80) RNMF_AX(96) RNMF_AX(112)
#undef RNMF_AX
        default: gemm_ax_kernel<128><<<grid, NT, 0, ctx->stream>>>(A, lda, X, sx_r, sx_c, out, so_r, so_c, M, N, K, accumulate ? 1 : 0); break;
    }
    return launch_done(ctx, K_GEMM_AX, 4.0 * ((double)M * K + (double)K * N + (double)M * N), 2.0 * M * N * K);
}

size_t gemm_atx_scratch_bytes(rnmf_ctx* ctx, int64_t M, int N, int64_t K) {
    if (xty8_fits(M, N)) return xty8_scratch_bytes(ctx, M, N, K);
    int splits;
    int64_t kc;
    atx_split(ctx, M, N, K, &splits, &kc);
    return splits > 1 ? (size_t)splits * M * N * sizeof(double) : 0;
}

bool launch_gemm_atx(rnmf_ctx* ctx, const float* A, int64_t lda, const float* X, int64_t sx_r, int64_t sx_c,
                     float* out, int64_t so_r, int64_t so_c, int64_t M, int N, int64_t K, double* scratch,
                     bool accumulate) {
    if (M <= 0 || N <= 0) return true;
    if (xty8_fits(M, N))  // out = A^T X: A (K x M) as X^T Y's first operand, X as its second
        return launch_xty8(ctx, A, lda, 1, (int)M, X, sx_r, sx_c, N, K, out, so_r, so_c, scratch, accumulate);
    int splits;
    int64_t kc;
    atx_split(ctx, M, N, K, &splits, &kc);
    if (use_big(M)) {
        const int ncb = big_ncb(N);
        dim3 g((unsigned)((M + GM - 1) / GM * ncb), (unsigned)splits);
        prof_begin(ctx);
        switch (big_np(N)) {
#define RNMF_BATX(NPV)                                                                                             \
    case NPV:                                                                                                      \
        cudaFuncSetAttribute(gemm_big_kernel<NPV, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,                 \
                             (int)GShape<NPV>::SMEM);                                                              \
        gemm_big_kernel<NPV, 1><<<g, NT, GShape<NPV>::SMEM, ctx->stream>>>(A, lda, X, sx_r, sx_c, out, so_r, so_c, \
                                                                           M, N, K, kc, scratch,                   \
                                                                           accumulate ? 1 : 0, ncb);               \
        break;
            RNMF_BATX(16) RNMF_BATX(32) RNMF_BATX(48)
            default: RNMF_BATX(64)
#undef RNMF_BATX
        }
    } else {
    dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)splits);
    prof_begin(ctx);
    switch (padded_n(N)) {
#define RNMF_ATX(NPV) \
    case NPV: gemm_atx_kernel<NPV><<<grid, NT, 0, ctx->stream>>>(A, lda, X, sx_r, sx_c, out, so_r, so_c, M, N, K, kc, scratch, accumulate ? 1 : 0); break;
        RNMF_ATX(16) RNMF_ATX(32) RNMF_ATX(48) RNMF_ATX(64) RNMF_ATX(80) RNMF_ATX(96) RNMF_ATX(112)
#undef RNMF_ATX
        default: gemm_atx_kernel<128><<<grid, NT, 0, ctx->stream>>>(A, lda, X, sx_r, sx_c, out, so_r, so_c, M, N, K, kc, scratch, accumulate ? 1 : 0); break;
    }
    }
    if (!launch_done(ctx, K_GEMM_ATX, 4.0 * ((double)M * K + (double)K * N + (double)M * N), 2.0 * M * N * K))
        return false;
    if (splits > 1) {
        const int64_t total = M * N;
        const int g = (int)((total + 31) / 32);
        prof_begin(ctx);
        splitk_reduce_kernel<<<g, 256, 0, ctx->stream>>>(scratch, splits, M, N, out, so_r, so_c, accumulate ? 1 : 0);
        return launch_done(ctx, K_SPLITK, 8.0 * splits * M * N + 4.0 * M * N, (double)splits * M * N);
    }
    return true;
}
