// batched.cu - kernels of the batched ragged randomized HALS path.
//
// Randomized QB (Section 2.3, Algorithm 1) for every problem of a batch in
// shared launches: tile kernels walk a list of row (column) tiles of all
// problems, taking the next tile from an atomic counter, so that problems of
// very different sizes share the GPU without one launch per problem.  The
// compressed sweeps (Section 3.2) then run with one thread-block cluster per
// problem: the rows of Q and W and the columns of H and B^T are split over the
// cluster's CTAs, the small matrices W~, S, T, V are replicated in every CTA's
// shared memory, and the partial sums behind them are combined through
// distributed shared memory in rank order (so every CTA holds the same values).
#include <cooperative_groups.h>

#include "async_copy.cuh"
#include "batched.cuh"
#include "philox.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int TNT = 256;  // threads of the tile kernels
constexpr int BK = 32;    // contraction slice of the tile products

constexpr uint32_t STREAM_OMEGA = 1, STREAM_W_INIT = 2, STREAM_H_INIT = 3;

__device__ __forceinline__ bool gated(const RbInst& d, int gate) { return d.q < gate; }

// ------------------------------------------------------------------ Omega
// One block row of the grid per problem; Box-Muller pairs (Gaussian) or words
// (uniform) of the row-major n x l matrix, stored in Z with pitch ldq and zero
// padding columns.
__global__ void __launch_bounds__(256) rb_omega_kernel(const RbInst* __restrict__ I, int count) {
    const int i = blockIdx.y;
    if (i >= count) return;
    const RbInst& d = I[i];
    const int l = d.l, ldq = d.ldq;
    const int64_t total = (int64_t)d.n * l;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float* Z = d.Z;
    if (d.omega_dist == 0) {
        for (int64_t b = t0; b < (total + 1) / 2; b += stride) {
            float z0, z1;
            rnmf_rng::gauss_pair(d.seed, STREAM_OMEGA, d.inst, (uint64_t)b, &z0, &z1);
            const int64_t e0 = 2 * b, e1 = e0 + 1;
            Z[(e0 / l) * ldq + e0 % l] = z0;
            if (e1 < total) Z[(e1 / l) * ldq + e1 % l] = z1;
        }
    } else {
        for (int64_t b = t0; b < (total + 3) / 4; b += stride) {
            uint32_t w[4];
            rnmf_rng::block(d.seed, STREAM_OMEGA, d.inst, (uint64_t)b, w);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int64_t e = 4 * b + t;
                if (e < total) Z[(e / l) * ldq + e % l] = (float)(w[t] >> 8) * 0x1p-24f;
            }
        }
    }
    if (ldq > l)
        for (int64_t r = t0; r < d.n; r += stride)
            for (int t = l; t < ldq; ++t) Z[r * ldq + t] = 0.f;
}

// W_init (m x k, stored transposed in Wc) and H_init (k x n) ~ U[0,1), key seed + 1.
__global__ void __launch_bounds__(256) rb_init_kernel(const RbInst* __restrict__ I, int count) {
    const int i = blockIdx.y;
    if (i >= count) return;
    const RbInst& d = I[i];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = d.k;
    const int64_t m = d.m, n = d.n;
    for (int64_t b = t0; b < (m * k + 3) / 4; b += stride) {
        uint32_t w[4];
        rnmf_rng::block(d.seed + 1, STREAM_W_INIT, d.inst, (uint64_t)b, w);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t e = 4 * b + t;
            if (e < m * k) d.Wc[(e % k) * m + e / k] = (float)(w[t] >> 8) * 0x1p-24f;
        }
    }
    for (int64_t b = t0; b < ((int64_t)k * n + 3) / 4; b += stride) {
        uint32_t w[4];
        rnmf_rng::block(d.seed + 1, STREAM_H_INIT, d.inst, (uint64_t)b, w);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t e = 4 * b + t;
            if (e < (int64_t)k * n) d.H[e] = (float)(w[t] >> 8) * 0x1p-24f;
        }
    }
}

// ------------------------------------------------------------------ tile products
// 4 x 4 register block: acc[a][b] += As[kk][r0 + a] * Xs[kk][c0 + b] over kk.
__device__ __forceinline__ void fma_block(float (&acc)[4][4], const float4 a, const float4 x) {
    const float av[4] = {a.x, a.y, a.z, a.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], xv[q], acc[p][q]);
}

__device__ __forceinline__ int next_tile(int* counter, int* s_tile) {
    __syncthreads();
    if (threadIdx.x == 0) *s_tile = atomicAdd(counter, 1);
    __syncthreads();
    return *s_tile;
}

// Row tiles: out rows [r0, r1) = src rows [r0, r1) (K columns) times X (K x l).
//   mode 0: Y = A Z; mode 1: Y = Y Rinv; mode 2: Z = Z Rinv (in place: a tile
//   reads all of its rows before it writes them).
__global__ void __launch_bounds__(TNT) rb_rows_kernel(const RbInst* __restrict__ I, const RbTile* __restrict__ tiles,
                                                      int ntiles, int* counter, int mode, int only_shifted, int gate) {
    __shared__ __align__(16) float As[BK][RB_BMAX + 4];
    __shared__ __align__(16) float Xs[BK][RB_MAX_L + 4];
    __shared__ int s_tile;
    const int tid = threadIdx.x;
    for (;;) {
        const int ti = next_tile(counter, &s_tile);
        if (ti >= ntiles) return;
        const RbTile tl = tiles[ti];
        const RbInst& d = I[tl.inst];
        if (gated(d, gate) || (only_shifted && !d.shifted)) continue;
        const int l = d.l, ldq = d.ldq;
        const float* src;
        const float* X;
        float* out;
        int64_t lds;
        int ldx, K;
        if (mode == 0) {
            src = d.A; lds = d.lda; X = d.Z; ldx = ldq; out = d.Y; K = d.n;
        } else if (mode == 1) {
            src = d.Y; lds = ldq; X = d.Rinv; ldx = l; out = d.Y; K = l;
        } else {
            src = d.Z; lds = ldq; X = d.Rinv; ldx = l; out = d.Z; K = l;
        }
        const int ncb = (l + 3) >> 2, nrb = d.bm >> 2;
        const int rows = tl.r1 - tl.r0;
        const int rb = tid / ncb, cb = tid % ncb;
        const bool active = tid < nrb * ncb;
        float acc[4][4] = {};
        for (int k0 = 0; k0 < K; k0 += BK) {
            for (int e = tid; e < d.bm * BK; e += TNT) {
                const int r = e / BK, kk = e % BK;
                As[kk][r] = (r < rows && k0 + kk < K) ? src[(int64_t)(tl.r0 + r) * lds + k0 + kk] : 0.f;
            }
            for (int e = tid; e < BK * ncb * 4; e += TNT) {
                const int kk = e / (ncb * 4), t = e % (ncb * 4);
                Xs[kk][t] = (k0 + kk < K && t < l) ? X[(int64_t)(k0 + kk) * ldx + t] : 0.f;
            }
            __syncthreads();
            if (active) {
                const int kend = K - k0 < BK ? K - k0 : BK;
                for (int kk = 0; kk < kend; ++kk)
                    fma_block(acc, *reinterpret_cast<const float4*>(&As[kk][rb * 4]),
                              *reinterpret_cast<const float4*>(&Xs[kk][cb * 4]));
            }
            __syncthreads();
        }
        if (active) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int r = rb * 4 + a;
                if (r >= rows) continue;
                float* o = out + (int64_t)(tl.r0 + r) * ldq;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int t = cb * 4 + b;
                    if (t < ldq) o[t] = t < l ? acc[a][b] : 0.f;
                }
            }
        }
    }
}

// Double-buffered products over A (the two passes per power iteration that read
// A from HBM).  Stage s + 1 is copied with cp.async while stage s is multiplied.
// A's rows are copied in 16-byte pieces when lda % 4 == 0 and A is 16-byte
// aligned, else element by element; pieces past the matrix edge are zero-filled.
constexpr int PB_BK = 32;                 // contraction slice per stage
constexpr int PB_PA = PB_BK + 4;          // sketch: A stage row pitch (rows of A are tile rows)
constexpr int PB_PT = RB_BMAX + 4;        // A^T Y: A stage row pitch (rows of A are the slice)
constexpr int PB_PX = RB_MAX_L + 4;       // X stage pitch
constexpr int SK_STAGE = RB_BMAX * PB_PA + PB_BK * PB_PX;
constexpr int AT_STAGE = PB_BK * PB_PT + PB_BK * PB_PX;

__device__ __forceinline__ bool a_vec_ok(const RbInst& d) {
    return (d.lda & 3) == 0 && (reinterpret_cast<uintptr_t>(d.A) & 15) == 0;
}

// X slice: rows [k0, k0 + PB_BK) of a row-major (K x ldq) matrix, zero past K.
__device__ __forceinline__ void stage_x(float* Xs, const float* X, int ldq, int64_t k0, int64_t K) {
    const int nc = ldq >> 2;
    for (int e = threadIdx.x; e < PB_BK * nc; e += TNT) {
        const int kk = e / nc, c = e % nc;
        const bool ok = k0 + kk < K;
        cp_async16_n(Xs + kk * PB_PX + 4 * c, ok ? X + (k0 + kk) * ldq + 4 * c : X, ok ? 16 : 0);
    }
}

// Y = A Z over row tiles (sketch and the second product of a power iteration).
__global__ void __launch_bounds__(TNT) rb_sketch_kernel(const RbInst* __restrict__ I,
                                                        const RbTile* __restrict__ tiles, int ntiles, int* counter,
                                                        int gate) {
    extern __shared__ __align__(16) float pbuf[];
    __shared__ int s_tile;
    const int tid = threadIdx.x;
    for (;;) {
        const int ti = next_tile(counter, &s_tile);
        if (ti >= ntiles) return;
        const RbTile tl = tiles[ti];
        const RbInst& d = I[tl.inst];
        if (gated(d, gate)) continue;
        const int l = d.l, ldq = d.ldq, bm = d.bm;
        const int64_t K = d.n, lda = d.lda;
        const float* A = d.A;
        const bool vec = a_vec_ok(d);
        const int ncb = (l + 3) >> 2, nrb = bm >> 2;
        const int rows = tl.r1 - tl.r0;
        const int rb = tid / ncb, cb = tid % ncb;
        const bool active = tid < nrb * ncb;
        auto load = [&](int stage, int64_t k0) {
            float* As = pbuf + stage * SK_STAGE;
            if (vec) {
                for (int e = tid; e < bm * (PB_BK / 4); e += TNT) {
                    const int r = e / (PB_BK / 4), c = e % (PB_BK / 4);
                    const int64_t kk = k0 + 4 * c;
                    int nb = 0;
                    if (r < rows && kk < K) nb = K - kk >= 4 ? 16 : (int)(K - kk) * 4;
                    cp_async16_n(As + r * PB_PA + 4 * c, nb ? A + (int64_t)(tl.r0 + r) * lda + kk : A, nb);
                }
            } else {
                for (int e = tid; e < bm * PB_BK; e += TNT) {
                    const int r = e / PB_BK, kk = e % PB_BK;
                    const bool ok = r < rows && k0 + kk < K;
                    cp_async4(As + r * PB_PA + kk, ok ? A + (int64_t)(tl.r0 + r) * lda + k0 + kk : A, ok);
                }
            }
            stage_x(As + RB_BMAX * PB_PA, d.Z, ldq, k0, K);
            cp_async_commit();
        };
        float acc[4][4] = {};
        const int nk = (int)((K + PB_BK - 1) / PB_BK);
        load(0, 0);
        for (int kt = 0; kt < nk; ++kt) {
            if (kt + 1 < nk) {
                load((kt + 1) & 1, (int64_t)(kt + 1) * PB_BK);
                cp_async_wait_1();
            } else {
                cp_async_wait_0();
            }
            __syncthreads();
            if (active) {
                const float* As = pbuf + (kt & 1) * SK_STAGE;
                const float* Xs = As + RB_BMAX * PB_PA;
#pragma unroll 2
                for (int k4 = 0; k4 < PB_BK / 4; ++k4) {
                    float4 a[4];
#pragma unroll
                    for (int p = 0; p < 4; ++p) a[p] = *reinterpret_cast<const float4*>(As + (rb * 4 + p) * PB_PA + 4 * k4);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 x = *reinterpret_cast<const float4*>(Xs + (4 * k4 + q) * PB_PX + cb * 4);
                        const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const float av = q == 0 ? a[p].x : q == 1 ? a[p].y : q == 2 ? a[p].z : a[p].w;
#pragma unroll
                            for (int b = 0; b < 4; ++b) acc[p][b] = fmaf(av, xv[b], acc[p][b]);
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (active) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int r = rb * 4 + a;
                if (r >= rows) continue;
                float* o = d.Y + (int64_t)(tl.r0 + r) * ldq;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int t = cb * 4 + b;
                    if (t < ldq) o[t] = t < l ? acc[a][b] : 0.f;
                }
            }
        }
    }
}

// Z = A^T Y over column tiles of A, contraction over the m rows.
__global__ void __launch_bounds__(TNT) rb_atx_kernel(const RbInst* __restrict__ I, const RbTile* __restrict__ tiles,
                                                     int ntiles, int* counter, int gate) {
    extern __shared__ __align__(16) float pbuf[];
    __shared__ int s_tile;
    const int tid = threadIdx.x;
    for (;;) {
        const int ti = next_tile(counter, &s_tile);
        if (ti >= ntiles) return;
        const RbTile tl = tiles[ti];
        const RbInst& d = I[tl.inst];
        if (gated(d, gate)) continue;
        const int l = d.l, ldq = d.ldq, bm = d.bm;
        const int64_t K = d.m, lda = d.lda;
        const float* A = d.A;
        const bool vec = a_vec_ok(d);
        const int ncb = (l + 3) >> 2, nrb = bm >> 2;
        const int cols = tl.r1 - tl.r0;
        const int rb = tid / ncb, cb = tid % ncb;
        const bool active = tid < nrb * ncb;
        auto load = [&](int stage, int64_t k0) {
            float* As = pbuf + stage * AT_STAGE;
            if (vec) {
                const int nc = bm >> 2;
                for (int e = tid; e < PB_BK * nc; e += TNT) {
                    const int kk = e / nc, c = e % nc;
                    int nb = 0;
                    if (k0 + kk < K && 4 * c < cols) nb = cols - 4 * c >= 4 ? 16 : (cols - 4 * c) * 4;
                    cp_async16_n(As + kk * PB_PT + 4 * c, nb ? A + (k0 + kk) * lda + tl.r0 + 4 * c : A, nb);
                }
            } else {
                for (int e = tid; e < PB_BK * bm; e += TNT) {
                    const int kk = e / bm, c = e % bm;
                    const bool ok = k0 + kk < K && c < cols;
                    cp_async4(As + kk * PB_PT + c, ok ? A + (k0 + kk) * lda + tl.r0 + c : A, ok);
                }
            }
            stage_x(As + PB_BK * PB_PT, d.Y, ldq, k0, K);
            cp_async_commit();
        };
        float acc[4][4] = {};
        const int nk = (int)((K + PB_BK - 1) / PB_BK);
        load(0, 0);
        for (int kt = 0; kt < nk; ++kt) {
            if (kt + 1 < nk) {
                load((kt + 1) & 1, (int64_t)(kt + 1) * PB_BK);
                cp_async_wait_1();
            } else {
                cp_async_wait_0();
            }
            __syncthreads();
            if (active) {
                const float* As = pbuf + (kt & 1) * AT_STAGE;
                const float* Xs = As + PB_BK * PB_PT;
#pragma unroll 4
                for (int kk = 0; kk < PB_BK; ++kk)
                    fma_block(acc, *reinterpret_cast<const float4*>(As + kk * PB_PT + rb * 4),
                              *reinterpret_cast<const float4*>(Xs + kk * PB_PX + cb * 4));
            }
            __syncthreads();
        }
        if (active) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int c = rb * 4 + a;
                if (c >= cols) continue;
                float* o = d.Z + (int64_t)(tl.r0 + c) * ldq;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int t = cb * 4 + b;
                    if (t < ldq) o[t] = t < l ? acc[a][b] : 0.f;
                }
            }
        }
    }
}

// ------------------------------------------------------------------ CholeskyQR
// Error-free accumulation: every product x*y is split exactly into p + e
// (e = fma(x, y, -p)) and added to a float pair (s, c) with TwoSum (Knuth), so
// s + c carries the chunk's sum to about 2^-48 relative.
__device__ __forceinline__ void pair_acc(float& s, float& c, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float e = fmaf(x, y, -p);
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
}

constexpr int GRAM_MAXP = (RB_MAX_L * (RB_MAX_L + 1) / 2 + TNT - 1) / TNT;

// Partial Gram matrix of rows [r0, r1) (at most RB_GR) of Y (which 0) or Z
// (which 1), written as float64 to chunk r0 / RB_GR of the problem's gpart.
__global__ void __launch_bounds__(TNT) rb_gram_kernel(const RbInst* __restrict__ I, const RbTile* __restrict__ tiles,
                                                      int ntiles, int* counter, int which, int only_shifted,
                                                      int gate) {
    __shared__ float Xs[64][RB_MAX_L + 1];
    __shared__ int s_tile;
    const int tid = threadIdx.x;
    for (;;) {
        const int ti = next_tile(counter, &s_tile);
        if (ti >= ntiles) return;
        const RbTile tl = tiles[ti];
        const RbInst& d = I[tl.inst];
        if (gated(d, gate) || (only_shifted && !d.shifted)) continue;
        const int l = d.l, ldq = d.ldq;
        const float* X = which ? d.Z : d.Y;
        const int P = l * (l + 1) / 2;
        int pa[GRAM_MAXP], pb[GRAM_MAXP];
        float s[GRAM_MAXP], c[GRAM_MAXP];
#pragma unroll
        for (int q = 0; q < GRAM_MAXP; ++q) {
            int p = tid + q * TNT, a = 0;
            if (p < P) {
                while (p >= l - a) {
                    p -= l - a;
                    ++a;
                }
                pa[q] = a;
                pb[q] = a + p;
            } else {
                pa[q] = pb[q] = -1;
            }
            s[q] = c[q] = 0.f;
        }
        for (int s0 = tl.r0; s0 < tl.r1; s0 += 64) {
            const int nr = tl.r1 - s0 < 64 ? tl.r1 - s0 : 64;
            __syncthreads();
            for (int e = tid; e < 64 * l; e += TNT) {
                const int rr = e / l, t = e % l;
                Xs[rr][t] = rr < nr ? X[(int64_t)(s0 + rr) * ldq + t] : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < GRAM_MAXP; ++q) {
                if (pa[q] < 0) continue;
                for (int rr = 0; rr < nr; ++rr) pair_acc(s[q], c[q], Xs[rr][pa[q]], Xs[rr][pb[q]]);
            }
        }
        double* G = d.gpart + (size_t)(tl.r0 / RB_GR) * l * l;
#pragma unroll
        for (int q = 0; q < GRAM_MAXP; ++q) {
            if (pa[q] < 0) continue;
            const double v = (double)s[q] + (double)c[q];
            G[pa[q] * l + pb[q]] = v;
            G[pb[q] * l + pa[q]] = v;
        }
    }
}

// One block per problem: G = sum of the partial Grams (fixed chunk order),
// upper Cholesky factor R (float64) and Rinv = R^{-1} (float32).
//   pass 0: a breakdown retries with the shift 11 (N l + l (l + 1)) 2^-53 trace(G)
//           (shifted CholeskyQR) and marks the problem `shifted`;
//   pass 1: no shift; pass 2: only for shifted problems.
// A breakdown that the shift does not cure sets the problem's status to
// RNMF_DEV_NOTPD and leaves Rinv = I.
constexpr int CNT = 128;

__global__ void __launch_bounds__(CNT) rb_chol_kernel(RbInst* __restrict__ I, int count, int which, int pass,
                                                      int gate) {
    __shared__ double Gs[RB_MAX_L * RB_MAX_L];
    __shared__ double diag[RB_MAX_L];
    __shared__ int fail;
    __shared__ double shift;
    const int i = blockIdx.x;
    if (i >= count) return;
    RbInst& d = I[i];
    if (gated(d, gate)) return;
    if (pass == 2 && !d.shifted) return;
    const int l = d.l, tid = threadIdx.x;
    const int64_t N = which ? d.n : d.m;
    const int nch = (int)((N + RB_GR - 1) / RB_GR);
    int used_shift = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
        for (int e = tid; e < l * l; e += CNT) {
            double g = 0.0;
            for (int ch = 0; ch < nch; ++ch) g += d.gpart[(size_t)ch * l * l + e];
            Gs[e] = g;
        }
        __syncthreads();
        if (tid == 0) {
            fail = 0;
            shift = 0.0;
            if (attempt == 1) {
                double tr = 0.0;
                for (int a = 0; a < l; ++a) tr += Gs[a * l + a];
                shift = 11.0 * ((double)N * l + (double)l * (l + 1)) * 0x1p-53 * tr;
            }
        }
        __syncthreads();
        for (int a = tid; a < l; a += CNT) Gs[a * l + a] += shift;
        __syncthreads();
        for (int j = 0; j < l; ++j) {
            if (tid == 0) {
                const double v = Gs[j * l + j];
                if (!(v > 0.0) || !isfinite(v))
                    fail = 1;
                else
                    Gs[j * l + j] = sqrt(v);
            }
            __syncthreads();
            if (fail) break;
            const double dj = Gs[j * l + j];
            for (int t = j + 1 + tid; t < l; t += CNT) Gs[j * l + t] /= dj;
            __syncthreads();
            for (int e = tid; e < (l - j - 1) * (l - j - 1); e += CNT) {
                const int ii = j + 1 + e / (l - j - 1), tt = j + 1 + e % (l - j - 1);
                if (tt >= ii) Gs[ii * l + tt] -= Gs[j * l + ii] * Gs[j * l + tt];
            }
            __syncthreads();
        }
        __syncthreads();
        if (!fail) break;
        if (pass != 0 || attempt == 1) {
            if (tid == 0) d.status = RNMF_DEV_NOTPD;
            for (int e = tid; e < l * l; e += CNT) d.Rinv[e] = (e / l == e % l) ? 1.f : 0.f;
            if (pass == 0 && tid == 0) d.shifted = 1;
            return;
        }
        used_shift = 1;
        __syncthreads();
    }
    // X = R^{-1} (upper); X[a][jc] kept in Gs[jc][a] (the unused lower part)
    for (int a = tid; a < l; a += CNT) diag[a] = Gs[a * l + a];
    __syncthreads();
    for (int a = tid; a < l; a += CNT) Gs[a * l + a] = 1.0 / diag[a];
    __syncthreads();
    for (int a = l - 2; a >= 0; --a) {
        for (int jc = a + 1 + tid; jc < l; jc += CNT) {
            double sum = 0.0;
            for (int t = a + 1; t <= jc; ++t) sum = fma(Gs[a * l + t], Gs[jc * l + t], sum);
            Gs[jc * l + a] = -sum / diag[a];
        }
        __syncthreads();
    }
    for (int e = tid; e < l * l; e += CNT) {
        const int a = e / l, b = e % l;
        d.Rinv[e] = a <= b ? (float)Gs[b * l + a] : 0.f;
    }
    if (pass == 0 && tid == 0) d.shifted = used_shift;
}

// ------------------------------------------------------------------ sweeps
// Partial sums of 4 x 4 output blocks are kept in registers by NT / blocks
// groups of threads; group sums are added in group order (fixed, so that every
// run and every CTA of a cluster rounds the same way).
template <int NT>
__device__ __forceinline__ void group_sum(const float (&acc)[4][4], bool act, int g, int blk, int nblk, int G,
                                          float* gred) {
    if (act)
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) gred[(g * nblk + blk) * 16 + p * 4 + q] = acc[p][q];
    __syncthreads();
}

__device__ __forceinline__ float group_read(const float* gred, int G, int nblk, int blk, int p, int q) {
    float s = 0.f;
    for (int g = 0; g < G; ++g) s += gred[(g * nblk + blk) * 16 + p * 4 + q];
    return s;
}

// out[a][b] (pitch KM, zeros outside A x B, outA rows) = sum over rows r in
// [r0, r1) of X(r, a) Y(r, b), X(r, a) = X[r xr + a xa], Y(r, b) = Y[r yr + b yb];
// rows are staged 32 at a time (used once per problem, for W~ = Q^T W_init).
template <int NT, int LQ, int KM>
__device__ void block_gram(const float* __restrict__ X, int64_t xr, int64_t xa, int A, const float* __restrict__ Y,
                           int64_t yr, int64_t yb, int B, int64_t r0, int64_t r1, float* stX, float* stY,
                           float* gred, float* out, int outA) {
    constexpr int PX = LQ + 4, PY = KM + 4;
    const int na = (A + 3) >> 2, nb = (B + 3) >> 2, nblk = na * nb;
    const int G = NT / nblk;
    const int tid = threadIdx.x, g = tid / nblk, blk = tid % nblk, ab = blk / nb, bb = blk % nb;
    const bool act = g < G;
    float acc[4][4] = {};
    for (int64_t s0 = r0; s0 < r1; s0 += 32) {
        const int rows = r1 - s0 < 32 ? (int)(r1 - s0) : 32;
        __syncthreads();
        for (int e = tid; e < 32 * na * 4; e += NT) {
            int rr, a;
            if (xa == 1) {
                rr = e / (na * 4);
                a = e % (na * 4);
            } else {
                a = e / 32;
                rr = e % 32;
            }
            stX[rr * PX + a] = (rr < rows && a < A) ? X[(s0 + rr) * xr + a * xa] : 0.f;
        }
        for (int e = tid; e < 32 * nb * 4; e += NT) {
            int rr, b;
            if (yb == 1) {
                rr = e / (nb * 4);
                b = e % (nb * 4);
            } else {
                b = e / 32;
                rr = e % 32;
            }
            stY[rr * PY + b] = (rr < rows && b < B) ? Y[(s0 + rr) * yr + b * yb] : 0.f;
        }
        __syncthreads();
        if (act)
            for (int rr = g; rr < rows; rr += G)
                fma_block(acc, *reinterpret_cast<const float4*>(&stX[rr * PX + ab * 4]),
                          *reinterpret_cast<const float4*>(&stY[rr * PY + bb * 4]));
    }
    __syncthreads();
    group_sum<NT>(acc, act, g, blk, nblk, G, gred);
    for (int e = tid; e < outA * KM; e += NT) {
        const int a = e / KM, b = e % KM;
        out[e] = (a < A && b < B) ? group_read(gred, G, nblk, (a >> 2) * nb + (b >> 2), a & 3, b & 3) : 0.f;
    }
    __syncthreads();
}

// dst[e * dst_stride] = sum over cluster ranks (in order) of slot[e], e < cnt.
template <int NT>
__device__ void cluster_sum(cg::cluster_group& cl, int C, float* slot, int cnt, float* dst, int dst_stride) {
    if (C == 1) {
        __syncthreads();
        for (int e = threadIdx.x; e < cnt; e += NT) dst[e * dst_stride] = slot[e];
        __syncthreads();
        return;
    }
    cl.sync();
    for (int e = threadIdx.x; e < cnt; e += NT) {
        float sum = 0.f;
        for (int r = 0; r < C; ++r) sum += cl.map_shared_rank(slot, r)[e];
        dst[e * dst_stride] = sum;
    }
    __syncthreads();
}

// Sum of v[] over the 32 lanes of a warp, scattered: after the call lane L holds
// the sums for indices rs_index<LQ>(L, i), i < rs_count<LQ>() (recursive halving:
// about LQ shuffles instead of 5 LQ).
template <int LQ>
__device__ __forceinline__ void warp_reduce_scatter(float (&v)[LQ], int lane) {
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int o = 16 >> s;
        if ((LQ >> s) >= 2) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < (LQ >> (s + 1)); ++i) {
                const float send = up ? v[i] : v[i + (LQ >> (s + 1))];
                const float keep = up ? v[i + (LQ >> (s + 1))] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
    }
}

template <int LQ>
__device__ __forceinline__ int rs_index(int lane, int i) {
    int base = 0, cnt = LQ;
#pragma unroll
    for (int s = 0; s < 5; ++s)
        if (cnt >= 2) {
            cnt >>= 1;
            if (lane & (16 >> s)) base += cnt;
        }
    return base + i;
}

template <int LQ>
constexpr int rs_count() {
    return LQ >= 32 ? LQ / 32 : 1;
}

template <int NT, int LQ, int KM>
struct SweepSmem {
    static constexpr int SLOT = LQ * KM + KM * KM;
    static constexpr int PH = KM + 4;
    static constexpr int STAGE = 32 * (LQ + 4) + 32 * (KM + 4);
    static constexpr int CHUNK = NT * PH > STAGE ? NT * PH : STAGE;
    static constexpr int floats = 2 * LQ * KM + 2 * KM * KM + LQ + 2 * SLOT + (NT / 32) * LQ + CHUNK + 16 * NT;
};

// One cluster per problem (list[blockIdx.x / C]).  CTA `rank` owns rows
// [m rank / C, m (rank + 1) / C) of Q and W and columns [n rank / C, ...) of H
// and B^T.  Per sweep: H half fused with T = B H^T and V = H H^T (one cluster
// reduction), the k columns of the W half (one reduction each), S = W^T W (one).
template <int NT, int LQ, int KM>
__global__ void __launch_bounds__(NT, 1) rb_sweeps_kernel(RbInst* __restrict__ I, const int* __restrict__ list,
                                                          int count, int iters_override) {
    using SM = SweepSmem<NT, LQ, KM>;
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int rank = (int)cl.block_rank();
    const int ci = blockIdx.x / C;
    if (ci >= count) return;  // whole clusters only: the grid is C * count
    const RbInst& d = I[list[ci]];
    const int m = d.m, n = d.n, k = d.k, l = d.l, ldq = d.ldq, gram_mode = d.gram_mode;
    const int iters = iters_override >= 0 ? iters_override : d.iters;
    const int64_t R0 = (int64_t)m * rank / C, R1 = (int64_t)m * (rank + 1) / C;
    const int64_t C0 = (int64_t)n * rank / C, C1 = (int64_t)n * (rank + 1) / C;
    const float* __restrict__ Q = d.Y;
    const float* __restrict__ Bt = d.Z;
    float* __restrict__ Hg = d.H;
    float* __restrict__ Wc = d.Wc;

    extern __shared__ __align__(16) float sm[];
    float* Wt = sm;                   // LQ x KM: W~
    float* S = Wt + LQ * KM;          // KM x KM
    float* T = S + KM * KM;           // LQ x KM
    float* V = T + LQ * KM;           // KM x KM (follows T: one reduction fills both)
    float* u = V + KM * KM;           // LQ
    float* slots = u + LQ;            // 2 x SLOT
    float* red = slots + 2 * SM::SLOT;
    float* chunk = red + (NT / 32) * LQ;  // NT x PH (H columns / W rows), or the 32-row stages
    float* gred = chunk + SM::CHUNK;
    int par = 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nbl = (l + 3) >> 2, nbk = (k + 3) >> 2;

    // S = W^T W over this CTA's rows, NT rows at a time through shared memory
    auto compute_S = [&]() {
        if (gram_mode == 0) {
            const int nblk = nbk * nbk, G = NT / nblk, g = tid / nblk, blk = tid % nblk;
            const int ib = blk / nbk, jb = blk % nbk;
            const bool act = g < G;
            float acc[4][4] = {};
            for (int64_t rb0 = R0; rb0 < R1; rb0 += NT) {
                const int64_t r = rb0 + tid;
                const int nrows = R1 - rb0 < NT ? (int)(R1 - rb0) : NT;
#pragma unroll
                for (int j = 0; j < KM; ++j) chunk[tid * SM::PH + j] = (r < R1 && j < k) ? Wc[(int64_t)j * m + r] : 0.f;
                __syncthreads();
                if (act)
                    for (int rr = g; rr < nrows; rr += G)
                        fma_block(acc, *reinterpret_cast<const float4*>(&chunk[rr * SM::PH + ib * 4]),
                                  *reinterpret_cast<const float4*>(&chunk[rr * SM::PH + jb * 4]));
                __syncthreads();
            }
            group_sum<NT>(acc, act, g, blk, nblk, G, gred);
            float* slot = slots + par * SM::SLOT;
            for (int e = tid; e < KM * KM; e += NT) {
                const int a = e / KM, b = e % KM;
                slot[e] = (a < k && b < k) ? group_read(gred, G, nblk, (a >> 2) * nbk + (b >> 2), a & 3, b & 3) : 0.f;
            }
            cluster_sum<NT>(cl, C, slot, KM * KM, S, 1);
            par ^= 1;
        } else {
            __syncthreads();
            for (int e = tid; e < KM * KM; e += NT) {
                const int a = e / KM, b = e % KM;
                float sum = 0.f;
                for (int t = 0; t < l; ++t) sum = fmaf(Wt[t * KM + a], Wt[t * KM + b], sum);
                S[e] = sum;
            }
            __syncthreads();
        }
    };

    // W~ = Q^T W_init
    block_gram<NT, LQ, KM>(Q, ldq, 1, l, Wc, 1, m, k, R0, R1, chunk, chunk + 32 * (LQ + 4), gred,
                           slots + par * SM::SLOT, LQ);
    cluster_sum<NT>(cl, C, slots + par * SM::SLOT, LQ * KM, Wt, 1);
    par ^= 1;
    compute_S();

    const int nbT = nbl * nbk, nblkTV = nbT + nbk * nbk;
    const int GTV = NT / nblkTV, gTV = tid / nblkTV, blkTV = tid % nblkTV;
    const bool actTV = gTV < GTV;
    for (int it = 0; it < iters; ++it) {
        // ---- H half (Section 3.2): each thread one column of H per chunk,
        //      Gauss-Seidel over the k rows; T and V accumulate from the chunk
        float accTV[4][4] = {};
        for (int64_t cb0 = C0; cb0 < C1; cb0 += NT) {
            const int64_t c = cb0 + tid;
            float h[KM];
            if (c < C1) {
                float R[KM];
#pragma unroll
                for (int j = 0; j < KM; ++j) R[j] = 0.f;
                const float* brow = Bt + c * ldq;
#pragma unroll
                for (int t4 = 0; t4 < LQ / 4; ++t4) {
                    if (4 * t4 >= ldq) break;
                    const float4 b = *reinterpret_cast<const float4*>(brow + 4 * t4);
                    const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float* wrow = Wt + (4 * t4 + q) * KM;
#pragma unroll
                        for (int j4 = 0; j4 < KM / 4; ++j4) {
                            const float4 w = *reinterpret_cast<const float4*>(wrow + 4 * j4);
                            R[4 * j4] = fmaf(bv[q], w.x, R[4 * j4]);
                            R[4 * j4 + 1] = fmaf(bv[q], w.y, R[4 * j4 + 1]);
                            R[4 * j4 + 2] = fmaf(bv[q], w.z, R[4 * j4 + 2]);
                            R[4 * j4 + 3] = fmaf(bv[q], w.w, R[4 * j4 + 3]);
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < KM; ++j) h[j] = j < k ? Hg[(int64_t)j * n + c] : 0.f;
#pragma unroll
                for (int j = 0; j < KM; ++j) {
                    const float sjj = S[j * KM + j];
                    if (sjj > 0.f) {
                        // four independent partial sums: the Gauss-Seidel step is a
                        // dependent chain from row to row, so keep each row's chain short
                        float g0 = R[j], g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
                        for (int i = 0; i < KM; i += 4) {
                            g0 = fmaf(-S[i * KM + j], h[i], g0);
                            g1 = fmaf(-S[(i + 1) * KM + j], h[i + 1], g1);
                            g2 = fmaf(-S[(i + 2) * KM + j], h[i + 2], g2);
                            g3 = fmaf(-S[(i + 3) * KM + j], h[i + 3], g3);
                        }
                        h[j] = fmaxf(0.f, h[j] + ((g0 + g1) + (g2 + g3)) / sjj);
                    }
                }
#pragma unroll
                for (int j = 0; j < KM; ++j)
                    if (j < k) Hg[(int64_t)j * n + c] = h[j];
            } else {
#pragma unroll
                for (int j = 0; j < KM; ++j) h[j] = 0.f;
            }
#pragma unroll
            for (int j4 = 0; j4 < KM / 4; ++j4)
                *reinterpret_cast<float4*>(&chunk[tid * SM::PH + 4 * j4]) =
                    make_float4(h[4 * j4], h[4 * j4 + 1], h[4 * j4 + 2], h[4 * j4 + 3]);
            __syncthreads();
            if (actTV) {
                const int ncols = C1 - cb0 < NT ? (int)(C1 - cb0) : NT;
                if (blkTV < nbT) {
                    const int tb = blkTV / nbk, jb = blkTV % nbk;
                    for (int cc = gTV; cc < ncols; cc += GTV)
                        fma_block(accTV, *reinterpret_cast<const float4*>(Bt + (cb0 + cc) * ldq + tb * 4),
                                  *reinterpret_cast<const float4*>(&chunk[cc * SM::PH + jb * 4]));
                } else {
                    const int vb = blkTV - nbT, ib = vb / nbk, jb = vb % nbk;
                    for (int cc = gTV; cc < ncols; cc += GTV)
                        fma_block(accTV, *reinterpret_cast<const float4*>(&chunk[cc * SM::PH + ib * 4]),
                                  *reinterpret_cast<const float4*>(&chunk[cc * SM::PH + jb * 4]));
                }
            }
            __syncthreads();
        }
        group_sum<NT>(accTV, actTV, gTV, blkTV, nblkTV, GTV, gred);
        {
            float* slot = slots + par * SM::SLOT;
            for (int e = tid; e < SM::SLOT; e += NT) {
                float v = 0.f;
                if (e < LQ * KM) {
                    const int a = e / KM, b = e % KM;
                    if (a < l && b < k) v = group_read(gred, GTV, nblkTV, (a >> 2) * nbk + (b >> 2), a & 3, b & 3);
                } else {
                    const int a = (e - LQ * KM) / KM, b = (e - LQ * KM) % KM;
                    if (a < k && b < k)
                        v = group_read(gred, GTV, nblkTV, nbT + (a >> 2) * nbk + (b >> 2), a & 3, b & 3);
                }
                slot[e] = v;
            }
            cluster_sum<NT>(cl, C, slot, SM::SLOT, T, 1);
            par ^= 1;
        }
        // ---- W half: for each column j, u = (T_j - W~ V_j without j) / V_jj,
        //      W_j = max(0, Q u), W~_j = Q^T W_j (thread t < LQ owns row t of W~)
        for (int j = 0; j < k; ++j) {
            const float vjj = V[j * KM + j];
            if (!(vjj > 0.f)) continue;
            if (tid < LQ) {
                float g = T[tid * KM + j];
                for (int i = 0; i < k; ++i)
                    if (i != j) g = fmaf(-Wt[tid * KM + i], V[i * KM + j], g);
                u[tid] = g / vjj;
            }
            __syncthreads();
            float acc[LQ];
#pragma unroll
            for (int t = 0; t < LQ; ++t) acc[t] = 0.f;
            // rows r and r + NT per iteration when the registers allow: both rows'
            // loads are in flight together
            constexpr int RPI = (3 * LQ + 64) * NT < 65536 ? 2 : 1;
            for (int64_t r0 = R0 + tid; r0 < R1; r0 += RPI * NT) {
                float q[RPI][LQ];
#pragma unroll
                for (int h2 = 0; h2 < RPI; ++h2) {
                    const int64_t r = r0 + h2 * NT;
                    const float* qrow = Q + r * ldq;
#pragma unroll
                    for (int t4 = 0; t4 < LQ / 4; ++t4) {
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (r < R1 && 4 * t4 < ldq) v = *reinterpret_cast<const float4*>(qrow + 4 * t4);
                        q[h2][4 * t4] = v.x;
                        q[h2][4 * t4 + 1] = v.y;
                        q[h2][4 * t4 + 2] = v.z;
                        q[h2][4 * t4 + 3] = v.w;
                    }
                }
#pragma unroll
                for (int h2 = 0; h2 < RPI; ++h2) {
                    const int64_t r = r0 + h2 * NT;
                    float z = 0.f;
#pragma unroll
                    for (int t4 = 0; t4 < LQ / 4; ++t4) {
                        const float4 uu = *reinterpret_cast<const float4*>(u + 4 * t4);
                        z = fmaf(q[h2][4 * t4], uu.x, z);
                        z = fmaf(q[h2][4 * t4 + 1], uu.y, z);
                        z = fmaf(q[h2][4 * t4 + 2], uu.z, z);
                        z = fmaf(q[h2][4 * t4 + 3], uu.w, z);
                    }
                    const float w = fmaxf(0.f, z);
                    if (r < R1) Wc[(int64_t)j * m + r] = w;
#pragma unroll
                    for (int t = 0; t < LQ; ++t) acc[t] = fmaf(q[h2][t], w, acc[t]);
                }
            }
            warp_reduce_scatter<LQ>(acc, lane);
            if (LQ >= 32 || (lane & 1) == 0)
#pragma unroll
                for (int i = 0; i < rs_count<LQ>(); ++i) red[warp * LQ + rs_index<LQ>(lane, i)] = acc[i];
            __syncthreads();
            if (C == 1) {
                if (tid < LQ) {
                    float sum = 0.f;
                    for (int w2 = 0; w2 < NT / 32; ++w2) sum += red[w2 * LQ + tid];
                    Wt[tid * KM + j] = sum;
                }
            } else {
                float* slot = slots + par * SM::SLOT;
                if (tid < LQ) {
                    float sum = 0.f;
                    for (int w2 = 0; w2 < NT / 32; ++w2) sum += red[w2 * LQ + tid];
                    slot[tid] = sum;
                }
                cl.sync();
                if (tid < LQ) {
                    float sum = 0.f;
                    for (int r = 0; r < C; ++r) sum += cl.map_shared_rank(slot, r)[tid];
                    Wt[tid * KM + j] = sum;
                }
                par ^= 1;
            }
        }
        compute_S();
    }
    __syncthreads();
    // W = (W^T)^T for this CTA's rows
    for (int64_t r = R0 + tid; r < R1; r += NT)
        for (int j = 0; j < k; ++j) d.W[r * k + j] = Wc[(int64_t)j * m + r];
    // no CTA leaves while another may still read its shared memory
    if (C > 1) cl.sync();
}

template <int NT, int LQ, int KM>
bool launch_sweeps_t(cudaStream_t s, RbInst* I, const int* list, int count, int csize, int iters_override) {
    const size_t smem = (size_t)SweepSmem<NT, LQ, KM>::floats * sizeof(float);
    if (cudaFuncSetAttribute(rb_sweeps_kernel<NT, LQ, KM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(count * csize));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, rb_sweeps_kernel<NT, LQ, KM>, I, list, count, iters_override) == cudaSuccess;
}

}  // namespace

int rb_tile_rows(int l) {
    const int ncb = (l + 3) / 4;
    int nrb = TNT / ncb;
    if (nrb > RB_BMAX / 4) nrb = RB_BMAX / 4;
    return 4 * nrb;
}

int rb_lq(int l) { return l <= 16 ? 16 : l <= 32 ? 32 : 64; }

int rb_km(int k) { return k <= 16 ? 16 : 32; }

bool rb_launch_omega(cudaStream_t s, RbInst* I, int count) {
    if (count <= 0) return true;
    rb_omega_kernel<<<dim3(16, (unsigned)count), 256, 0, s>>>(I, count);
    return cudaGetLastError() == cudaSuccess;
}

bool rb_launch_init(cudaStream_t s, RbInst* I, int count) {
    if (count <= 0) return true;
    rb_init_kernel<<<dim3(16, (unsigned)count), 256, 0, s>>>(I, count);
    return cudaGetLastError() == cudaSuccess;
}

bool rb_launch_rows(cudaStream_t s, int grid, RbInst* I, const RbTile* tiles, int ntiles, int* counter, int mode,
                    int only_shifted, int gate) {
    if (ntiles <= 0) return true;
    if (mode == 0) {
        const size_t smem = 2 * SK_STAGE * sizeof(float);
        if (cudaFuncSetAttribute(rb_sketch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return false;
        rb_sketch_kernel<<<grid, TNT, smem, s>>>(I, tiles, ntiles, counter, gate);
    } else {
        rb_rows_kernel<<<grid, TNT, 0, s>>>(I, tiles, ntiles, counter, mode, only_shifted, gate);
    }
    return cudaGetLastError() == cudaSuccess;
}

bool rb_launch_atx(cudaStream_t s, int grid, RbInst* I, const RbTile* tiles, int ntiles, int* counter, int gate) {
    if (ntiles <= 0) return true;
    const size_t smem = 2 * AT_STAGE * sizeof(float);
    if (cudaFuncSetAttribute(rb_atx_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return false;
    rb_atx_kernel<<<grid, TNT, smem, s>>>(I, tiles, ntiles, counter, gate);
    return cudaGetLastError() == cudaSuccess;
}

bool rb_launch_gram(cudaStream_t s, int grid, RbInst* I, const RbTile* tiles, int ntiles, int* counter, int which,
                    int only_shifted, int gate) {
    if (ntiles <= 0) return true;
    rb_gram_kernel<<<grid, TNT, 0, s>>>(I, tiles, ntiles, counter, which, only_shifted, gate);
    return cudaGetLastError() == cudaSuccess;
}

bool rb_launch_chol(cudaStream_t s, RbInst* I, int count, int which, int pass, int gate) {
    if (count <= 0) return true;
    rb_chol_kernel<<<count, CNT, 0, s>>>(I, count, which, pass, gate);
    return cudaGetLastError() == cudaSuccess;
}

bool rb_launch_sweeps(cudaStream_t s, RbInst* I, const int* list, int count, int csize, int lq, int km, int nt,
                      int iters_override) {
    if (count <= 0) return true;
    if (lq == 64) return launch_sweeps_t<256, 64, 32>(s, I, list, count, csize, iters_override);
    if (nt == 512) {
        if (lq == 16) return launch_sweeps_t<512, 16, 16>(s, I, list, count, csize, iters_override);
        if (km == 16) return launch_sweeps_t<512, 32, 16>(s, I, list, count, csize, iters_override);
        return launch_sweeps_t<512, 32, 32>(s, I, list, count, csize, iters_override);
    }
    if (lq == 16) return launch_sweeps_t<256, 16, 16>(s, I, list, count, csize, iters_override);
    if (km == 16) return launch_sweeps_t<256, 32, 16>(s, I, list, count, csize, iters_override);
    return launch_sweeps_t<256, 32, 32>(s, I, list, count, csize, iters_override);
}
