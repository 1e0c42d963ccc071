// gram.cu - G = X^T X (c x c, c <= 128).
//
// Used for the Gram matrix of CholeskyQR (the orthonormalisation qr() of
// Section 2.3 / Algorithm 1), and for S = W^T W and V = H H^T of a sweep
// (Algorithm 1 loop body).  Two arithmetic forms, both on CUDA cores in float32
// (float64 throughput is low on this GPU):
//   exact = true : every product x_i x_j is split exactly into p + e
//                  (p = x_i x_j, e = fma(x_i, x_j, -p)) and accumulated as a
//                  float32 pair (hi, lo) with TwoSum - a float64-class Gram for
//                  the ill-conditioned sketch Y of CholeskyQR;
//   exact = false: float32 products summed over 32-row stages, stage sums
//                  folded into a (sum, compensation) pair with TwoSum.
// Each thread owns 4 x 4 blocks of the upper triangle; rows are split over
// blocks of the grid and the block partials, (sum, compensation) pairs, are
// added as two-sum pairs in a fixed order (pair_sum.cuh; float64 arithmetic is
// slow on this GPU).
#include "async_copy.cuh"
#include "f32x2.cuh"
#include "pair_sum.cuh"
#include "rnmf_internal.cuh"

namespace {

constexpr int NT = 256;
constexpr int RB = 32;  // rows per shared-memory stage

__device__ __forceinline__ void two_sum(float& s, float& c, float v) {
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    c += __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    s = t;
}

template <int CP, bool EXACT>
__global__ void __launch_bounds__(NT) gram_partial_kernel(const float* __restrict__ X, int64_t s_r, int64_t s_c,
                                                          int64_t N, int c, int64_t rchunk,
                                                          float2* __restrict__ partial,
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
    // stage loader: element e of a RB x CP tile (row-fast when X rows are strided)
    constexpr int EPT = RB * CP / NT;   // elements per thread per stage
    auto stage_elem = [&](int e, int& rr, int& j) {
        if (s_c == 1) {
            rr = e / CP;
            j = e % CP;
        } else {
            j = e / RB;
            rr = e % RB;
        }
    };
    float nxt[EPT];
    auto fetch = [&](int64_t r0) {
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            int rr, j;
            stage_elem(threadIdx.x + q * NT, rr, j);
            const int64_t r = r0 + rr;
            nxt[q] = (j < c && r < rend) ? X[r * s_r + (int64_t)j * s_c] : 0.f;
        }
    };
    if (rbeg < rend) fetch(rbeg);
    for (int64_t r0 = rbeg; r0 < rend; r0 += RB) {
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            int rr, j;
            stage_elem(threadIdx.x + q * NT, rr, j);
            Xs[rr][j] = nxt[q];
        }
        __syncthreads();
        if (r0 + RB < rend) fetch(r0 + RB);
#pragma unroll
        for (int q = 0; q < BPT; ++q) {
            if (threadIdx.x + q * NT >= NBLK) continue;
            if (EXACT) {
                // two entries (y, y + 1) per packed operation: the same IEEE operations
                // in the same order as one entry at a time (p = a b, e = fma(a, b, -p),
                // TwoSum of p into (hi, lo), then lo += e), so the sums are bit-identical
                const float2 neg1 = make_float2(-1.f, -1.f);
                for (int rr = 0; rr < RB; ++rr) {
                    const float4 a = *reinterpret_cast<const float4*>(&Xs[rr][4 * bi[q]]);
                    const float4 b = *reinterpret_cast<const float4*>(&Xs[rr][4 * bj[q]]);
                    const float av[4] = {a.x, a.y, a.z, a.w};
                    const float2 b2[2] = {lo2(b), hi2(b)};
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        const float2 a2 = make_float2(av[x], av[x]);
#pragma unroll
                        for (int y2 = 0; y2 < 2; ++y2) {
                            const int e0 = 4 * x + 2 * y2;
                            const float2 h = make_float2(hi[q][e0], hi[q][e0 + 1]);
                            float2 lw = make_float2(lo[q][e0], lo[q][e0 + 1]);
                            const float2 p = f2_mul(a2, b2[y2]);
                            const float2 e = f2_fma(a2, b2[y2], f2_mul(p, neg1));
                            const float2 t = f2_add(h, p);
                            const float2 bp = f2_sub(t, h);
                            lw = f2_add(lw, f2_add(f2_sub(h, f2_sub(t, bp)), f2_sub(p, bp)));
                            lw = f2_add(lw, e);
                            hi[q][e0] = t.x;
                            hi[q][e0 + 1] = t.y;
                            lo[q][e0] = lw.x;
                            lo[q][e0 + 1] = lw.y;
                        }
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
            partial[((int64_t)blockIdx.x * NBLK + b) * 16 + e] = make_float2(hi[q][e], lo[q][e]);
    }
}

// Column-major input (s_r == 1: X(r, j) = X[j * s_c + r], e.g. X = W stored as
// W^T, or X = H^T): the 32-row stage is kept transposed, XsT[j][r], so the
// fills are contiguous; 16-byte chunks of each XsT row are XOR-swizzled with
// (j / 4) mod 8 so that the float4 reads of 32 different 4 x 4 blocks spread
// over all banks.  Thread work and accumulation as in gram_partial_kernel.
template <int CP, bool EXACT>
__global__ void __launch_bounds__(NT) gram_partial_cm_kernel(const float* __restrict__ X, int64_t s_c, int64_t N,
                                                             int c, int64_t rchunk, float2* __restrict__ partial,
                                                             const int* __restrict__ skip_if_zero) {
    if (skip_if_zero && *skip_if_zero == 0) return;
    constexpr int NB = CP / 4;
    constexpr int NBLK = NB * (NB + 1) / 2;
    constexpr int BPT = (NBLK + NT - 1) / NT;
    constexpr int EPT = RB * CP / NT;
    __shared__ __align__(16) float XsT[CP][RB];
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
    auto swz = [](int j, int rr) { return (((rr >> 2) ^ ((j >> 2) & 7)) << 2) | (rr & 3); };
    float nxt[EPT];
    auto fetch = [&](int64_t r0) {
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int e = threadIdx.x + q * NT;
            const int j = e / RB, rr = e % RB;
            const int64_t r = r0 + rr;
            nxt[q] = (j < c && r < rend) ? X[(int64_t)j * s_c + r] : 0.f;
        }
    };
    if (rbeg < rend) fetch(rbeg);
    for (int64_t r0 = rbeg; r0 < rend; r0 += RB) {
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int e = threadIdx.x + q * NT;
            const int j = e / RB, rr = e % RB;
            XsT[j][swz(j, rr)] = nxt[q];
        }
        __syncthreads();
        if (r0 + RB < rend) fetch(r0 + RB);
#pragma unroll
        for (int q = 0; q < BPT; ++q) {
            if (threadIdx.x + q * NT >= NBLK) continue;
            float st[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) st[e] = 0.f;
            for (int rr = 0; rr < RB; rr += 4) {
                float a[4][4], b[4][4];  // [x][t]: rows 4bi + x (4bj + y), stage rows rr + t
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    const int ja = 4 * bi[q] + x, jb = 4 * bj[q] + x;
                    const float4 va = *reinterpret_cast<const float4*>(&XsT[ja][swz(ja, rr)]);
                    const float4 vb = *reinterpret_cast<const float4*>(&XsT[jb][swz(jb, rr)]);
                    a[x][0] = va.x; a[x][1] = va.y; a[x][2] = va.z; a[x][3] = va.w;
                    b[x][0] = vb.x; b[x][1] = vb.y; b[x][2] = vb.z; b[x][3] = vb.w;
                }
#pragma unroll
                for (int t = 0; t < 4; ++t)
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) {
                            if (EXACT) {
                                const float pr = __fmul_rn(a[x][t], b[y][t]);
                                const float er = fmaf(a[x][t], b[y][t], -pr);
                                two_sum(hi[q][4 * x + y], lo[q][4 * x + y], pr);
                                lo[q][4 * x + y] += er;
                            } else {
                                st[4 * x + y] = fmaf(a[x][t], b[y][t], st[4 * x + y]);
                            }
                        }
            }
            if (!EXACT) {
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
            partial[((int64_t)blockIdx.x * NBLK + b) * 16 + e] = make_float2(hi[q][e], lo[q][e]);
    }
}

// Sum the block partials and scatter the upper-triangle entries of the 4 x 4
// blocks into the symmetric G (double), G32 (float) and Gp (float pairs
// hi + lo, |lo| <= ulp(hi) / 2); each output is optional.  A block handles 32
// consecutive partial entries with 8 groups of threads (group pg adds the
// (sum, compensation) pairs of blocks b = pg (mod 8) as a two-sum pair); the
// group sums are added in group order (fixed order).
template <int CP>
__global__ void __launch_bounds__(256) gram_reduce_kernel(const float2* __restrict__ partial, int nblk, int c,
                                                          double* __restrict__ G, float* __restrict__ G32,
                                                          float2* __restrict__ Gp,
                                                          const int* __restrict__ skip_if_zero) {
    if (skip_if_zero && *skip_if_zero == 0) return;
    constexpr int NB = CP / 4;
    constexpr int NBLK = NB * (NB + 1) / 2;
    __shared__ float2 red[8][32];
    const int el = threadIdx.x & 31, pg = threadIdx.x >> 5;
    const int t = blockIdx.x * 32 + el;
    float2 a = make_float2(0.f, 0.f);
    if (t < NBLK * 16) {
        for (int b0 = pg; b0 < nblk; b0 += 8 * 8) {
            float2 v[8];  // eight loads in flight; past the end adds (+0, +0)
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[u] = b0 + 8 * u < nblk ? partial[(int64_t)(b0 + 8 * u) * NBLK * 16 + t] : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) a = pair_add(a, v[u]);
        }
    }
    red[pg][el] = a;
    __syncthreads();
    if (pg != 0 || t >= NBLK * 16) return;
    int blk = t / 16, i = 0;
    const int e = t % 16;
    while (blk >= NB - i) {
        blk -= NB - i;
        ++i;
    }
    const int gi = 4 * i + e / 4, gj = 4 * (i + blk) + e % 4;
    if (gi >= c || gj >= c || gi > gj) return;  // lower entries of diagonal blocks: mirrored from above
    float2 s = red[0][el];
#pragma unroll
    for (int q = 1; q < 8; ++q) s = pair_add(s, red[q][el]);
    if (G) {
        const double sd = (double)s.x + (double)s.y;
        G[gi * c + gj] = sd;
        G[gj * c + gi] = sd;
    }
    if (G32) {
        G32[gi * c + gj] = pair_value(s);
        G32[gj * c + gi] = pair_value(s);
    }
    if (Gp) {
        const float h = __fadd_rn(s.x, s.y);
        const float2 pn = make_float2(h, __fsub_rn(s.y, __fsub_rn(h, s.x)));  // normalised: |lo| <= ulp(hi) / 2
        Gp[gi * c + gj] = pn;
        Gp[gj * c + gi] = pn;
    }
}

// Non-exact Gram of a column-major X (X(r, j) = X[j s_c + r]) on 8 x 8 output
// tiles - the sweep's S = W^T W and V = H H^T.  Thread (tile, grp) owns one
// 8 x 8 tile of the upper triangle of the CP x CP output and the 4-row chunks
// ch = grp (mod G) of every 32-row stage; a chunk costs 16 float4 reads (8
// rows of the tile's row block, 8 of its column block) for 256 FMAs, twice the
// work per read of 4 x 4 tiles.  Stages are double-buffered with cp.async and
// kept transposed, XsT[j][r], with 16-byte chunks XOR-swizzled by (j / 8) mod 8
// so that threads reading different tiles hit different banks.  A thread sums
// its rows of the block (a few hundred at most: two blocks per SM) in float32;
// the G row groups are added in group order in shared memory; one float32
// partial per block, laid out [entry][tile] for coalesced stores.
template <int CP>
struct Gram8 {
    static constexpr int T8 = CP / 8;
    static constexpr int NTILE = T8 * (T8 + 1) / 2;
    static constexpr int G0 = NT / NTILE;
    static constexpr int G = G0 > 8 ? 8 : G0;
    static constexpr int E = NTILE * 64;
};

__device__ __forceinline__ void tile_of(int tile, int t8, int& ti, int& tj) {
    int i = 0, b = tile;
    while (b >= t8 - i) {
        b -= t8 - i;
        ++i;
    }
    ti = i;
    tj = i + b;
}

template <int CP>
__global__ void __launch_bounds__(NT, 2) gram8_cm_kernel(const float* __restrict__ X, int64_t s_c, int64_t N, int c,
                                                        int64_t rchunk, float* __restrict__ partial,
                                                        const int* __restrict__ skip_if_zero, int vec) {
    if (skip_if_zero && *skip_if_zero == 0) return;
    using P = Gram8<CP>;
    static_assert(P::G >= 1, "an 8 x 8 tile per thread");
    static_assert(P::G == 1 || P::NTILE * 64 <= 2 * CP * RB, "the group sums fit the stage buffers");
    __shared__ __align__(16) float XsT[2][CP][RB];
    const int tid = threadIdx.x;
    const int tile = tid % P::NTILE, grp = tid / P::NTILE;
    const bool active = grp < P::G;
    int ti, tj;
    tile_of(tile, P::T8, ti, tj);
    const int64_t rbeg = (int64_t)blockIdx.x * rchunk;
    const int64_t rend = rbeg + rchunk < N ? rbeg + rchunk : N;
    auto load_stage = [&](int buf, int64_t r0) {
        if (vec) {
            for (int e = tid; e < CP * (RB / 4); e += NT) {
                const int j = e / (RB / 4), q = e % (RB / 4);
                const int64_t r = r0 + 4 * q;
                const int bytes = (j < c && r < rend) ? (rend - r >= 4 ? 16 : (int)(rend - r) * 4) : 0;
                cp_async16_n(&XsT[buf][j][(q ^ ((j >> 3) & 7)) * 4], bytes ? X + (int64_t)j * s_c + r : X, bytes);
            }
        } else {
            for (int e = tid; e < CP * RB; e += NT) {
                const int j = e / RB, rr = e % RB;
                const int64_t r = r0 + rr;
                const bool ok = j < c && r < rend;
                cp_async4(&XsT[buf][j][(((rr >> 2) ^ ((j >> 3) & 7)) << 2) | (rr & 3)],
                          ok ? X + (int64_t)j * s_c + r : X, ok);
            }
        }
        cp_async_commit();
    };
    float hi[8][8];
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
            for (int ch = grp; ch < RB / 4; ch += P::G) {
                float4 bb[8];
#pragma unroll
                for (int y = 0; y < 8; ++y)
                    bb[y] = *reinterpret_cast<const float4*>(&XsT[buf][8 * tj + y][(ch ^ (tj & 7)) * 4]);
                // one operand row at a time keeps the live registers to 64 sums + 36
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    const float4 a = *reinterpret_cast<const float4*>(&XsT[buf][8 * ti + x][(ch ^ (ti & 7)) * 4]);
#pragma unroll
                    for (int y = 0; y < 8; ++y) hi[x][y] = fmaf(a.x, bb[y].x, hi[x][y]);
#pragma unroll
                    for (int y = 0; y < 8; ++y) hi[x][y] = fmaf(a.y, bb[y].y, hi[x][y]);
#pragma unroll
                    for (int y = 0; y < 8; ++y) hi[x][y] = fmaf(a.z, bb[y].z, hi[x][y]);
#pragma unroll
                    for (int y = 0; y < 8; ++y) hi[x][y] = fmaf(a.w, bb[y].w, hi[x][y]);
                }
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    if (P::G > 1) {
        float* red = &XsT[0][0][0];  // [64][NTILE]
        for (int g = 1; g < P::G; ++g) {
            if (grp == g)
#pragma unroll
                for (int e = 0; e < 64; ++e) red[e * P::NTILE + tile] = hi[e / 8][e % 8];
            __syncthreads();
            if (grp == 0)
#pragma unroll
                for (int e = 0; e < 64; ++e) hi[e / 8][e % 8] += red[e * P::NTILE + tile];
            __syncthreads();
        }
    }
    if (grp == 0)
#pragma unroll
        for (int e = 0; e < 64; ++e)
            partial[((int64_t)blockIdx.x * 64 + e) * P::NTILE + tile] = hi[e / 8][e % 8];
}

// Sum of the gram8 block partials in a fixed order (group pg adds blocks
// pg, pg + 8, ... as a two-sum pair, the eight groups are added in order) and
// scatter of the upper-triangle entries into the symmetric G and G32.
template <int CP>
__global__ void __launch_bounds__(256) gram8_reduce_kernel(const float* __restrict__ partial, int nblk, int c,
                                                           double* __restrict__ G, float* __restrict__ G32,
                                                           const int* __restrict__ skip_if_zero) {
    if (skip_if_zero && *skip_if_zero == 0) return;
    using P = Gram8<CP>;
    __shared__ float2 red[8][32];
    const int el = threadIdx.x & 31, pg = threadIdx.x >> 5;
    const int t = blockIdx.x * 32 + el;
    float2 a = make_float2(0.f, 0.f);
    if (t < P::E) {
        for (int b0 = pg; b0 < nblk; b0 += 8 * 16) {
            float v[16];  // sixteen loads in flight; past the end adds +0
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = b0 + 8 * u < nblk ? partial[(int64_t)(b0 + 8 * u) * P::E + t] : 0.f;
#pragma unroll
            for (int u = 0; u < 16; ++u) two_sum_add(a, v[u]);
        }
    }
    red[pg][el] = a;
    __syncthreads();
    if (pg != 0 || t >= P::E) return;
    const int e = t / P::NTILE, tile = t % P::NTILE;
    int ti, tj;
    tile_of(tile, P::T8, ti, tj);
    const int gi = 8 * ti + e / 8, gj = 8 * tj + e % 8;
    if (gi >= c || gj >= c || gi > gj) return;  // lower entries of diagonal tiles: mirrored from above
    float2 s = red[0][el];
#pragma unroll
    for (int q = 1; q < 8; ++q) s = pair_add(s, red[q][el]);
    const double sd = (double)s.x + (double)s.y;
    G[gi * c + gj] = sd;
    G[gj * c + gi] = sd;
    if (G32) {
        G32[gi * c + gj] = pair_value(s);
        G32[gj * c + gi] = pair_value(s);
    }
}

// Padded width: the smallest instantiated multiple of 8 that holds c (the
// thread blocks cover the upper triangle of CP / 4 x CP / 4 blocks, so a tight
// CP avoids up to (128 / c)^2 wasted work for c just above a power of two).
int cpad(int c) {
    const int opts[] = {16, 32, 48, 64, 80, 96, 104, 112, 120, 128};
    for (int v : opts)
        if (c <= v) return v;
    return 128;
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

// Two gram8 blocks per SM.
void gram8_split(rnmf_ctx* ctx, int64_t N, int* nblk, int64_t* rchunk) {
    int64_t target = (int64_t)ctx->num_sms * 2;
    int64_t rc = (N + target - 1) / target;
    rc = (rc + RB - 1) / RB * RB;
    if (rc < RB) rc = RB;
    int64_t nb = (N + rc - 1) / rc;
    *nblk = (int)(nb < 1 ? 1 : nb);
    *rchunk = rc;
}

template <int CP>
bool gram_launch(rnmf_ctx* ctx, const float* X, int64_t s_r, int64_t s_c, int64_t N, int c, double* G, float* G32,
                 double* scratch, const int* skip, bool exact, float2* Gp) {
    int nb;
    int64_t rc;
    if (s_r == 1 && s_c != 1 && !exact) {
        if (Gp) return false;  // the 8 x 8-tile form writes G and G32 only
        gram8_split(ctx, N, &nb, &rc);
        const int vec = (s_c % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
        prof_begin(ctx);
        float* part8 = reinterpret_cast<float*>(scratch);  // [block][entry] float32 partials
        gram8_cm_kernel<CP><<<nb, NT, 0, ctx->stream>>>(X, s_c, N, c, rc, part8, skip, vec);
        if (!launch_done(ctx, K_GRAM, 4.0 * N * c, (double)N * c * (c + 1))) return false;
        prof_begin(ctx);
        gram8_reduce_kernel<CP><<<(Gram8<CP>::E + 31) / 32, 256, 0, ctx->stream>>>(part8, nb, c, G, G32, skip);
        return launch_done(ctx, K_GRAM, 8.0 * nb * Gram8<CP>::E + 12.0 * c * c, (double)nb * Gram8<CP>::E);
    }
    gram_split(ctx, N, &nb, &rc);
    float2* part = reinterpret_cast<float2*>(scratch);  // [block][entry] (sum, compensation) pairs
    prof_begin(ctx);
    if (s_r == 1 && s_c != 1) {
        if (exact)
            gram_partial_cm_kernel<CP, true><<<nb, NT, 0, ctx->stream>>>(X, s_c, N, c, rc, part, skip);
        else
            gram_partial_cm_kernel<CP, false><<<nb, NT, 0, ctx->stream>>>(X, s_c, N, c, rc, part, skip);
    } else if (exact) {
        gram_partial_kernel<CP, true><<<nb, NT, 0, ctx->stream>>>(X, s_r, s_c, N, c, rc, part, skip);
    } else {
        gram_partial_kernel<CP, false><<<nb, NT, 0, ctx->stream>>>(X, s_r, s_c, N, c, rc, part, skip);
    }
    if (!launch_done(ctx, K_GRAM, 4.0 * N * c, (double)N * c * (c + 1))) return false;
    constexpr int NBLK = (CP / 4) * (CP / 4 + 1) / 2;
    prof_begin(ctx);
    gram_reduce_kernel<CP><<<(NBLK * 16 + 31) / 32, 256, 0, ctx->stream>>>(part, nb, c, G, G32, Gp, skip);
    return launch_done(ctx, K_GRAM, 8.0 * nb * NBLK * 16 + 12.0 * c * c, (double)nb * NBLK * 16);
}

}  // namespace

size_t gram_scratch_bytes(rnmf_ctx* ctx, int64_t N, int c) {
    int nb, nb8;
    int64_t rc;
    gram_split(ctx, N, &nb, &rc);
    gram8_split(ctx, N, &nb8, &rc);
    const int nbk = cpad(c) / 4, t8 = cpad(c) / 8;
    const size_t a = (size_t)nb * (nbk * (nbk + 1) / 2) * 16 * sizeof(double);
    const size_t b = (size_t)nb8 * (t8 * (t8 + 1) / 2) * 64 * sizeof(float);
    return a > b ? a : b;
}

bool launch_gram(rnmf_ctx* ctx, const float* X, int64_t s_r, int64_t s_c, int64_t N, int c, double* G, float* G32,
                 double* scratch, const int* skip_if_zero, bool exact, float2* Gp) {
    switch (cpad(c)) {
        case 16: return gram_launch<16>(ctx, X, s_r, s_c, N, c, G, G32, scratch, skip_if_zero, exact, Gp);
        case 32: return gram_launch<32>(ctx, X, s_r, s_c, N, c, G, G32, scratch, skip_if_zero, exact, Gp);
        case 48: return gram_launch<48>(ctx, X, s_r, s_c, N, c, G, G32, scratch, skip_if_zero, exact, Gp);
        case 64: return gram_launch<64>(ctx, X, s_r, s_c, N, c, G, G32, scratch, skip_if_zero, exact, Gp);
        case 80: return gram_launch<80>(ctx, X, s_r, s_c, N, c, G, G32, scratch, skip_if_zero, exact, Gp);
        case 96: return gram_launch<96>(ctx, X, s_r, s_c, N, c, G, G32, scratch, skip_if_zero, exact, Gp);
        case 104: return gram_launch<104>(ctx, X, s_r, s_c, N, c, G, G32, scratch, skip_if_zero, exact, Gp);
        case 112: return gram_launch<112>(ctx, X, s_r, s_c, N, c, G, G32, scratch, skip_if_zero, exact, Gp);
        case 120: return gram_launch<120>(ctx, X, s_r, s_c, N, c, G, G32, scratch, skip_if_zero, exact, Gp);
        default: return gram_launch<128>(ctx, X, s_r, s_c, N, c, G, G32, scratch, skip_if_zero, exact, Gp);
    }
}
