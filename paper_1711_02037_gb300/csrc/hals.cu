// hals.cu - the HALS block updates of a sweep.
//
// (1) hals_rows: the Gauss-Seidel row recurrence shared by
//       - the H rows of randomized HALS (Section 3.2 H rule; Algorithm 1):
//         x = H(:, c), rhs = R(c, :) with R = B^T W~, Gram S = W^T W;
//       - the H rows of deterministic HALS (Section 3.1): rhs = (A^T W)(c, :);
//       - the W columns of deterministic HALS: x = W(r, :), rhs = (A H^T)(r, :),
//         Gram V = H H^T.
//     For j = 1..k: x_j <- max(0, x_j + (rhs_j - sum_i x_i S_ij) / S_jj), with
//     x_i already updated for i < j.  Every vector is independent (one thread
//     each).  The j loop runs in chunks of 8: the sums over all entries are
//     formed first (one shared-memory read of x_i feeds 8 FMAs, issued as 4
//     packed f32x2 FMAs), then the 8 sequential steps run in registers.  One block per SM, sized so that a
//     single round covers every vector where shared memory allows, shares one
//     copy of S.
//
// (2) whalf: the W half of a randomized sweep (Section 3.2 W~ rule and
//     reprojection; Algorithm 1), Gauss-Seidel over columns j:
//       u   = W~_j + (T_:j - W~ V_:j) / V_jj      (l-vector, every block)
//       W_j = max(0, Q u)                         (row-local)
//       W~_j = Q^T W_j                            (sum over all m rows)
//     One persistent block per SM owns a slice of rows; the sum over rows is an
//     exact fixed-point (integer) sum of the per-block partials.  Each block
//     adds its term and a count into 64-bit words with one atomic, and polls
//     the words until every block's term has landed.  There is no grid
//     barrier; the poll is bounded (RNMF_ETIMEOUT instead of a hang).
#include "async_copy.cuh"
#include "f32x2.cuh"
#include "rnmf_internal.cuh"
#include "sync.cuh"

namespace {

constexpr int ROWS_NT_MAX = 512;         // threads per block at most (one block per SM holds a round)
constexpr int CH = 8;
// one thread per vector; xs row pitch vpb + 4

// Regularised rule (Section 3.4, reg != 0): x_j <- max(0, (S_jj x_j + g - beta) / (S_jj + alpha)),
// with g = Rhs_j - sum_i S_ij x_i; reg == 0 keeps the plain rule x_j + g / S_jj.
// Chunk j0..j0+7: g_j = Rhs_j - sum_i x_i S_ij over all i with the current x
// (entries before the chunk already updated, the chunk and later ones not),
// then the chunk's 8 steps in registers, each step's change x_j' - x_j folded
// into the remaining g of the chunk - so every step sees the entries updated
// before it, as the Gauss-Seidel order requires.
__global__ void __launch_bounds__(ROWS_NT_MAX, 1) hals_rows_kernel(float* __restrict__ X, int64_t sv, int64_t se,
                                                            const float* __restrict__ Rhs, int64_t srv,
                                                            int64_t srj, const float* __restrict__ S,
                                                            int64_t count, int k, int reg, float alpha,
                                                            float beta) {
    extern __shared__ __align__(16) float sm[];
    const int kp = (k + CH - 1) / CH * CH;
    float* Ss = sm;                 // kp x kp, zero padded
    const int nt = blockDim.x, vpb = nt, xsp = vpb + 4;
    float* xs = sm + kp * kp;       // kp x xsp: x_i of vector vl at xs[i*xsp + vl]
    float* sinv = xs + kp * xsp;    // kp: 1 / S_jj (1 / (S_jj + alpha) with penalties), 0 where S_jj <= 0
    const int t = threadIdx.x;
    const int vl = t;
    for (int e = t; e < kp * kp; e += nt) {
        int i = e / kp, j = e % kp;
        Ss[e] = (i < k && j < k) ? S[i * k + j] : 0.f;
    }
    for (int j = t; j < kp; j += nt) {
        const float sjj = j < k ? S[j * k + j] : 0.f;
        sinv[j] = sjj > 0.f ? 1.f / (reg ? sjj + alpha : sjj) : 0.f;
    }
    __syncthreads();
    // persistent over groups of vpb vectors (each thread owns one vector at a time
    // and its column xs[.][vl]: no barrier inside the loop)
    const int64_t ngroups = (count + vpb - 1) / vpb;
    for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int64_t v = grp * vpb + vl;
        if (v >= count) continue;
        for (int i = 0; i < kp; ++i) {
            const bool ok = i < k;
            cp_async4(&xs[i * xsp + vl], ok ? X + v * sv + (int64_t)i * se : X, ok);
        }
        cp_async_wait_all();
        float gn[CH];
#pragma unroll
        for (int jj = 0; jj < CH; ++jj) gn[jj] = jj < k ? Rhs[v * srv + (int64_t)jj * srj] : 0.f;
        for (int j0 = 0; j0 < k; j0 += CH) {
            // g, h as packed pairs (g[2 q], g[2 q + 1]) = g2[q]
            float2 g2[CH / 2], h2[CH / 2];
#pragma unroll
            for (int q = 0; q < CH / 2; ++q) {
                g2[q] = make_float2(gn[2 * q], gn[2 * q + 1]);
                h2[q] = make_float2(0.f, 0.f);
            }
            // right-hand side of the next chunk, in flight while this chunk is processed
            if (j0 + CH < k) {
#pragma unroll
                for (int jj = 0; jj < CH; ++jj)
                    gn[jj] = (j0 + CH + jj < k) ? Rhs[v * srv + (int64_t)(j0 + CH + jj) * srj] : 0.f;
            }
            // entries before the chunk (already updated) on one accumulator set, the chunk
            // and those after it (not yet updated) on another
#pragma unroll 4
            for (int i = 0; i < j0; ++i) {
                const float nxi = -xs[i * xsp + vl];
                const float2 nx = make_float2(nxi, nxi);
                const float4 s0 = *reinterpret_cast<const float4*>(&Ss[i * kp + j0]);
                const float4 s1 = *reinterpret_cast<const float4*>(&Ss[i * kp + j0 + 4]);
                g2[0] = f2_fma(nx, lo2(s0), g2[0]);
                g2[1] = f2_fma(nx, hi2(s0), g2[1]);
                g2[2] = f2_fma(nx, lo2(s1), g2[2]);
                g2[3] = f2_fma(nx, hi2(s1), g2[3]);
            }
#pragma unroll 4
            for (int i = j0; i < kp; ++i) {
                const float nxi = -xs[i * xsp + vl];
                const float2 nx = make_float2(nxi, nxi);
                const float4 s0 = *reinterpret_cast<const float4*>(&Ss[i * kp + j0]);
                const float4 s1 = *reinterpret_cast<const float4*>(&Ss[i * kp + j0 + 4]);
                h2[0] = f2_fma(nx, lo2(s0), h2[0]);
                h2[1] = f2_fma(nx, hi2(s0), h2[1]);
                h2[2] = f2_fma(nx, lo2(s1), h2[2]);
                h2[3] = f2_fma(nx, hi2(s1), h2[3]);
            }
            float g[CH], xc[CH];
#pragma unroll
            for (int q = 0; q < CH / 2; ++q) {
                const float2 t = f2_add(g2[q], h2[q]);
                g[2 * q] = t.x;
                g[2 * q + 1] = t.y;
            }
#pragma unroll
            for (int jj = 0; jj < CH; ++jj) xc[jj] = xs[(j0 + jj) * xsp + vl];
            // the chunk's own recurrence, in registers
#pragma unroll
            for (int jj = 0; jj < CH; ++jj) {
                const float sjj = Ss[(j0 + jj) * kp + j0 + jj];
                if (j0 + jj < k && sjj > 0.f) {
                    // the step's division as a product with the block's reciprocal: one
                    // multiply on the recurrence's dependent chain
                    const float si = sinv[j0 + jj];
                    const float xn = reg ? fmaxf(0.f, (fmaf(sjj, xc[jj], g[jj]) - beta) * si)
                                         : fmaxf(0.f, fmaf(g[jj], si, xc[jj]));
                    const float d = xn - xc[jj];
                    xc[jj] = xn;
#pragma unroll
                    for (int jn = jj + 1; jn < CH; ++jn) g[jn] = fmaf(-d, Ss[(j0 + jj) * kp + j0 + jn], g[jn]);
                }
            }
#pragma unroll
            for (int jj = 0; jj < CH; ++jj) xs[(j0 + jj) * xsp + vl] = xc[jj];
        }
        for (int i = 0; i < k; ++i) X[v * sv + (int64_t)i * se] = xs[i * xsp + vl];
    }
}

constexpr int LP = 128;                 // padded l (l <= 128)
constexpr int WH_SROWS = 4;             // streamed rows in flight per 8-lane group
constexpr int WH_TCH = 4;               // tensor-memory rows per load (one 64-column load)
constexpr int WH_NACC = 4;              // copies of each fixed-point sum (block b adds into copy b % 4)

// Shape of a W-half block: NT threads (a multiple of 128), REGR rows of Q in
// registers per 8-lane group; every 8-lane group also holds TMEM_ROWS rows in
// tensor memory (warps w, w + 4, ... share the lanes of one quarter and split
// its 512 columns).
template <int NT, int REGR>
struct WhShape {
    static constexpr int WARPS = NT / 32;
    static constexpr int GROUPS = WARPS * 4;            // 8-lane groups (one row of Q at a time each)
    static constexpr int RROWS = GROUPS * REGR;         // register-resident rows per block
    static constexpr int TMEM_COLS = 512 / (WARPS / 4);  // tensor-memory columns per thread
    static constexpr int TMEM_ROWS = TMEM_COLS / 16;     // tensor-memory rows per 8-lane group
    static constexpr int TROWS = GROUPS * TMEM_ROWS;     // tensor-memory rows per block (512)
    static constexpr int FIXED_FLOATS = 6 * LP + WARPS * LP;  // V, T double buffers, u, s_part, warp partials
    static_assert(WARPS % 4 == 0 && TMEM_ROWS % WH_TCH == 0, "W-half block shape");
};
constexpr size_t WH_SMEM_MAX = 232448;  // dynamic shared memory per block on sm_103
constexpr size_t WH_SMEM_ONE_PER_SM = 120 * 1024;  // above half of the SM's 228 KB

__device__ __forceinline__ unsigned long long wh_ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Tensor-memory rows of Q (32x32b shape: thread t of a warp reads and writes
// lane 32 (warp % 4) + t; consecutive columns are consecutive 32-bit words).
__device__ __forceinline__ void wh_tmem_st16(uint32_t taddr, const float4 (&q)[4]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(q[0].x)), "r"(__float_as_uint(q[0].y)), "r"(__float_as_uint(q[0].z)),
        "r"(__float_as_uint(q[0].w)), "r"(__float_as_uint(q[1].x)), "r"(__float_as_uint(q[1].y)),
        "r"(__float_as_uint(q[1].z)), "r"(__float_as_uint(q[1].w)), "r"(__float_as_uint(q[2].x)),
        "r"(__float_as_uint(q[2].y)), "r"(__float_as_uint(q[2].z)), "r"(__float_as_uint(q[2].w)),
        "r"(__float_as_uint(q[3].x)), "r"(__float_as_uint(q[3].y)), "r"(__float_as_uint(q[3].z)),
        "r"(__float_as_uint(q[3].w))
        : "memory");
}

#define WH_O4(b) "=r"(r[b]), "=r"(r[b + 1]), "=r"(r[b + 2]), "=r"(r[b + 3])
#define WH_O16(b) WH_O4(b), WH_O4(b + 4), WH_O4(b + 8), WH_O4(b + 12)
#define WH_P4(b) "+r"(r[b]), "+r"(r[b + 1]), "+r"(r[b + 2]), "+r"(r[b + 3])
#define WH_P16(b) WH_P4(b), WH_P4(b + 4), WH_P4(b + 8), WH_P4(b + 12)

// WH_TCH = 4 consecutive rows (64 columns) of this thread's lane.  The wait
// names the loaded registers, so no use of them can move above it.
__device__ __forceinline__ void wh_tmem_ld4rows(uint32_t taddr, float4 (&q)[WH_TCH][4]) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, "
        "%36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, "
        "%57, %58, %59, %60, %61, %62, %63}, [%64];"
        : WH_O16(0), WH_O16(16), WH_O16(32), WH_O16(48)
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : WH_P16(0), WH_P16(16), WH_P16(32), WH_P16(48)::"memory");
#pragma unroll
    for (int t = 0; t < WH_TCH; ++t)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            q[t][i] = make_float4(__uint_as_float(r[16 * t + 4 * i]), __uint_as_float(r[16 * t + 4 * i + 1]),
                                  __uint_as_float(r[16 * t + 4 * i + 2]), __uint_as_float(r[16 * t + 4 * i + 3]));
}
#undef WH_O4
#undef WH_O16
#undef WH_P4
#undef WH_P16

// q . u over one lane's 16 entries as packed pairs: lanes (.x, .y) and (.z, .w) of
// each float4 form two running sums, added pairwise at the end.
__device__ __forceinline__ float dot16(const float4 (&q)[4], const float4 (&u)[4]) {
    float2 s0 = f2_mul(lo2(q[0]), lo2(u[0])), s1 = f2_mul(lo2(q[1]), lo2(u[1]));
    float2 s2 = f2_mul(lo2(q[2]), lo2(u[2])), s3 = f2_mul(lo2(q[3]), lo2(u[3]));
    s0 = f2_fma(hi2(q[0]), hi2(u[0]), s0);
    s1 = f2_fma(hi2(q[1]), hi2(u[1]), s1);
    s2 = f2_fma(hi2(q[2]), hi2(u[2]), s2);
    s3 = f2_fma(hi2(q[3]), hi2(u[3]), s3);
    s0 = f2_add(f2_add(s0, s1), f2_add(s2, s3));
    return s0.x + s0.y;
}

__device__ __forceinline__ void axpy16(float w, const float4 (&q)[4], float4 (&p)[4]) {
    const float2 ww = make_float2(w, w);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 a = f2_fma(ww, lo2(q[i]), lo2(p[i]));
        const float2 b = f2_fma(ww, hi2(q[i]), hi2(p[i]));
        p[i] = make_float4(a.x, a.y, b.x, b.y);
    }
}

// Persistent W half-sweep.  Block b owns rows [r0, r0 + R) of Q: the first 192
// are held in registers (6 rows x 16 floats per lane of each 8-lane group),
// the next (up to 512) in tensor memory (16 rows x 16 floats per lane: every
// thread owns 256 columns of its TMEM lane, read back 4 rows per tcgen05.ld),
// the next Rs in shared memory, the rest are read from L2.  Per column j:
//   u_j  = W~_j + (T_:j - z_j) / V_jj, z_j = (W~ V)_:j
//   w_r  = max(0, Q_r u_j), W(r, j) = w_r
//   p_b  = sum_r w_r Q_r, rounded to an integer term t_b = p_b 2^S (|t_b| < 2^46)
//          and added with one 64-bit atomic per entry into copy b % 4 of the
//          column's counted words: bits 0..55 hold sum (t_b + 2^47), bits
//          56..63 count the blocks that have added.  A block waits until the
//          counts of all four copies are complete (bounded spin) - the data
//          and its count arrive in the same atomic word, so no fence or
//          separate barrier counter is needed, and integer addition makes the
//          sum exact and independent of arrival order.
//   W~_j = (sum of the copies - count 2^47) 2^-S rounded once to float32
//          (bit-identical in every block and in every run)
// The scale S is the same in every block: it comes from M = max_i |u_i| (u is
// bit-identical everywhere) and the once-per-Q factor bf >= |Q|_F max_i |Q_:i|
// sqrt(128), through |sum_{r in b} w_r Q_ri| <= |Q u| |Q_:i| <= |Q|_F sqrt(l) M
// max_i |Q_:i| (Cauchy-Schwarz; |w_r| <= |Q_r u|), which holds for any Q.
// Every column has its own words (zeroed before the launch), so no word is
// reused within a launch.
// While block b waits at the barrier it already sums z_{j+1} over every column
// except j (those columns do not change at this step), so after the barrier
// only the column-j term remains: u_{j+1} costs one FMA per entry.
// Thread (rt = tid / 2, rq = tid % 2) owns entry rt of the l-vectors.
template <int WH_NT, int WH_REG_ROWS>
__global__ void __launch_bounds__(WH_NT, 1) whalf_kernel(const float* __restrict__ Qp, int64_t m, int l, int lp, int k,
                                                         int rs_max, float* __restrict__ Wc, float* __restrict__ Wt_g,
                                                         const float* __restrict__ Tt_g, const float* __restrict__ V_g,
                                                         unsigned long long* acc, int* status, long long spin_limit,
                                                         int reg, float alpha, float beta,
                                                         const float* __restrict__ q1, const float* __restrict__ bf_g,
                                                         int jbeg, int jend) {
    using Sh = WhShape<WH_NT, WH_REG_ROWS>;
    constexpr int WH_WARPS = Sh::WARPS, WH_GROUPS = Sh::GROUPS, WH_RROWS = Sh::RROWS;
    constexpr int WH_TMEM_COLS = Sh::TMEM_COLS, WH_TROWS = Sh::TROWS;
    extern __shared__ __align__(16) float sm[];
    float* Vb = sm;                       // [2][LP] rows j, j+1 of V
    float* Tb = Vb + 2 * LP;              // [2][LP] columns j, j+1 of T
    float* u = Tb + 2 * LP;               // [LP]
    float* spart = u + LP;                // [LP] z_{j+1} without column j
    float* red = spart + LP;              // [WH_WARPS][LP]
    float* Ws = red + WH_WARPS * LP;      // [l][k + 1]  W~ (padded pitch)
    const int kp1 = k + 1;
    float* Qc = Ws + ((l * kp1 + 3) & ~3);  // [Rs][lp]
    const float bound0 = __ldg(bf_g);  // |term| <= bound0 M before scaling
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int rt = tid >> 1, rq = tid & 1;
    const int nch = lp >> 2;
    const int nblk = (int)gridDim.x;
    const int64_t rpb = (m + nblk - 1) / nblk;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int R = (int)(r0 >= m ? 0 : (r0 + rpb <= m ? rpb : m - r0));
    const int RR = R < WH_RROWS ? R : WH_RROWS;               // register rows [0, RR)
    const int RT = (R - RR) < WH_TROWS ? (R - RR) : WH_TROWS;  // tensor-memory rows [RR, RR + RT)
    const int RB = RR + RT;
    const int RS = (R - RB) < rs_max ? (R - RB) : rs_max;     // shared rows [RB, RB + RS)
    const int g = lane >> 3, g8 = lane & 7, grp = warp * 4 + g;
    // tensor-memory slots per group in use (row RR + WH_GROUPS s + grp in slot s),
    // a multiple of WH_TCH; unused slots hold zeros
    const int nts = ((RT + WH_GROUPS - 1) / WH_GROUPS + WH_TCH - 1) / WH_TCH * WH_TCH;
    const bool use_tmem = RT > 0;  // block-uniform
    if (use_tmem && warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // warps w, w + 4, .. share TMEM lanes 32 (w % 4) ..; they split the 512 columns
    const uint32_t tbase =
        use_tmem ? s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * WH_TMEM_COLS) : 0u;
    auto release_tmem = [&]() {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (use_tmem && warp == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(s_tmem) : "memory");
        }
    };
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4* Qg4 = reinterpret_cast<const float4*>(Qp + r0 * lp);
    // register-resident rows: group (warp, g) holds rows (warp * 4 + g) * WH_REG_ROWS + s
    float4 qr[WH_REG_ROWS > 0 ? WH_REG_ROWS : 1][4];
#pragma unroll
    for (int s2 = 0; s2 < WH_REG_ROWS; ++s2) {
        const int r = (warp * 4 + g) * WH_REG_ROWS + s2;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = g8 + 8 * i;
            qr[s2][i] = (r < RR && c < nch) ? __ldg(Qg4 + (int64_t)r * nch + c) : z4;
        }
    }
    for (int s2 = 0; s2 < nts; ++s2) {
        const int rr = s2 * WH_GROUPS + grp;
        float4 q[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = g8 + 8 * i;
            q[i] = (rr < RT && c < nch) ? __ldg(Qg4 + (int64_t)(RR + rr) * nch + c) : z4;
        }
        wh_tmem_st16(tbase + 16u * s2, q);
    }
    if (use_tmem) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    {
        const float4* src = Qg4 + (int64_t)RB * nch;
        float4* dst = reinterpret_cast<float4*>(Qc);
        for (int e = tid; e < RS * nch; e += WH_NT) cp_async16(dst + e, src + e, true);
    }
    for (int e = tid; e < l * k; e += WH_NT) cp_async4(&Ws[(e / k) * kp1 + (e % k)], Wt_g + e, true);
    cp_async_wait_all();
    for (int e = tid; e < LP; e += WH_NT) {
        Vb[(jbeg & 1) * LP + e] = e < k ? V_g[(int64_t)jbeg * k + e] : 0.f;
        Tb[(jbeg & 1) * LP + e] = e < l ? Tt_g[(int64_t)jbeg * l + e] : 0.f;
        u[e] = 0.f;
    }
    __syncthreads();
    const float4* Qc4 = reinterpret_cast<const float4*>(Qc);
    bool u_ready = false;  // u already holds u_j (computed at the end of column j-1)
    for (int j = jbeg; j < jend; ++j) {
        const int cur = j & 1;
        float pv = 0.f, pt = 0.f;
        if (j + 1 < jend && tid < LP) {
            pv = tid < k ? V_g[(int64_t)(j + 1) * k + tid] : 0.f;
            pt = tid < l ? Tt_g[(int64_t)(j + 1) * l + tid] : 0.f;
        }
        const float vjj = Vb[cur * LP + j];
        if (!(vjj > 0.f)) {  // dead component: column left unchanged (same decision in every block)
            if (j + 1 < jend && tid < LP) {
                Vb[(cur ^ 1) * LP + tid] = pv;
                Tb[(cur ^ 1) * LP + tid] = pt;
            }
            u_ready = false;
            __syncthreads();
            continue;
        }
        if (!u_ready) {
            float s = 0.f;
            if (rt < l)
                for (int i = rq; i < k; i += 2) s = fmaf(Ws[rt * kp1 + i], Vb[cur * LP + i], s);
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            if (rt < l && rq == 0) {
                if (reg)  // Section 3.4 W~ rule: (V_jj w + T_j - beta Q^T 1 - W~ V_j) / (V_jj + alpha)
                    u[rt] = (fmaf(vjj, Ws[rt * kp1 + j], Tb[cur * LP + rt] - s) - beta * q1[rt]) / (vjj + alpha);
                else
                    u[rt] = Ws[rt * kp1 + j] + (Tb[cur * LP + rt] - s) / vjj;
            }
            __syncthreads();
        }
        float4 uu[4], pp[4];
        float mu = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uu[i] = reinterpret_cast<const float4*>(u)[g8 + 8 * i];
            pp[i] = z4;
            mu = fmaxf(mu, fmaxf(fmaxf(fabsf(uu[i].x), fabsf(uu[i].y)), fmaxf(fabsf(uu[i].z), fabsf(uu[i].w))));
        }
        // M = max_i |u_i| (exact, so equal in every block) and the scale S
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) mu = fmaxf(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        int S = 0;
        {
            const float bound = bound0 * mu;
            if (bound > 0.f && bound <= 3.0e38f) {
                int e;
                frexpf(bound, &e);  // bound < 2^e
                S = 46 - e;
            }
        }
        // register rows
        {
            float d[WH_REG_ROWS > 0 ? WH_REG_ROWS : 1];
#pragma unroll
            for (int s2 = 0; s2 < WH_REG_ROWS; ++s2) d[s2] = dot16(qr[s2], uu);
#pragma unroll
            for (int o = 1; o < 8; o <<= 1)
#pragma unroll
                for (int s2 = 0; s2 < WH_REG_ROWS; ++s2) d[s2] += __shfl_xor_sync(0xffffffffu, d[s2], o);
#pragma unroll
            for (int s2 = 0; s2 < WH_REG_ROWS; ++s2) {
                const int r = (warp * 4 + g) * WH_REG_ROWS + s2;
                const float w = r < RR ? fmaxf(0.f, d[s2]) : 0.f;
                if (g8 == 0 && r < RR) Wc[(int64_t)j * m + r0 + r] = w;
                axpy16(w, qr[s2], pp);
            }
        }
        // tensor-memory rows, WH_TCH per load
        for (int s0 = 0; s0 < nts; s0 += WH_TCH) {
            float4 q[WH_TCH][4];
            wh_tmem_ld4rows(tbase + 16u * s0, q);
            float d[WH_TCH];
#pragma unroll
            for (int t = 0; t < WH_TCH; ++t) d[t] = dot16(q[t], uu);
#pragma unroll
            for (int o = 1; o < 8; o <<= 1)
#pragma unroll
                for (int t = 0; t < WH_TCH; ++t) d[t] += __shfl_xor_sync(0xffffffffu, d[t], o);
#pragma unroll
            for (int t = 0; t < WH_TCH; ++t) {
                const int rr = (s0 + t) * WH_GROUPS + grp;
                const float w = rr < RT ? fmaxf(0.f, d[t]) : 0.f;
                if (g8 == 0 && rr < RT) Wc[(int64_t)j * m + r0 + RR + rr] = w;
                axpy16(w, q[t], pp);
            }
        }
        // streamed rows: first the shared-memory copy, then L2; each loop issues
        // one kind of load only.  Row index past the tensor-memory rows:
        // rr = base + g + 32 s2 with base running over multiples of 4 per warp.
        auto stream = [&](const float4* src, int64_t src_off, int lo, int hi) {
            for (int wb = lo + warp * 4; wb < hi; wb += WH_WARPS * 4 * WH_SROWS) {
                float4 q[WH_SROWS][4];
#pragma unroll
                for (int s2 = 0; s2 < WH_SROWS; ++s2) {
                    const int rr = wb + g + WH_WARPS * 4 * s2;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int c = g8 + 8 * i;
                        q[s2][i] = (rr < hi && c < nch) ? src[(int64_t)(rr - src_off) * nch + c] : z4;
                    }
                }
                float d[WH_SROWS];
#pragma unroll
                for (int s2 = 0; s2 < WH_SROWS; ++s2) d[s2] = dot16(q[s2], uu);
#pragma unroll
                for (int o = 1; o < 8; o <<= 1)
#pragma unroll
                    for (int s2 = 0; s2 < WH_SROWS; ++s2) d[s2] += __shfl_xor_sync(0xffffffffu, d[s2], o);
#pragma unroll
                for (int s2 = 0; s2 < WH_SROWS; ++s2) {
                    const int rr = wb + g + WH_WARPS * 4 * s2;
                    const float w = rr < hi ? fmaxf(0.f, d[s2]) : 0.f;
                    if (g8 == 0 && rr < hi) Wc[(int64_t)j * m + r0 + RB + rr] = w;
                    axpy16(w, q[s2], pp);
                }
            }
        };
        stream(Qc4, 0, 0, RS);                                  // shared-memory rows [0, RS)
        stream(Qg4 + (int64_t)RB * nch, 0, RS, R - RB);         // L2 rows [RS, R - RB)
        // warp partial: sum the four 8-lane groups, group 0 stores it
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int o = 8; o < 32; o <<= 1) {
                pp[i].x += __shfl_xor_sync(0xffffffffu, pp[i].x, o);
                pp[i].y += __shfl_xor_sync(0xffffffffu, pp[i].y, o);
                pp[i].z += __shfl_xor_sync(0xffffffffu, pp[i].z, o);
                pp[i].w += __shfl_xor_sync(0xffffffffu, pp[i].w, o);
            }
            if (g == 0) reinterpret_cast<float4*>(red + warp * LP)[g8 + 8 * i] = pp[i];
        }
        if (j + 1 < jend && tid < LP) {
            Vb[(cur ^ 1) * LP + tid] = pv;
            Tb[(cur ^ 1) * LP + tid] = pt;
        }
        __syncthreads();
        unsigned long long* accj = acc + (size_t)j * WH_NACC * LP;
        {
            float s = 0.f;
            if (rt < l)
                for (int w = rq; w < WH_WARPS; w += 2) s += red[w * LP + rt];
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            if (rt < l && rq == 0) {
                const float sc = ldexpf(s, S);
                // in range by the bound; a non-finite partial adds 0 so the counts stay intact
                const long long term = fabsf(sc) < 0x1p46f ? __float2ll_rn(sc) : 0ll;
                atomicAdd(accj + (blockIdx.x % WH_NACC) * LP + rt,
                          (unsigned long long)(term + (1ll << 47)) + (1ull << 56));
            }
        }
        // while the other blocks add: z_{j+1} over every column except j
        const bool next = j + 1 < jend && Vb[(cur ^ 1) * LP + j + 1] > 0.f;
        if (next) {
            float a0 = 0.f, a1 = 0.f;
            if (rt < l) {
                const float* wrow = Ws + rt * kp1;
                const float* vrow = Vb + (cur ^ 1) * LP;
                int i = rq;
                for (; i + 2 < k; i += 4) {
                    a0 = fmaf(i == j ? 0.f : wrow[i], vrow[i], a0);
                    a1 = fmaf(i + 2 == j ? 0.f : wrow[i + 2], vrow[i + 2], a1);
                }
                for (; i < k; i += 2) a0 = fmaf(i == j ? 0.f : wrow[i], vrow[i], a0);
            }
            float sp = a0 + a1;
            sp += __shfl_xor_sync(0xffffffffu, sp, 1);
            if (rt < l && rq == 0) spart[rt] = sp;
        }
        // wait until every block's term of entry rt has landed (all four copies
        // read per round trip); bounded by spin_limit and the status word
        int ok = 1;
        unsigned long long tot = 0ull;
        if (rt < l && rq == 0) {
            const long long t0 = clock64();
            for (;;) {
                unsigned long long w[WH_NACC];
#pragma unroll
                for (int c = 0; c < WH_NACC; ++c) w[c] = wh_ld_relaxed(accj + c * LP + rt);
                bool done = true;
                long long cnt = 0;
                tot = 0ull;
#pragma unroll
                for (int c = 0; c < WH_NACC; ++c) {
                    const int need = (nblk - c + WH_NACC - 1) / WH_NACC;  // blocks b < nblk with b % WH_NACC == c
                    done = done && (int)(w[c] >> 56) >= need;
                    tot += w[c] & ((1ull << 56) - 1);
                    cnt += need;
                }
                if (done) {
                    tot -= (unsigned long long)cnt << 47;  // remove the offsets: the exact sum of the terms
                    break;
                }
                if (clock64() - t0 > spin_limit || rnmf_ld_volatile(status) != RNMF_DEV_OK) {
                    atomicCAS(status, RNMF_DEV_OK, RNMF_DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        if (!__syncthreads_and(ok)) {
            release_tmem();
            return;
        }
        if (rt < l && rq == 0) {
            // W~_j: the exact integer sum, one rounding to float32
            const float wj = ldexpf(__ll2float_rn((long long)tot), -S);
            Ws[rt * kp1 + j] = wj;
            if (next) {
                const float vn = Vb[(cur ^ 1) * LP + j + 1];
                const float z = fmaf(wj, Vb[(cur ^ 1) * LP + j], spart[rt]);
                if (reg)
                    u[rt] = (fmaf(vn, Ws[rt * kp1 + j + 1], Tb[(cur ^ 1) * LP + rt] - z) - beta * q1[rt]) /
                            (vn + alpha);
                else
                    u[rt] = Ws[rt * kp1 + j + 1] + (Tb[(cur ^ 1) * LP + rt] - z) / vn;
            }
        }
        u_ready = next;
        __syncthreads();
    }
    if (blockIdx.x == 0)
        for (int e = tid; e < l * k; e += WH_NT) Wt_g[e] = Ws[(e / k) * kp1 + (e % k)];
    release_tmem();
}

// Q^T 1 (l column sums of Q, rows padded to lp): one block per column, fixed
// reduction order.
__global__ void __launch_bounds__(256) colsum_kernel(const float* __restrict__ Qp, int64_t m, int lp,
                                                     float* __restrict__ out) {
    __shared__ double red[256];
    const int t = blockIdx.x;
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < m; r += 256) s += Qp[r * lp + t];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[t] = (float)red[0];
}

// Sum of squares of every column of Q (one block per column, fixed reduction order).
__global__ void __launch_bounds__(256) q_colsq_kernel(const float* __restrict__ Qp, int64_t m, int lp,
                                                      double* __restrict__ out) {
    __shared__ double red[256];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < m; r += 256) {
        const double v = Qp[r * lp + c];
        s = fma(v, v, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
}

// bf = |Q|_F max_i |Q_:i| sqrt(128), 1% over for rounding (one thread, fixed order).
__global__ void q_bound_kernel(const double* __restrict__ colsq, int l, float* __restrict__ bf) {
    double f2 = 0.0, c2 = 0.0;
    for (int i = 0; i < l; ++i) {
        f2 += colsq[i];
        c2 = colsq[i] > c2 ? colsq[i] : c2;
    }
    *bf = (float)(sqrt(f2 * c2) * 11.313708498984761 * 1.01);
}

// whalf scratch: the bound factor bf (float) at 0, then the counted words of
// every column, [k][WH_NACC][LP] u64 (zeroed before each launch; the column
// square sums of Q pass through them once, before the first launch)
constexpr size_t WH_SCR_ACC = 128;
size_t wh_acc_bytes(int k) { return (size_t)k * WH_NACC * LP * sizeof(unsigned long long); }

struct WhalfLaunch {
    int grid;
    int rs_max;
    size_t smem;
};

// The W-half block shape in use: threads per block, register rows per 8-lane group.
constexpr int WH_NT = 256, WH_REGR = 6;
using WhCur = WhShape<WH_NT, WH_REGR>;

WhalfLaunch whalf_config(rnmf_ctx* ctx, int64_t m, int lp, int l, int k) {
    constexpr int WH_RROWS = WhCur::RROWS, WH_TROWS = WhCur::TROWS, WH_FIXED_FLOATS = WhCur::FIXED_FLOATS;
    WhalfLaunch c;
    // at most 256 blocks: 64 per copy, within the 8-bit count and the 56-bit sum of the words
    c.grid = ctx->num_sms < 256 ? ctx->num_sms : 256;
    int64_t byrows = (m + 31) / 32;
    if (c.grid > byrows) c.grid = (int)byrows;
    if (c.grid < 1) c.grid = 1;
    int64_t rpb = (m + c.grid - 1) / c.grid - WH_RROWS - WH_TROWS;
    if (rpb < 0) rpb = 0;
    const size_t fixed = ((size_t)WH_FIXED_FLOATS + (((size_t)l * (k + 1) + 3) & ~size_t(3))) * sizeof(float);
    int64_t fit = (int64_t)((WH_SMEM_MAX - fixed - 256) / ((size_t)lp * sizeof(float)));
    c.rs_max = (int)(rpb < fit ? rpb : fit);
    c.smem = fixed + (size_t)c.rs_max * lp * sizeof(float);
    // A block with tensor-memory rows allocates all 512 columns of its SM's
    // tensor memory, so no second block may share the SM: more than half of
    // the SM's shared memory per block makes that so.
    if ((m + c.grid - 1) / c.grid > WH_RROWS && c.smem < WH_SMEM_ONE_PER_SM) c.smem = WH_SMEM_ONE_PER_SM;
    return c;
}

}  // namespace

bool launch_hals_rows(rnmf_ctx* ctx, float* X, int64_t sv, int64_t se, const float* Rhs, int64_t srv, int64_t srj,
                      const float* S, int64_t count, int k, float alpha, float beta) {
    if (count <= 0) return true;
    const int kp = (k + CH - 1) / CH * CH;
    // one block per SM large enough that a single round covers every vector, when
    // shared memory (S plus the block's vectors) and the thread limit allow
    const size_t smem_max = 227 * 1024;
    int vmax = (int)(((int64_t)(smem_max / sizeof(float)) - (int64_t)kp * kp) / kp) - 16;
    if (vmax > ROWS_NT_MAX) vmax = ROWS_NT_MAX;
    vmax = vmax / 32 * 32;
    if (vmax < 32) vmax = 32;
    const int64_t per_sm = (count + ctx->num_sms - 1) / ctx->num_sms;
    int vpb = (int)((per_sm + 31) / 32 * 32);
    if (vpb > vmax) vpb = vmax;
    if (vpb < 32) vpb = 32;
    const int nt = vpb;
    size_t smem = ((size_t)kp * kp + (size_t)kp * (vpb + 4) + (size_t)kp) * sizeof(float);
    cudaFuncSetAttribute(hals_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hals_rows_kernel, nt, smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    const int64_t groups = (count + vpb - 1) / vpb;
    const int64_t slots = (int64_t)ctx->num_sms * occ;
    unsigned grid = (unsigned)(groups < slots ? groups : slots);
    prof_begin(ctx);
    const int reg = alpha != 0.f || beta != 0.f;
    hals_rows_kernel<<<grid, nt, smem, ctx->stream>>>(X, sv, se, Rhs, srv, srj, S, count, k, reg, alpha, beta);
    return launch_done(ctx, K_HALS_ROWS, 12.0 * count * k + 4.0 * k * k, 2.0 * count * k * k);
}

bool launch_colsum(rnmf_ctx* ctx, const float* Qp, int64_t m, int l, int lp, float* out) {
    prof_begin(ctx);
    colsum_kernel<<<l, 256, 0, ctx->stream>>>(Qp, m, lp, out);
    return launch_done(ctx, K_WHALF, 4.0 * m * l, (double)m * l);
}

size_t whalf_scratch_bytes(rnmf_ctx*, int64_t, int l, int k) {
    const size_t a = wh_acc_bytes(k), b = (size_t)l * sizeof(double);
    return WH_SCR_ACC + (a > b ? a : b);
}

bool launch_whalf_prepare(rnmf_ctx* ctx, const float* Qp, int64_t m, int l, int lp, char* scratch) {
    double* colsq = reinterpret_cast<double*>(scratch + WH_SCR_ACC);
    prof_begin(ctx);
    q_colsq_kernel<<<l, 256, 0, ctx->stream>>>(Qp, m, lp, colsq);
    if (!launch_done(ctx, K_TRANSPOSE, 4.0 * m * l, 2.0 * m * l)) return false;
    prof_begin(ctx);
    q_bound_kernel<<<1, 1, 0, ctx->stream>>>(colsq, l, reinterpret_cast<float*>(scratch));
    return launch_done(ctx, K_TRANSPOSE, 8.0 * l, 2.0 * l);
}

bool launch_whalf(rnmf_ctx* ctx, const float* Qp, int64_t m, int l, int lp, int k, float* Wc, float* Wt,
                  const float* Tt, const float* V, char* scratch, long long spin_limit, float alpha, float beta,
                  const float* q1, int jbeg, int jend) {
    if (jend < 0) jend = k;
    if (jbeg >= jend) return true;
    WhalfLaunch c = whalf_config(ctx, m, lp, l, k);
    cudaFuncSetAttribute(whalf_kernel<WH_NT, WH_REGR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
    // the counted words of columns [jbeg, jend) start at zero
    const size_t col_bytes = wh_acc_bytes(1);
    if (cudaMemsetAsync(scratch + WH_SCR_ACC + (size_t)jbeg * col_bytes, 0, (size_t)(jend - jbeg) * col_bytes,
                        ctx->stream) != cudaSuccess)
        return false;
    prof_begin(ctx);
    // blocks poll words that every other block adds to: a cooperative launch
    if (!launch_cooperative(ctx, whalf_kernel<WH_NT, WH_REGR>, (unsigned)c.grid, WH_NT, c.smem, Qp, m, l, lp, k, c.rs_max, Wc, Wt, Tt,
                            V, reinterpret_cast<unsigned long long*>(scratch + WH_SCR_ACC), ctx->d_status,
                            spin_limit > 0 ? spin_limit : RNMF_DEFAULT_SPIN_LIMIT,
                            (alpha != 0.f || beta != 0.f) ? 1 : 0, alpha, beta, q1,
                            reinterpret_cast<const float*>(scratch), jbeg, jend))
        return false;
    // compulsory traffic: Q once, W written once; flops: Q u and Q^T w for each column
    const double cols = jend - jbeg;
    return launch_done(ctx, K_WHALF, 4.0 * m * l + 4.0 * m * cols, 4.0 * m * l * cols);
}
