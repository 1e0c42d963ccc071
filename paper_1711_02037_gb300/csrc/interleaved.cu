// interleaved.cu - the interleaved cyclic update order W_1 -> H_1 -> ... -> W_k -> H_k
// (Section 3.2), two passes per component.
//
// Every block update of this order reads the factor it changes once and the
// products the next update needs come from the same columns, so one pass over
// a pair (X, Y) does both:
//   * W pass (component j): X = Q (m x lp, rows padded), Y = W^T (k x m).  Per
//     row r: W_j(r) = max(0, Q_r u) with u the W~ rule of Section 3.2 from
//     T_:j, V_:j; then W~_:j = Q^T W_j (the reprojection) and S_:j = W^T W_j.
//   * H pass (component j, then jn): X = B^T (n x l), Y = H (k x n).  Per column
//     c: H_j(c) from the H rule with R_j(c) = B_:c . W~_:j and S_:j; then the
//     next W update's T_:jn = B H_jn^T and V_:jn = H H_jn^T with the new row j.
// A block owns a contiguous range of rows (columns of Y), streamed through
// shared memory in tiles of IL_TC, three stages deep: one thread issues two TMA
// box loads per tile (X: IL_TC rows x a padded row pitch, the pad columns
// zero-filled as out of range; Y: k rows x IL_YP columns) that complete on the
// stage's mbarrier, every wait bounded; shapes whose rows are not 16-byte
// multiples take per-thread cp.async copies instead.  A thread's
// float32 tile sums are added into a two-sum pair (pair_sum.cuh), the block
// partials are such pairs, and the block that draws the last ticket adds them
// the same way in block order, so results are bit-identical from run to run.
#include <cstring>

#include "async_copy.cuh"
#include "pair_sum.cuh"
#include "rnmf_internal.cuh"
#include "tma.cuh"

namespace {

constexpr int IL_NT = 512;
constexpr int IL_TC = 64;           // rows of X (columns of Y) per tile
constexpr int IL_YP = IL_TC + 4;    // Y tile row pitch (17 16-byte units): float4 reads down a column are conflict-free
constexpr int IL_MAX = 128;         // l, lp and k are at most 128
constexpr int IL_STAGES = 3;
constexpr int IL_NE = 2 * IL_MAX;   // partial entries: P (X^T y) then S (Y y)

// Smallest X tile row pitch >= round4(pitch) that is 4 mod 32 floats: a float4
// read of the same column by 8 consecutive rows then touches 8 different
// 16-byte bank groups (no bank conflict).
__host__ __device__ inline int il_xp(int pitch) {
    int p = (pitch + 3) / 4 * 4;
    while (p % 32 != 4) p += 4;
    return p;
}

struct IlPass {
    const float* X;  // rows of `pitch` floats, entries [0, lx) used
    int pitch, lx;
    float* Y;        // k x N, row stride N
    int64_t N;
    int k;
    int mode;        // 0: H rule on row j; 1: W rule on row j (reprojection); -1: no update
    int j, jn;       // updated row, row whose products are formed (-1: none)
    // H rule: a = W~_:j (column j of Wt, l x k), s = S_:j; W rule: u from W~, T_:j, V_:j
    const float* Wt;
    const float* S_row;
    const float* T_row;
    const float* V_row;
    const float* q1;
    int reg;
    float alpha, beta;
    int gram_mode;   // W pass: 1 forms S_:j = W~^T W~_j instead of W^T W_j
    // outputs of the products (float32, written by the last block)
    float* P_out;
    int64_t P_stride;
    float* S_out;
    int64_t rchunk;  // rows per block, a multiple of 4
    float2* partial;  // [gridDim.x][IL_NE] (sum, compensation)
    unsigned* ticket;  // zero before the launch; the last block resets it
    int use_tma;       // 1: TMA boxes (pitch and N multiples of 4, 16-byte aligned bases)
    int* status;       // RNMF_DEV_TIMEOUT when a tile's copies do not land within spin_limit cycles
    long long spin_limit;
};

__host__ __device__ inline size_t il_align128(size_t b) { return (b + 127) / 128 * 128; }
// float offset of stage s (stages start on 128-byte boundaries, X box first)
__host__ __device__ inline size_t il_stage_floats(int pitch, int k) {
    return (il_align128((size_t)IL_TC * il_xp(pitch) * 4) + il_align128((size_t)k * IL_YP * 4)) / 4;
}

__global__ void __launch_bounds__(IL_NT, 1) il_pass_kernel(const __grid_constant__ CUtensorMap tmX,
                                                           const __grid_constant__ CUtensorMap tmY, IlPass a) {
    extern __shared__ __align__(128) float ilsm_raw[];
    // the dynamic buffer is over-allocated by 128 bytes: stages start 128-byte aligned
    float* ilsm = ilsm_raw + ((128 - (smem_u32(ilsm_raw) & 127)) & 127) / 4;
    const int XP = il_xp(a.pitch);
    const int st_f = (int)il_stage_floats(a.pitch, a.k);
    float* stage0 = ilsm;
    float* vec = ilsm + IL_STAGES * st_f;  // [IL_MAX] a or u, [IL_MAX] s
    float* red = vec + 2 * IL_MAX;                  // [8][IL_TC]
    float2* dred = reinterpret_cast<float2*>(red + 8 * IL_TC);  // [IL_NE]
    __shared__ int s_last;
    __shared__ int s_alive;
    __shared__ __align__(8) uint64_t full_bar[IL_STAGES];
    const int tid = threadIdx.x;
    const int k = a.k;
    const int64_t rbeg = (int64_t)blockIdx.x * a.rchunk;
    const int64_t rend = rbeg + a.rchunk < a.N ? rbeg + a.rchunk : a.N;
    const int ntile = rbeg < rend ? (int)((rend - rbeg + IL_TC - 1) / IL_TC) : 0;
    const bool xvec = (a.pitch % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.X) & 15) == 0);
    const bool yvec = (a.N % 4 == 0) && ((reinterpret_cast<uintptr_t>(a.Y) & 15) == 0);

    const uint32_t bytes_tile = (uint32_t)(IL_TC * XP + k * IL_YP) * 4;
    auto load_tile = [&](int t) {
        float* xs = stage0 + (t % IL_STAGES) * st_f;
        float* ys = xs + (st_f - (int)(il_align128((size_t)k * IL_YP * 4) / 4));
        const int64_t r0 = rbeg + (int64_t)t * IL_TC;
        if (a.use_tma) {
            if (tid == 0) {
                const uint32_t bar = smem_u32(&full_bar[t % IL_STAGES]);
                fence_proxy_async();  // generic-proxy writes of this stage's last use come first
                mbar_expect_tx(bar, bytes_tile);
                tma_load_2d(smem_u32(xs), &tmX, 0, (int)r0, bar);
                tma_load_2d(smem_u32(ys), &tmY, (int)r0, 0, bar);
            }
            return;
        }
        const int nr = (int)(rend - r0 < IL_TC ? rend - r0 : IL_TC);
        if (xvec) {
            const int q4 = XP / 4, pq = a.pitch / 4;
            for (int e = tid; e < IL_TC * q4; e += IL_NT) {
                const int r = e / q4, q = e % q4;
                const bool ok = r < nr && q < pq;
                cp_async16_n(xs + r * XP + 4 * q, ok ? a.X + (r0 + r) * a.pitch + 4 * q : a.X, ok ? 16 : 0);
            }
        } else {
            for (int e = tid; e < IL_TC * XP; e += IL_NT) {
                const int r = e / XP, q = e % XP;
                const bool ok = r < nr && q < a.pitch;
                cp_async4(xs + e, ok ? a.X + (r0 + r) * a.pitch + q : a.X, ok);
            }
        }
        if (yvec) {
            constexpr int q4 = IL_YP / 4;
            for (int e = tid; e < k * q4; e += IL_NT) {
                const int i = e / q4, q = e % q4;
                const int rem = nr - 4 * q;
                const int bytes = q < IL_TC / 4 && rem > 0 ? (rem >= 4 ? 16 : rem * 4) : 0;
                cp_async16_n(ys + i * IL_YP + 4 * q, bytes ? a.Y + (int64_t)i * a.N + r0 + 4 * q : a.Y, bytes);
            }
        } else {
            for (int e = tid; e < k * IL_YP; e += IL_NT) {
                const int i = e / IL_YP, c = e % IL_YP;
                const bool ok = c < nr;
                cp_async4(ys + e, ok ? a.Y + (int64_t)i * a.N + r0 + c : a.Y, ok);
            }
        }
    };

    if (a.use_tma) {
        if (tid == 0) {
            for (int st = 0; st < IL_STAGES; ++st) mbar_init(smem_u32(&full_bar[st]), 1);
            fence_barrier_init();
        }
        __syncthreads();
    }
    // the first tiles are in flight while the rule's vector is formed
    for (int t = 0; t < IL_STAGES - 1; ++t) {
        if (t < ntile) load_tile(t);
        cp_async_commit();
    }
    const int j = a.j;
    // vec[0, IL_MAX): W~_:j (H rule) or u (W rule), zero beyond l; vec[IL_MAX + i]: S_ij (H rule)
    if (tid < IL_MAX) vec[IL_MAX + tid] = (a.mode == 0 && tid < k) ? a.S_row[tid] : 0.f;
    if (tid == 0) s_alive = a.mode == 1 ? (a.V_row[j] > 0.f) : (a.mode == 0 ? (a.S_row[j] > 0.f) : 0);
    if (a.mode == 1) {
        // u = W~_:j + (T_:j - W~ V_:j) / V_jj  (Section 3.4 form when reg), four threads per entry
        const float vjj = a.V_row[j];
        const int i = tid >> 2, part = tid & 3;
        float s = 0.f;
        if (i < a.lx) {
            // eight independent loads in flight per step; the sum keeps q order
            for (int q0 = part; q0 < k; q0 += 32) {
                float wv[8], vv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int q = q0 + 4 * u;
                    wv[u] = q < k ? a.Wt[(int64_t)i * k + q] : 0.f;
                    vv[u] = q < k ? a.V_row[q] : 0.f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) s = fmaf(wv[u], vv[u], s);
            }
        }
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        if (part == 0) {
            float u = 0.f;
            if (i < a.lx && vjj > 0.f) {
                const float w = a.Wt[(int64_t)i * k + j], t = a.T_row[i];
                const float bq = a.beta != 0.f ? a.beta * a.q1[i] : 0.f;
                u = a.reg ? (fmaf(vjj, w, t - s) - bq) / (vjj + a.alpha) : w + (t - s) / vjj;
            }
            vec[i] = u;
        }
    } else if (tid < IL_MAX) {
        vec[tid] = (a.mode == 0 && tid < a.lx) ? a.Wt[(int64_t)tid * k + j] : 0.f;
    }
    __syncthreads();
    const bool alive = s_alive != 0;
    const float djj = a.mode == 0 ? vec[IL_MAX + j] : 0.f;

    const int c_own = tid & (IL_TC - 1), part = tid >> 6;  // update phase: column, eighth of the dot
    const int e_own = tid & (IL_NE - 1), half = tid >> 8;  // product phase: entry, half of the tile
    float2 acc = make_float2(0.f, 0.f);
    for (int t = 0; t < ntile; ++t) {
        bool landed = true;
        if (a.use_tma)
            landed = mbar_wait_bounded(smem_u32(&full_bar[t % IL_STAGES]), (t / IL_STAGES) & 1, a.spin_limit);
        else
            cp_async_wait_1();
        if (!__syncthreads_and(landed)) {
            // a tile did not land: record it, wait (bounded) for the copies still in flight, leave
            if (tid == 0) {
                atomicCAS(a.status, RNMF_DEV_OK, RNMF_DEV_TIMEOUT);
                for (int u = t; u < ntile && u < t + IL_STAGES - 1; ++u)
                    mbar_wait_bounded(smem_u32(&full_bar[u % IL_STAGES]), (u / IL_STAGES) & 1, a.spin_limit);
            }
            __syncthreads();
            return;
        }
        if (t + IL_STAGES - 1 < ntile) load_tile(t + IL_STAGES - 1);
        cp_async_commit();
        float* xs = stage0 + (t % IL_STAGES) * st_f;
        float* ys = xs + (st_f - (int)(il_align128((size_t)k * IL_YP * 4) / 4));
        const int64_t r0 = rbeg + (int64_t)t * IL_TC;
        const int nr = (int)(rend - r0 < IL_TC ? rend - r0 : IL_TC);
        if (a.mode >= 0) {
            // X_c . (a or u) - (H rule) Y_:c . s, split in eight parts
            float d = 0.f;
            const float4* xr = reinterpret_cast<const float4*>(xs + c_own * XP);
            const float4* v4 = reinterpret_cast<const float4*>(vec);
            for (int q = part; 4 * q < a.lx; q += 8) {
                const float4 x = xr[q], w = v4[q];
                d = fmaf(x.x, w.x, d);
                d = fmaf(x.y, w.y, d);
                d = fmaf(x.z, w.z, d);
                d = fmaf(x.w, w.w, d);
            }
            if (a.mode == 0)
                for (int i = part; i < k; i += 8) d = fmaf(-ys[i * IL_YP + c_own], vec[IL_MAX + i], d);
            red[part * IL_TC + c_own] = d;
            __syncthreads();
            if (tid < IL_TC) {
                float g = 0.f;
#pragma unroll
                for (int p = 0; p < 8; ++p) g += red[p * IL_TC + tid];
                float* yj = ys + j * IL_YP + tid;
                const float old = *yj;
                float nv = old;
                if (tid >= nr) {
                    nv = 0.f;
                } else if (alive) {
                    if (a.mode == 1)
                        nv = fmaxf(0.f, g);
                    else if (a.reg)
                        nv = fmaxf(0.f, (fmaf(djj, old, g) - a.beta) / (djj + a.alpha));
                    else
                        nv = fmaxf(0.f, old + g / djj);
                    a.Y[(int64_t)j * a.N + r0 + tid] = nv;
                }
                *yj = nv;
            }
            __syncthreads();
        }
        if (nr < IL_TC && a.jn >= 0) {
            // rows past the block's range (zeros, or the next block's rows in a TMA box) add nothing
            if (tid >= nr && tid < IL_TC) ys[a.jn * IL_YP + tid] = 0.f;
            __syncthreads();
        }
        if (a.jn >= 0) {
            // P_i = sum_c X(c, i) y(c), S_i = sum_c Y(i, c) y(c), y = row jn after the update
            const float* y = ys + a.jn * IL_YP;
            const int cb = half * (IL_TC / 2);
            float s = 0.f;
            if (e_own < IL_MAX) {
                if (e_own < a.lx)
#pragma unroll 8
                    for (int c = cb; c < cb + IL_TC / 2; ++c) s = fmaf(xs[c * XP + e_own], y[c], s);
            } else if (e_own - IL_MAX < k) {
                const float4* yr = reinterpret_cast<const float4*>(ys + (e_own - IL_MAX) * IL_YP + cb);
                const float4* y4 = reinterpret_cast<const float4*>(y + cb);
#pragma unroll
                for (int q = 0; q < IL_TC / 8; ++q) {
                    const float4 u = yr[q], w = y4[q];
                    s = fmaf(u.x, w.x, s);
                    s = fmaf(u.y, w.y, s);
                    s = fmaf(u.z, w.z, s);
                    s = fmaf(u.w, w.w, s);
                }
            }
            two_sum_add(acc, s);
        }
    }
    cp_async_wait_0();
    if (a.jn < 0) return;
    // block partial: the two halves in order
    if (half == 1) dred[e_own] = acc;
    __syncthreads();
    if (half == 0) a.partial[(int64_t)blockIdx.x * IL_NE + e_own] = pair_add(acc, dred[e_own]);
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the last block: the block partials added in block order (two halves, then in order)
    const int nb = gridDim.x, hb = (nb + 1) / 2;
    const int bend = (half + 1) * hb < nb ? (half + 1) * hb : nb;
    float2 v = make_float2(0.f, 0.f);
    for (int b0 = half * hb; b0 < bend; b0 += 16) {
        float2 pv[16];  // sixteen loads in flight, added in block order
#pragma unroll
        for (int u = 0; u < 16; ++u)
            pv[u] = b0 + u < bend ? __ldcg(a.partial + (int64_t)(b0 + u) * IL_NE + e_own) : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 16; ++u) v = pair_add(v, pv[u]);
    }
    __syncthreads();
    if (half == 1) dred[e_own] = v;
    __syncthreads();
    float* tot = red;  // [IL_NE] the final sums
    if (half == 0) tot[e_own] = pair_value(pair_add(v, dred[e_own]));
    __syncthreads();
    if (tid == 0) *a.ticket = 0u;
    if (a.mode == 1) {
        // W~_:j = Q^T W_j (a dead column keeps W~_:j); S_:j from W or from W~
        if (tid < a.lx && alive) a.P_out[(int64_t)tid * a.P_stride] = tot[tid];
        if (a.gram_mode == 0) {
            if (tid < k) a.S_out[tid] = tot[IL_MAX + tid];
        } else if (tid < k) {
            float2 sv = make_float2(0.f, 0.f);
            for (int r = 0; r < a.lx; ++r) {
                const float wj = alive ? tot[r] : a.Wt[(int64_t)r * k + j];
                const float wi = tid == j ? wj : a.Wt[(int64_t)r * k + tid];
                const float p = __fmul_rn(wi, wj);  // not contracted into the two-sum
                two_sum_add(sv, p);
                sv.y += fmaf(wi, wj, -p);  // the product's rounding error
            }
            a.S_out[tid] = pair_value(sv);
        }
    } else {
        if (tid < a.lx) a.P_out[(int64_t)tid * a.P_stride] = tot[tid];
        if (tid < k) a.S_out[tid] = tot[IL_MAX + tid];
    }
}

size_t il_smem_bytes(int pitch, int k) {
    return 128 + ((size_t)IL_STAGES * il_stage_floats(pitch, k) + 2 * IL_MAX + 8 * IL_TC) * sizeof(float) +
           IL_NE * sizeof(float2);
}

// 2-D float32 tensor map: `rows` rows of `inner` elements, `pitch` elements apart,
// box `bx` x `by`; out-of-range elements are read as zeros
bool il_map(CUtensorMap* tm, const float* base, int64_t inner, int64_t rows, int64_t pitch, int bx, int by) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    memset(tm, 0, sizeof *tm);
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
    cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by}, estr[2] = {1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool il_launch(rnmf_ctx* ctx, IlPass& a, char* scratch, int cls, double bytes, double flops) {
    const int target = ctx->num_sms;
    int64_t rc = (a.N + target - 1) / target;
    rc = (rc + 3) / 4 * 4;
    if (rc < 4) rc = 4;
    const int nb = (int)((a.N + rc - 1) / rc);
    a.rchunk = rc;
    a.ticket = reinterpret_cast<unsigned*>(scratch);
    a.partial = reinterpret_cast<float2*>(scratch + 256);
    a.status = ctx->d_status;
    a.spin_limit = RNMF_DEFAULT_SPIN_LIMIT;
    // TMA boxes need 16-byte row strides and bases; the Y box's first column r0 is a multiple of 4
    CUtensorMap tmX, tmY;
    memset(&tmX, 0, sizeof tmX);
    memset(&tmY, 0, sizeof tmY);
    a.use_tma = a.pitch % 4 == 0 && a.N % 4 == 0 && (reinterpret_cast<uintptr_t>(a.X) & 15) == 0 &&
                (reinterpret_cast<uintptr_t>(a.Y) & 15) == 0 &&
                il_map(&tmX, a.X, a.pitch, a.N, a.pitch, il_xp(a.pitch), IL_TC) &&
                il_map(&tmY, a.Y, a.N, a.k, a.N, IL_YP, a.k);
    const size_t smem = il_smem_bytes(a.pitch, a.k);
    cudaFuncSetAttribute(il_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prof_begin(ctx);
    il_pass_kernel<<<nb < 1 ? 1 : nb, IL_NT, smem, ctx->stream>>>(tmX, tmY, a);
    return launch_done(ctx, cls, bytes, flops);
}

}  // namespace

size_t il_scratch_bytes(rnmf_ctx* ctx) {
    return 256 + (size_t)(ctx->num_sms > 0 ? ctx->num_sms : 1) * IL_NE * sizeof(float2);
}

bool il_begin(rnmf_ctx* ctx, char* scratch) {
    return cudaMemsetAsync(scratch, 0, 256, ctx->stream) == cudaSuccess;
}

bool launch_il_wpass(rnmf_ctx* ctx, const float* Qp, int64_t m, int l, int lp, int k, int j, float* Wc, float* Wt,
                     const float* T_row, const float* V_row, const float* q1, float alpha, float beta, int gram_mode,
                     float* S_row_out, char* scratch) {
    IlPass a{};
    a.X = Qp; a.pitch = lp; a.lx = l;
    a.Y = Wc; a.N = m; a.k = k;
    a.mode = 1; a.j = j; a.jn = j;
    a.Wt = Wt; a.T_row = T_row; a.V_row = V_row; a.q1 = q1;
    a.reg = (alpha != 0.f || beta != 0.f) ? 1 : 0; a.alpha = alpha; a.beta = beta;
    a.gram_mode = gram_mode;
    a.P_out = Wt + j; a.P_stride = k; a.S_out = S_row_out;
    return il_launch(ctx, a, scratch, K_IL_PASS, 4.0 * m * (lp + k + 1), 2.0 * m * (2.0 * l + k));
}

bool launch_il_hpass(rnmf_ctx* ctx, const float* Bt, int64_t n, int l, int k, int j, int jn, float* H,
                     const float* Wt, const float* S_row, float alpha, float beta, float* T_out, float* V_out,
                     char* scratch) {
    IlPass a{};
    a.X = Bt; a.pitch = l; a.lx = l;
    a.Y = H; a.N = n; a.k = k;
    a.mode = j >= 0 ? 0 : -1; a.j = j; a.jn = jn;
    a.Wt = Wt; a.S_row = S_row;
    a.reg = (alpha != 0.f || beta != 0.f) ? 1 : 0; a.alpha = alpha; a.beta = beta;
    a.P_out = T_out; a.P_stride = 1; a.S_out = V_out;
    return il_launch(ctx, a, scratch, K_IL_PASS, 4.0 * n * (l + k + 1), 2.0 * n * 2.0 * (l + k));
}
