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
//     each).  The j loop runs in chunks of 8: the contribution of the entries
//     outside the chunk is summed first (one shared-memory read of x_i feeds 8
//     FMAs), then the 8 sequential steps run in registers.
//
// (2) whalf: the W half of a randomized sweep (Section 3.2 W~ rule and
//     reprojection; Algorithm 1), Gauss-Seidel over columns j:
//       u   = W~_j + (T_:j - W~ V_:j) / V_jj      (l-vector, every block)
//       W_j = max(0, Q u)                         (row-local)
//       W~_j = Q^T W_j                            (sum over all m rows)
//     One persistent block per SM owns a slice of rows; the sum over rows is a
//     fixed-order reduction of per-block partials behind a grid barrier whose
//     wait is bounded (RNMF_ETIMEOUT instead of a hang).
#include "rnmf_internal.cuh"
#include "sync.cuh"

namespace {

constexpr int ROWS_NT = 128;
constexpr int CH = 8;

__global__ void __launch_bounds__(ROWS_NT) hals_rows_kernel(float* __restrict__ X, int64_t sv, int64_t se,
                                                            const float* __restrict__ Rhs, int64_t srv,
                                                            int64_t srj, const float* __restrict__ S,
                                                            int64_t count, int k) {
    extern __shared__ __align__(16) float sm[];
    const int kp = (k + CH - 1) / CH * CH;
    float* Ss = sm;                 // kp x kp, zero padded
    float* xs = sm + kp * kp;       // kp x ROWS_NT: x_i of thread t at xs[i*ROWS_NT + t]
    const int t = threadIdx.x;
    for (int e = t; e < kp * kp; e += ROWS_NT) {
        int i = e / kp, j = e % kp;
        Ss[e] = (i < k && j < k) ? S[i * k + j] : 0.f;
    }
    const int64_t v = (int64_t)blockIdx.x * ROWS_NT + t;
    const bool valid = v < count;
    for (int i = 0; i < kp; ++i) xs[i * ROWS_NT + t] = (valid && i < k) ? X[v * sv + (int64_t)i * se] : 0.f;
    __syncthreads();
    if (valid) {
        for (int j0 = 0; j0 < k; j0 += CH) {
            float g[CH];
#pragma unroll
            for (int jj = 0; jj < CH; ++jj) g[jj] = (j0 + jj < k) ? Rhs[v * srv + (int64_t)(j0 + jj) * srj] : 0.f;
            // entries outside the chunk (already final for i < j0, old for i >= j0 + CH)
            for (int i = 0; i < kp; ++i) {
                if (i == j0) {
                    i += CH - 1;
                    continue;
                }
                const float xi = xs[i * ROWS_NT + t];
                const float4 s0 = *reinterpret_cast<const float4*>(&Ss[i * kp + j0]);
                const float4 s1 = *reinterpret_cast<const float4*>(&Ss[i * kp + j0 + 4]);
                g[0] = fmaf(-xi, s0.x, g[0]);
                g[1] = fmaf(-xi, s0.y, g[1]);
                g[2] = fmaf(-xi, s0.z, g[2]);
                g[3] = fmaf(-xi, s0.w, g[3]);
                g[4] = fmaf(-xi, s1.x, g[4]);
                g[5] = fmaf(-xi, s1.y, g[5]);
                g[6] = fmaf(-xi, s1.z, g[6]);
                g[7] = fmaf(-xi, s1.w, g[7]);
            }
            float xc[CH];
#pragma unroll
            for (int jj = 0; jj < CH; ++jj) xc[jj] = xs[(j0 + jj) * ROWS_NT + t];
#pragma unroll
            for (int jj = 0; jj < CH; ++jj) {
                if (j0 + jj < k) {
                    const float sjj = Ss[(j0 + jj) * kp + j0 + jj];
                    float val = g[jj];
#pragma unroll
                    for (int ii = 0; ii < CH; ++ii) val = fmaf(-xc[ii], Ss[(j0 + ii) * kp + j0 + jj], val);
                    if (sjj > 0.f) xc[jj] = fmaxf(0.f, xc[jj] + val / sjj);
                }
            }
#pragma unroll
            for (int jj = 0; jj < CH; ++jj) xs[(j0 + jj) * ROWS_NT + t] = xc[jj];
        }
        for (int i = 0; i < k; ++i) X[v * sv + (int64_t)i * se] = xs[i * ROWS_NT + t];
    }
}

constexpr int WH_NT = 512;
constexpr int WH_WARPS = WH_NT / 32;
constexpr int LP = 128;  // padded l

struct WhalfSmem {
    // offsets in floats
    static __host__ __device__ size_t bytes(int l, int k) {
        return ((size_t)l * k * 2 + (size_t)k * k + LP + (size_t)WH_WARPS * LP) * sizeof(float);
    }
};

__global__ void __launch_bounds__(WH_NT, 1) whalf_kernel(const float* __restrict__ Q, int64_t m, int l, int k,
                                                         float* __restrict__ Wc, float* __restrict__ Wt_g,
                                                         const float* __restrict__ T_g,
                                                         const float* __restrict__ V_g, float* part,
                                                         unsigned* bar, int* status, long long spin_limit) {
    extern __shared__ __align__(16) float sm[];
    float* Wt = sm;                     // l x k
    float* T = Wt + l * k;              // l x k
    float* V = T + l * k;               // k x k
    float* u = V + k * k;               // LP
    float* red = u + LP;                // WH_WARPS x LP
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    for (int e = tid; e < l * k; e += WH_NT) {
        Wt[e] = Wt_g[e];
        T[e] = T_g[e];
    }
    for (int e = tid; e < k * k; e += WH_NT) V[e] = V_g[e];
    const int64_t rpb = (m + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
    __syncthreads();
    unsigned nbar = 0;
    // thread -> (t = tid / 4, quarter q = tid % 4) for the l-vector reductions
    const int rt = tid >> 2, rq = tid & 3;
    for (int j = 0; j < k; ++j) {
        const float vjj = V[j * k + j];
        if (!(vjj > 0.f)) continue;  // dead component: column left unchanged (uniform over blocks)
        // u = W~_j + (T_:j - W~ V_:j) / V_jj
        {
            float s = 0.f;
            if (rt < l)
                for (int i = rq; i < k; i += 4) s = fmaf(Wt[rt * k + i], V[i * k + j], s);
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            if (rt < l && rq == 0) u[rt] = Wt[rt * k + j] + (T[rt * k + j] - s) / vjj;
        }
        __syncthreads();
        float uu[4], p[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int tt = lane + 32 * c;
            uu[c] = tt < l ? u[tt] : 0.f;
            p[c] = 0.f;
        }
        for (int64_t r = r0 + warp; r < r1; r += WH_WARPS) {
            const float* qr = Q + r * l;
            float q[4];
            float d = 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int tt = lane + 32 * c;
                q[c] = tt < l ? __ldg(qr + tt) : 0.f;
                d = fmaf(q[c], uu[c], d);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            const float w = fmaxf(0.f, d);
            if (lane == 0) Wc[(int64_t)j * m + r] = w;
#pragma unroll
            for (int c = 0; c < 4; ++c) p[c] = fmaf(w, q[c], p[c]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) red[warp * LP + lane + 32 * c] = p[c];
        __syncthreads();
        float* pj = part + ((size_t)(nbar & 1) * gridDim.x + blockIdx.x) * LP;
        {
            float s = 0.f;
            if (rt < l)
                for (int w = rq; w < WH_WARPS; w += 4) s += red[w * LP + rt];
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            if (rt < l && rq == 0) pj[rt] = s;
        }
        ++nbar;
        if (!rnmf_grid_barrier(bar, nbar * gridDim.x, status, spin_limit)) return;
        // W~_j = sum over blocks, fixed order, float64
        {
            const float* pb = part + (size_t)((nbar - 1) & 1) * gridDim.x * LP;
            double s = 0.0;
            if (rt < l)
                for (int b = rq; b < (int)gridDim.x; b += 4) s += (double)__ldcg(pb + (size_t)b * LP + rt);
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            if (rt < l && rq == 0) Wt[rt * k + j] = (float)s;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0)
        for (int e = tid; e < l * k; e += WH_NT) Wt_g[e] = Wt[e];
}

int whalf_grid(rnmf_ctx* ctx, int64_t m, int l, int k) {
    size_t smem = WhalfSmem::bytes(l, k);
    int occ = 0;
    cudaFuncSetAttribute(whalf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, whalf_kernel, WH_NT, smem);
    if (occ < 1) occ = 1;
    int64_t g = (int64_t)ctx->num_sms * occ;
    int64_t byrows = (m + 31) / 32;
    if (g > byrows) g = byrows;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

bool launch_hals_rows(rnmf_ctx* ctx, float* X, int64_t sv, int64_t se, const float* Rhs, int64_t srv, int64_t srj,
                      const float* S, int64_t count, int k) {
    if (count <= 0) return true;
    const int kp = (k + CH - 1) / CH * CH;
    size_t smem = ((size_t)kp * kp + (size_t)kp * ROWS_NT) * sizeof(float);
    cudaFuncSetAttribute(hals_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    unsigned grid = (unsigned)((count + ROWS_NT - 1) / ROWS_NT);
    prof_begin(ctx);
    hals_rows_kernel<<<grid, ROWS_NT, smem, ctx->stream>>>(X, sv, se, Rhs, srv, srj, S, count, k);
    return launch_done(ctx, K_HALS_ROWS, 12.0 * count * k + 4.0 * k * k, 2.0 * count * k * k);
}

size_t whalf_scratch_bytes(rnmf_ctx* ctx, int64_t m, int l, int k) {
    return (size_t)2 * whalf_grid(ctx, m, l, k) * LP * sizeof(float);
}

bool launch_whalf(rnmf_ctx* ctx, const float* Q, int64_t m, int l, int k, float* Wc, float* Wt, const float* T,
                  const float* V, char* scratch, long long spin_limit) {
    int grid = whalf_grid(ctx, m, l, k);
    size_t smem = WhalfSmem::bytes(l, k);
    if (cudaMemsetAsync(ctx->d_bar, 0, sizeof(unsigned), ctx->stream) != cudaSuccess) return false;
    prof_begin(ctx);
    whalf_kernel<<<grid, WH_NT, smem, ctx->stream>>>(Q, m, l, k, Wc, Wt, T, V, reinterpret_cast<float*>(scratch),
                                                      ctx->d_bar, ctx->d_status,
                                                      spin_limit > 0 ? spin_limit : RNMF_DEFAULT_SPIN_LIMIT);
    // compulsory traffic: Q once, W written once; flops: Q u and Q^T w for each column
    return launch_done(ctx, K_WHALF, 4.0 * m * l + 4.0 * m * k, 4.0 * m * l * k);
}
