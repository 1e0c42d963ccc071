// adjoint.cu - reverse mode through T compressed HALS sweeps (Algorithm 1 loop,
// Section 3.2 update rules) for L = <G, W_T H_T>, with per-sweep checkpoints.
//
// Forward sweep t maps (W_{t-1}, W~_{t-1}, H_{t-1}) to (W_t, W~_t, H_t):
//   H half: R = B^T W~_{t-1}, S = W_{t-1}^T W_{t-1} (or W~^T W~);
//           a_j = (R_:j - sum_{i != j} S_ij x_i) / S_jj, x_j <- max(0, a_j)
//           (the own term x_j cancels in x_j + (R_:j - H^T S_:j)/S_jj);
//   W half: T = B H_t^T, V = H_t H_t^T;
//           u_j = (T_:j - sum_{i != j} W~_i V_ij) / V_jj, W_j = max(0, Q u_j),
//           W~_j = Q^T W_j.
// Reverse of a step j, given the adjoint of its output:
//   H: da = [x_j > 0] dx_j, dR_cj = da / S_jj, dx_i -= dR_cj S_ij (i != j),
//      dS_ij -= dR_cj x_i (i != j), dS_jj -= dR_cj x_j;
//   W: dz = [W_j > 0] (dW_j + Q dW~_j), du = Q^T dz (a grid-wide sum),
//      dT_:j = du / V_jj, dW~_i -= du V_ij / V_jj (i != j),
//      dV_ij -= (du . W~_i) / V_jj (i != j), dV_jj -= (du . u_j) / V_jj.
// Every value a reverse step needs is recomputed from the checkpointed states
// before and after the sweep (masks from the outputs, x_i from the input or
// output state), so a sweep's tape is its two boundary states.
#include "rnmf_internal.cuh"
#include "sync.cuh"

namespace {

constexpr int HR_NT = 64;
constexpr int WR_NT = 256;
constexpr int WR_WARPS = WR_NT / 32;
constexpr int LPA = 128;

// H-half reverse: one thread per column c of H.
//   Ho = H_{t-1}, Hn = H_t, dHn = dL/dH_t (k x n); S (k x k).
//   dHo = dL/dH_{t-1} (k x n); DA (n x k) = dL/dR.
__global__ void __launch_bounds__(HR_NT) hrev_kernel(const float* __restrict__ Ho, const float* __restrict__ Hn,
                                                      const float* __restrict__ dHn, const float* __restrict__ S,
                                                      int64_t n, int k, float* __restrict__ dHo,
                                                      float* __restrict__ DA) {
    extern __shared__ float sm[];
    float* Ss = sm;                         // k x k
    float* xs = Ss + k * k;                 // [4][k][HR_NT]: xo, xn, gn, go
    const int t = threadIdx.x;
    auto X = [&](int a, int i) -> float& { return xs[((size_t)a * k + i) * HR_NT + t]; };
    for (int e = t; e < k * k; e += HR_NT) Ss[e] = S[e];
    const int64_t c = (int64_t)blockIdx.x * HR_NT + t;
    const bool valid = c < n;
    for (int i = 0; i < k; ++i) {
        X(0, i) = valid ? Ho[(int64_t)i * n + c] : 0.f;
        X(1, i) = valid ? Hn[(int64_t)i * n + c] : 0.f;
        X(2, i) = valid ? dHn[(int64_t)i * n + c] : 0.f;
        X(3, i) = 0.f;
    }
    __syncthreads();
    if (!valid) return;
    for (int j = k - 1; j >= 0; --j) {
        const float sjj = Ss[j * k + j];
        const float g = X(2, j);
        if (!(sjj > 0.f)) {  // skipped step: x_j passes through
            X(3, j) += g;
            DA[c * k + j] = 0.f;
            continue;
        }
        const float da = X(1, j) > 0.f ? g : 0.f;
        const float f = da / sjj;
        DA[c * k + j] = f;
        if (f != 0.f) {
            for (int i = 0; i < j; ++i) X(2, i) = fmaf(-f, Ss[i * k + j], X(2, i));
            for (int i = j + 1; i < k; ++i) X(3, i) = fmaf(-f, Ss[i * k + j], X(3, i));
        }
    }
    for (int i = 0; i < k; ++i) dHo[(int64_t)i * n + c] = X(3, i);
}

// W-half reverse: persistent, one grid-wide reduction per column (reverse order).
//   Q (m x l), Wn = W~_t, Wo = W~_{t-1} (l x k), Wct = W_t^T (k x m, masks),
//   dWct = dL/dW_t stored transposed (k x m), dWn = dL/dW~_t (l x k), T (l x k), V (k x k).
// Outputs: dT (l x k), dV (k x k), dWo = the W-half's part of dL/dW~_{t-1} (l x k),
//   dWpass (k x m): dL/dW_{t-1} passed through skipped columns (zero elsewhere).
__global__ void __launch_bounds__(WR_NT, 1) wrev_kernel(const float* __restrict__ Q, int64_t m, int l, int k,
                                                        const float* __restrict__ Wn_g, const float* __restrict__ Wo_g,
                                                        const float* __restrict__ Wct, const float* __restrict__ dWct,
                                                        const float* __restrict__ dWn_g, const float* __restrict__ T_g,
                                                        const float* __restrict__ V_g, float* __restrict__ dT_g,
                                                        float* __restrict__ dV_g, float* __restrict__ dWo_g,
                                                        float* __restrict__ dWpass, float* part, unsigned* bar,
                                                        int* status, long long spin_limit) {
    extern __shared__ __align__(16) float sm[];
    const int lk = l * k;
    float* sWn = sm;
    float* sWo = sWn + lk;
    float* sdWn = sWo + lk;
    float* sdWo = sdWn + lk;
    float* sT = sdWo + lk;
    float* sV = sT + lk;                 // k x k
    float* sdV = sV + k * k;             // k x k
    float* u = sdV + k * k;              // LPA
    float* gv = u + LPA;                 // LPA
    float* du = gv + LPA;                // LPA
    float* red = du + LPA;               // WR_WARPS x LPA
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int rt = tid >> 1, rq = tid & 1;
    for (int e = tid; e < lk; e += WR_NT) {
        sWn[e] = Wn_g[e];
        sWo[e] = Wo_g[e];
        sdWn[e] = dWn_g[e];
        sdWo[e] = 0.f;
        sT[e] = T_g[e];
    }
    for (int e = tid; e < k * k; e += WR_NT) {
        sV[e] = V_g[e];
        sdV[e] = 0.f;
    }
    const int64_t rpb = (m + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
    __syncthreads();
    unsigned nbar = 0;
    for (int j = k - 1; j >= 0; --j) {
        const float vjj = sV[j * k + j];
        if (!(vjj > 0.f)) {  // skipped column: W~_j and W_j pass through
            if (rt < l && rq == 0) sdWo[rt * k + j] += sdWn[rt * k + j];
            for (int64_t r = r0 + tid; r < r1; r += WR_NT) dWpass[(int64_t)j * m + r] = dWct[(int64_t)j * m + r];
            __syncthreads();
            continue;
        }
        {
            float s = 0.f;
            if (rt < l)
                for (int i = rq; i < k; i += 2)
                    if (i != j) s = fmaf(i < j ? sWn[rt * k + i] : sWo[rt * k + i], sV[i * k + j], s);
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            if (rt < l && rq == 0) {
                u[rt] = (sT[rt * k + j] - s) / vjj;
                gv[rt] = sdWn[rt * k + j];
            }
        }
        __syncthreads();
        float p[4] = {0.f, 0.f, 0.f, 0.f}, g[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) g[c] = (lane + 32 * c) < l ? gv[lane + 32 * c] : 0.f;
        for (int64_t r = r0 + warp; r < r1; r += WR_WARPS) {
            float q[4], d = 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int tt = lane + 32 * c;
                q[c] = tt < l ? Q[r * l + tt] : 0.f;
                d = fmaf(q[c], g[c], d);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            const bool on = Wct[(int64_t)j * m + r] > 0.f;
            const float dz = on ? dWct[(int64_t)j * m + r] + d : 0.f;
            if (lane == 0) dWpass[(int64_t)j * m + r] = 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) p[c] = fmaf(dz, q[c], p[c]);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) red[warp * LPA + lane + 32 * c] = p[c];
        __syncthreads();
        float* pj = part + ((size_t)(nbar & 1) * gridDim.x + blockIdx.x) * LPA;
        {
            float s = 0.f;
            if (rt < l)
                for (int w = rq; w < WR_WARPS; w += 2) s += red[w * LPA + rt];
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            if (rt < l && rq == 0) pj[rt] = s;
        }
        ++nbar;
        if (!rnmf_grid_barrier(bar, nbar * gridDim.x, status, spin_limit)) return;
        if (rt < l && rq == 0) {
            const float* pb = part + (size_t)((nbar - 1) & 1) * gridDim.x * LPA;
            float s = 0.f;
            for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(pb + (size_t)b * LPA + rt);
            du[rt] = s;
        }
        __syncthreads();
        // dT_:j, dW~ (columns i != j), dV (column j)
        if (rt < l) {
            const float dut = du[rt];
            if (rq == 0 && blockIdx.x == 0) dT_g[rt * k + j] = dut / vjj;
            for (int i = rq; i < k; i += 2) {
                if (i == j) continue;
                const float coef = sV[i * k + j] / vjj;
                if (i < j)
                    sdWn[rt * k + i] = fmaf(-coef, dut, sdWn[rt * k + i]);
                else
                    sdWo[rt * k + i] = fmaf(-coef, dut, sdWo[rt * k + i]);
            }
        }
        if (tid < k) {
            const int i = tid;
            float d = 0.f;
            if (i == j) {
                for (int t2 = 0; t2 < l; ++t2) d = fmaf(du[t2], u[t2], d);
            } else {
                const float* src = i < j ? sWn : sWo;
                for (int t2 = 0; t2 < l; ++t2) d = fmaf(du[t2], src[t2 * k + i], d);
            }
            sdV[i * k + j] -= d / vjj;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0) {
        for (int e = tid; e < lk; e += WR_NT) dWo_g[e] = sdWo[e];
        for (int e = tid; e < k * k; e += WR_NT) dV_g[e] = sdV[e];
        // columns j that were skipped never wrote dT
        for (int j = 0; j < k; ++j)
            if (!(sV[j * k + j] > 0.f))
                for (int t2 = tid; t2 < l; t2 += WR_NT) dT_g[t2 * k + j] = 0.f;
    }
}

// dSym[i][j] = D(i, j) + D(j, i) with D(i, j) = -(i <= j ? P1T[j][i] : P0T[j][i]); when
// P0T == NULL: D(i, j) = P1T[i][j] (plain symmetrisation).
__global__ void sym_kernel(const float* __restrict__ P1T, const float* __restrict__ P0T, int k, float* __restrict__ out) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
        const int i = e / k, j = e % k;
        float a, b;
        if (P0T) {
            a = -(i <= j ? P1T[j * k + i] : P0T[j * k + i]);
            b = -(j <= i ? P1T[i * k + j] : P0T[i * k + j]);
        } else {
            a = P1T[i * k + j];
            b = P1T[j * k + i];
        }
        out[e] = a + b;
    }
}

// dA (m x n) = Q (m x l) dBt^T (l x n): 64 x 64 output tiles, contraction l <= 128.
__global__ void __launch_bounds__(256) outer_kernel(const float* __restrict__ Q, const float* __restrict__ dBt,
                                                    int64_t m, int64_t n, int l, float* __restrict__ dA) {
    __shared__ float Qs[32][65], Bs[32][65];
    const int64_t i0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[4][4] = {};
    for (int t0 = 0; t0 < l; t0 += 32) {
        for (int e = threadIdx.x; e < 32 * 64; e += 256) {
            const int r = e / 32, t = e % 32;
            Qs[t][r] = (i0 + r < m && t0 + t < l) ? Q[(i0 + r) * l + t0 + t] : 0.f;
            Bs[t][r] = (c0 + r < n && t0 + t < l) ? dBt[(c0 + r) * l + t0 + t] : 0.f;
        }
        __syncthreads();
        for (int t = 0; t < 32; ++t)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(Qs[t][ty * 4 + a], Bs[t][tx * 4 + b], acc[a][b]);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t i = i0 + ty * 4 + a, c = c0 + tx * 4 + b;
            if (i < m && c < n) dA[i * n + c] = acc[a][b];
        }
}

int wrev_grid(rnmf_ctx* ctx, int64_t m) {
    int64_t g = (m + 31) / 32;
    if (g > ctx->num_sms) g = ctx->num_sms;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

size_t adjoint_ckpt_floats(int64_t m, int64_t n, int l, int k) {
    return (size_t)k * m + (size_t)l * k + (size_t)k * n;
}

size_t wrev_scratch_bytes(rnmf_ctx* ctx, int64_t m) { return (size_t)2 * wrev_grid(ctx, m) * LPA * sizeof(float); }

bool launch_hrev(rnmf_ctx* ctx, const float* Ho, const float* Hn, const float* dHn, const float* S, int64_t n, int k,
                 float* dHo, float* DA) {
    const size_t smem = ((size_t)k * k + (size_t)4 * k * HR_NT) * sizeof(float);
    cudaFuncSetAttribute(hrev_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prof_begin(ctx);
    hrev_kernel<<<(unsigned)((n + HR_NT - 1) / HR_NT), HR_NT, smem, ctx->stream>>>(Ho, Hn, dHn, S, n, k, dHo, DA);
    return launch_done(ctx, K_ADJOINT, 16.0 * n * k, 2.0 * n * k * k);
}

bool launch_wrev(rnmf_ctx* ctx, const float* Q, int64_t m, int l, int k, const float* Wn, const float* Wo,
                 const float* Wct, const float* dWct, const float* dWn, const float* T, const float* V, float* dT,
                 float* dV, float* dWo, float* dWpass, char* scratch, long long spin_limit) {
    const int grid = wrev_grid(ctx, m);
    const size_t smem = ((size_t)5 * l * k + (size_t)2 * k * k + (size_t)(3 + WR_WARPS) * LPA) * sizeof(float);
    cudaFuncSetAttribute(wrev_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaMemsetAsync(ctx->d_bar, 0, sizeof(unsigned), ctx->stream) != cudaSuccess) return false;
    prof_begin(ctx);
    // blocks meet at a grid barrier: a cooperative launch
    if (!launch_cooperative(ctx, wrev_kernel, (unsigned)grid, WR_NT, smem, Q, m, l, k, Wn, Wo, Wct, dWct, dWn, T, V, dT,
                            dV, dWo, dWpass, reinterpret_cast<float*>(scratch), ctx->d_bar, ctx->d_status,
                            spin_limit > 0 ? spin_limit : RNMF_DEFAULT_SPIN_LIMIT))
        return false;
    return launch_done(ctx, K_ADJOINT, 4.0 * m * l + 12.0 * m * k, 4.0 * m * l * k);
}

bool launch_sym(rnmf_ctx* ctx, const float* P1T, const float* P0T, int k, float* out) {
    prof_begin(ctx);
    sym_kernel<<<(k * k + 255) / 256, 256, 0, ctx->stream>>>(P1T, P0T, k, out);
    return launch_done(ctx, K_ADJOINT, 12.0 * k * k, 0);
}

bool launch_outer(rnmf_ctx* ctx, const float* Q, const float* dBt, int64_t m, int64_t n, int l, float* dA) {
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)((m + 63) / 64));
    prof_begin(ctx);
    outer_kernel<<<grid, 256, 0, ctx->stream>>>(Q, dBt, m, n, l, dA);
    return launch_done(ctx, K_ADJOINT, 4.0 * ((double)m * n + (double)(m + n) * l), 2.0 * m * n * l);
}
