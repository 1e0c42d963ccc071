// init_svd.cu - SVD-based initial factors from the randomized QB (the
// initialisation remark after Algorithm 1 and Section 4: NNDSVD of the
// randomized SVD A ~ Q B = (Q U_B) diag(s) V^T).
//
//   G = B B^T (l x l, float64, error-free Gram of B^T)
//   G = U_B diag(s^2) U_B^T         cyclic Jacobi in one block (float64)
//   U = Q U_B(:, :k), V = B^T U_B(:, :k) diag(1/s)      (float32 products)
//   NNDSVD per component j: |u_1|, |v_1| for j = 0; else the larger of the
//   (positive, negative) part pairs by |u.| |v.|, scaled by sqrt(s_j m).
// U and V are computed in the storage of W (transposed, k x m) and H (k x n)
// and turned into the factors in place.
#include "rnmf_internal.cuh"

namespace {

constexpr int JT = 256;          // threads of the Jacobi block
constexpr int MAX_SWEEPS = 30;

// Cyclic Jacobi with the round-robin (tournament) ordering: each step rotates
// L/2 disjoint pairs (p, q) at once (A <- J^T A J, J = [[c, s], [-s, c]] on
// rows/columns p, q, with (c, s) zeroing A_pq: tau = (A_qq - A_pp) / (2 A_pq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c).
// Sweeps stop when the off-diagonal mass is below 1e-28 of the total (or after
// MAX_SWEEPS).  Eigenpairs are returned in descending order of eigenvalue
// (ties by index): evals[r], evecs column r (row-major l x l).
__global__ void __launch_bounds__(JT) jacobi_eig_kernel(const double* __restrict__ G, int l, double* __restrict__ evals,
                                                        double* __restrict__ evecs, double* __restrict__ V) {
    extern __shared__ double jsm[];
    const int L = l + (l & 1);
    const int P = L + 1;  // row pitch
    double* A = jsm;                      // [L][P]
    double* cs = A + L * P;               // [L/2]
    double* sn = cs + L / 2;              // [L/2]
    double* red = sn + L / 2;             // [JT]
    int* top = reinterpret_cast<int*>(red + JT);
    int* bot = top + L / 2;
    const int tid = threadIdx.x;
    for (int e = tid; e < L * L; e += JT) {
        const int i = e / L, j = e % L;
        A[i * P + j] = (i < l && j < l) ? G[i * l + j] : 0.0;
        V[e] = i == j ? 1.0 : 0.0;  // V stored by columns: V(i, p) at V[p L + i]
    }
    for (int t = tid; t < L / 2; t += JT) {
        top[t] = 2 * t;
        bot[t] = 2 * t + 1;
    }
    __syncthreads();
    for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
        // off-diagonal and total mass (fixed-order tree: the same decision in every run)
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < L * L; e += JT) {
            const double a = A[(e / L) * P + e % L];
            tot += a * a;
            if (e / L != e % L) off += a * a;
        }
        red[tid] = off;
        __syncthreads();
        for (int o = JT / 2; o > 0; o >>= 1) {
            if (tid < o) red[tid] += red[tid + o];
            __syncthreads();
        }
        off = red[0];
        __syncthreads();
        red[tid] = tot;
        __syncthreads();
        for (int o = JT / 2; o > 0; o >>= 1) {
            if (tid < o) red[tid] += red[tid + o];
            __syncthreads();
        }
        tot = red[0];
        __syncthreads();
        if (!(off > 1e-28 * tot)) break;
        for (int step = 0; step < L - 1; ++step) {
            for (int t = tid; t < L / 2; t += JT) {
                const int p = top[t], q = bot[t];
                const double apq = A[p * P + q];
                double c = 1.0, s = 0.0;
                if (apq != 0.0) {
                    const double tau = (A[q * P + q] - A[p * P + p]) / (2.0 * apq);
                    const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + tt * tt);
                    s = tt * c;
                }
                cs[t] = c;
                sn[t] = s;
            }
            __syncthreads();
            // rows p, q of every pair
            for (int e = tid; e < (L / 2) * L; e += JT) {
                const int t = e / L, j = e % L;
                const int p = top[t], q = bot[t];
                const double a = A[p * P + j], b = A[q * P + j];
                A[p * P + j] = cs[t] * a - sn[t] * b;
                A[q * P + j] = sn[t] * a + cs[t] * b;
            }
            __syncthreads();
            // columns p, q of every pair, and of V
            for (int e = tid; e < (L / 2) * L; e += JT) {
                const int t = e / L, i = e % L;
                const int p = top[t], q = bot[t];
                const double a = A[i * P + p], b = A[i * P + q];
                A[i * P + p] = cs[t] * a - sn[t] * b;
                A[i * P + q] = sn[t] * a + cs[t] * b;
                const double va = V[(size_t)p * L + i], vb = V[(size_t)q * L + i];
                V[(size_t)p * L + i] = cs[t] * va - sn[t] * vb;
                V[(size_t)q * L + i] = sn[t] * va + cs[t] * vb;
            }
            __syncthreads();
            // next pairing: top[0] stays, the others move one place round the table
            if (tid == 0 && L > 2) {
                const int h = L / 2;
                const int tlast = top[h - 1], b0 = bot[0];
                for (int t = h - 1; t >= 2; --t) top[t] = top[t - 1];
                top[1] = b0;
                for (int t = 0; t < h - 1; ++t) bot[t] = bot[t + 1];
                bot[h - 1] = tlast;
            }
            __syncthreads();
        }
    }
    // descending order, ties by index (eigen-index i < l only)
    for (int i = tid; i < l; i += JT) {
        const double li = A[i * P + i];
        int r = 0;
        for (int j = 0; j < l; ++j) {
            const double lj = A[j * P + j];
            r += (lj > li || (lj == li && j < i)) ? 1 : 0;
        }
        evals[r] = li;
        for (int row = 0; row < l; ++row) evecs[row * l + r] = V[(size_t)i * L + row];
    }
}

// U_B(:, j) and U_B(:, j) / s_j for j < k as float32 l x k (row-major), s_j = sqrt(max(lambda_j, 0)).
__global__ void ub_kernel(const double* __restrict__ evals, const double* __restrict__ evecs, int l, int k,
                          float* __restrict__ ub, float* __restrict__ ubs, double* __restrict__ sv) {
    for (int e = threadIdx.x; e < l * k; e += blockDim.x) {
        const int i = e / k, j = e % k;
        const double s = sqrt(fmax(evals[j], 0.0));
        ub[e] = (float)evecs[i * l + j];
        ubs[e] = s > 0.0 ? (float)(evecs[i * l + j] / s) : 0.f;
        if (i == 0) sv[j] = s;
    }
}

// Per component j: |x+|^2, |x-|^2 of row j of X (len entries), fixed-order tree.
__global__ void __launch_bounds__(256) part_norms_kernel(const float* __restrict__ X, int64_t len,
                                                         double* __restrict__ out /* [k][2] */) {
    __shared__ double rp[256], rn[256];
    const int j = blockIdx.x;
    double p = 0.0, q = 0.0;
    for (int64_t c = threadIdx.x; c < len; c += 256) {
        const double v = X[(int64_t)j * len + c];
        if (v > 0.0) p += v * v;
        else q += v * v;
    }
    rp[threadIdx.x] = p;
    rn[threadIdx.x] = q;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            rp[threadIdx.x] += rp[threadIdx.x + o];
            rn[threadIdx.x] += rn[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * j] = rp[0];
        out[2 * j + 1] = rn[0];
    }
}

// Row j of X (U^T or V^T storage) -> the NNDSVD factor row in place.
__global__ void __launch_bounds__(256) nndsvd_apply_kernel(float* __restrict__ X, int64_t len, int which,
                                                           const double* __restrict__ un /* [k][2] */,
                                                           const double* __restrict__ vn, const double* __restrict__ sv,
                                                           int k) {
    const int j = blockIdx.y;
    const double s = sv[j];
    const double upn = sqrt(un[2 * j]), unn = sqrt(un[2 * j + 1]);
    const double vpn = sqrt(vn[2 * j]), vnn = sqrt(vn[2 * j + 1]);
    double scale;
    int sign;  // +1: positive part, -1: negative part, 0: |x|
    if (j == 0) {
        scale = sqrt(s);
        sign = 0;
    } else {
        const double mp = upn * vpn, mn = unn * vnn;
        const bool pos = mp > mn;
        const double mm = pos ? mp : mn;
        const double own = which == 0 ? (pos ? upn : unn) : (pos ? vpn : vnn);
        scale = own > 0.0 ? sqrt(s * mm) / own : 0.0;
        sign = pos ? 1 : -1;
    }
    float* row = X + (int64_t)j * len;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < len; c += (int64_t)gridDim.x * blockDim.x) {
        const float v = row[c];
        const float part = sign == 0 ? fabsf(v) : (sign > 0 ? fmaxf(v, 0.f) : fmaxf(-v, 0.f));
        row[c] = (float)(scale * (double)part);
    }
    (void)k;
}

}  // namespace

size_t svd_init_bytes(int l, int k) {
    const int L = l + (l & 1);
    return 3 * arena_round((size_t)l * l * 8) + arena_round((size_t)L * L * 8) + arena_round((size_t)l * 8) +
           2 * arena_round((size_t)l * k * 4) + 3 * arena_round((size_t)k * 2 * 8) + arena_round((size_t)k * 8);
}

// W (transposed, Wc k x m) and H (k x n) from Q (m x l) and B^T (n x l).
bool launch_svd_init(rnmf_ctx* ctx, const float* Q, const float* Bt, int64_t m, int64_t n, int l, int k, float* Wc,
                     float* H, double* gram_scratch) {
    const int L = l + (l & 1);
    double* G = (double*)arena_take(ctx, (size_t)l * l * 8);
    double* evecs = (double*)arena_take(ctx, (size_t)l * l * 8);
    (void)arena_take(ctx, (size_t)l * l * 8);
    double* V = (double*)arena_take(ctx, (size_t)L * L * 8);
    double* evals = (double*)arena_take(ctx, (size_t)l * 8);
    float* ub = (float*)arena_take(ctx, (size_t)l * k * 4);
    float* ubs = (float*)arena_take(ctx, (size_t)l * k * 4);
    double* un = (double*)arena_take(ctx, (size_t)k * 2 * 8);
    double* vn = (double*)arena_take(ctx, (size_t)k * 2 * 8);
    (void)arena_take(ctx, (size_t)k * 2 * 8);
    double* sv = (double*)arena_take(ctx, (size_t)k * 8);
    // G = B B^T = (B^T)^T (B^T), error-free products
    if (!launch_gram(ctx, Bt, l, 1, n, l, G, nullptr, gram_scratch, nullptr, true)) return false;
    const size_t smem = ((size_t)L * (L + 1) + L + JT) * sizeof(double) + (size_t)L * sizeof(int);
    cudaFuncSetAttribute(jacobi_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prof_begin(ctx);
    jacobi_eig_kernel<<<1, JT, smem, ctx->stream>>>(G, l, evals, evecs, V);
    if (!launch_done(ctx, K_CHOL, 8.0 * l * l * 3, 8.0 * l * l * l)) return false;
    prof_begin(ctx);
    ub_kernel<<<1, 256, 0, ctx->stream>>>(evals, evecs, l, k, ub, ubs, sv);
    if (!launch_done(ctx, K_CHOL, 8.0 * l * k, 0)) return false;
    // U^T (k x m) into Wc, V^T (k x n) into H
    if (!launch_gemm_ax(ctx, Q, l, ub, k, 1, Wc, 1, m, m, k, l)) return false;
    if (!launch_gemm_ax(ctx, Bt, l, ubs, k, 1, H, 1, n, n, k, l)) return false;
    prof_begin(ctx);
    part_norms_kernel<<<k, 256, 0, ctx->stream>>>(Wc, m, un);
    if (!launch_done(ctx, K_TRANSPOSE, 4.0 * m * k, 2.0 * m * k)) return false;
    prof_begin(ctx);
    part_norms_kernel<<<k, 256, 0, ctx->stream>>>(H, n, vn);
    if (!launch_done(ctx, K_TRANSPOSE, 4.0 * n * k, 2.0 * n * k)) return false;
    const int64_t cap = (int64_t)ctx->num_sms * 4 / (k > 0 ? k : 1) + 1;
    auto gx = [&](int64_t len) { const int64_t g = (len + 255) / 256; return (unsigned)(g < cap ? g : cap); };
    prof_begin(ctx);
    nndsvd_apply_kernel<<<dim3(gx(m), k), 256, 0, ctx->stream>>>(Wc, m, 0, un, vn, sv, k);
    if (!launch_done(ctx, K_TRANSPOSE, 8.0 * m * k, 2.0 * m * k)) return false;
    prof_begin(ctx);
    nndsvd_apply_kernel<<<dim3(gx(n), k), 256, 0, ctx->stream>>>(H, n, 1, un, vn, sv, k);
    return launch_done(ctx, K_TRANSPOSE, 8.0 * n * k, 2.0 * n * k);
}
