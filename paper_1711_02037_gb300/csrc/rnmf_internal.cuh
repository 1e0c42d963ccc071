// rnmf_internal.cuh - shared declarations of the CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <utility>
#include <vector>

#include "../../include/rnmf.h"

#define RNMF_MAX_L 128

// Device status word values (same numbering as rnmf_status).
#define RNMF_DEV_OK 0
#define RNMF_DEV_NOTPD 4
#define RNMF_DEV_TIMEOUT 5

// Kernel classes timed by the profiling facility (rnmf_profile).
enum KernelClass {
    K_OMEGA = 0, K_UNIFORM, K_GEMM_AX, K_GEMM_ATX, K_SPLITK, K_GRAM, K_CHOL, K_HALS_ROWS, K_WHALF, K_RELERR,
    K_TRANSPOSE, K_TC_AX, K_TC_ATX, K_TC_PACK, K_TC_REDUCE, K_ADJOINT, K_IL_PASS, K_COMPOBJ, K_RTILE, K_TVTILE,
    K_R_TC, K_TV_TC, K_S_TC, K_COUNT
};

struct ProfPending {
    int cls;
    cudaEvent_t a, b;
    double bytes, flops;
};

struct rnmf_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    int* d_status = nullptr;      // device status word (RNMF_DEV_*)
    unsigned* d_bar = nullptr;    // grid-barrier counters
    int* d_flags = nullptr;       // small device flags (CholeskyQR shift used, ...)
    char* arena = nullptr;        // scratch arena
    size_t arena_size = 0;
    size_t scratch_limit = 0;     // cap on arena + staging + batch workspace bytes (0: none)
    size_t arena_used = 0;
    float* stage_A = nullptr;     // device staging of A for rnmf_host
    size_t stage_A_bytes = 0;
    long long launches = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
    std::string last_error;
    // profiling (rnmf_profile): events around every launch when enabled
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<ProfPending> pending;
    cudaEvent_t prof_open = nullptr;
    void* batch_plan = nullptr;   // plan of the last batched call (batched_api.cu)
    int batch_policy = -1;        // autotuner override: cluster threshold index (-1: tune)
    int batch_threads = 0;        // autotuner override: threads per CTA for l <= 32 (0: tune)
    cudaStream_t copy_stream = nullptr;   // host -> device copies of the streamed QB (streamed.cu)
    cudaEvent_t copy_events[4] = {};
    cudaStream_t side_stream = nullptr;   // a sweep's S = W^T W next to the next sweep's R (rnmf_api.cu)
    cudaEvent_t side_events[2] = {};      // fork (main -> side), join (side -> main)
    long long prof_launches[K_COUNT] = {};
    double prof_ms[K_COUNT] = {}, prof_bytes[K_COUNT] = {}, prof_flops[K_COUNT] = {};
};

// Profiling hooks (rnmf_api.cu): begin records an event before a launch, end
// records one after it with the launch's algorithmic bytes and flops.
void prof_begin(rnmf_ctx* ctx);
void prof_end(rnmf_ctx* ctx, int cls, double bytes, double flops);
void prof_resolve(rnmf_ctx* ctx);
// Streamed QB (streamed.cu): A in host memory, column blocks of bc columns.
int64_t streamed_block_cols(int64_t m, int64_t n, int64_t requested);
size_t streamed_qb_bytes(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int64_t bc, int precision);
rnmf_status run_qb_streamed(rnmf_ctx* ctx, const float* A_host, int64_t m, int64_t n, int64_t lda, int l, int q,
                            uint64_t seed, int omega_dist, int64_t bc, int precision, float* Q, float* Bt);
// Frees the batched plan (graph, workspace, streams) of a context; its workspace bytes.
void rb_plan_release(rnmf_ctx* ctx);
size_t rb_plan_bytes(rnmf_ctx* ctx);

// ------------------------------------------------------------------ arena
// Bump allocation from the context arena; 256-byte aligned.  reserve() grows
// the arena (reallocating) when a call needs more than it has.
rnmf_status arena_reserve(rnmf_ctx* ctx, size_t bytes);
void* arena_take(rnmf_ctx* ctx, size_t bytes);
inline void arena_reset(rnmf_ctx* ctx) { ctx->arena_used = 0; }
inline size_t arena_round(size_t b) { return (b + 255) & ~size_t(255); }

// ------------------------------------------------------------- launchers
// All launchers enqueue on ctx->stream and count the launches; they return
// false on a launch error (the caller reports RNMF_ECUDA).

// Random draws (gen.cu).
bool launch_omega(rnmf_ctx* ctx, float* out, int64_t n, int l, uint64_t seed, int dist,
                  int64_t s_row, int64_t s_col);
bool launch_uniform_matrix(rnmf_ctx* ctx, float* out, int64_t rows, int64_t cols, uint64_t seed,
                           uint32_t stream_id, int64_t s_row, int64_t s_col);

// FP32 CUDA-core products with compensated accumulation (gemm_simt.cu).
//   out[i*so_r + j*so_c] = sum_r A[i*lda + r] * X[r*sx_r + j*sx_c]        (ax)
//   out[i*so_r + j*so_c] = sum_r A[r*lda + i] * X[r*sx_r + j*sx_c]        (atx)
// M x N output, contraction length K; N <= 128.  accumulate: out += product.
// ax: scratch (gemm_ax_scratch_bytes, or null: no split of the contraction) lets
// large products split the contraction to fill the last wave of blocks.
bool launch_gemm_ax(rnmf_ctx* ctx, const float* A, int64_t lda, const float* X, int64_t sx_r,
                    int64_t sx_c, float* out, int64_t so_r, int64_t so_c, int64_t M, int N, int64_t K,
                    bool accumulate = false, double* scratch = nullptr);
size_t gemm_ax_scratch_bytes(rnmf_ctx* ctx, int64_t M, int N, int64_t K);
size_t gemm_atx_scratch_bytes(rnmf_ctx* ctx, int64_t M, int N, int64_t K);
// streamed.cu: the GPU's own loads of an m x w block of pinned host memory
// (src_dev: its device address) into dst (rows w apart); the device address of
// a pinned host pointer, or nullptr for pageable memory
bool launch_pull_rows(rnmf_ctx* ctx, cudaStream_t stream, const float* src_dev, int64_t lda, int64_t m, int64_t w,
                      float* dst);
const float* host_device_view(const float* host);
// order.cu: the shuffled update order (gathers of the stored components)
struct OrderBufs {
    int* sigma;  // slot -> component held there
    int* rho;    // gather source slot of each destination slot
    float* tmp;  // k x max(m, n) floats (also the small gathers)
    char* il;    // interleaved order: the fused passes' scratch (il_scratch_bytes)
};
size_t order_bytes(int64_t m, int64_t n, int l, int k);
OrderBufs order_take(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int k);
bool order_begin(rnmf_ctx* ctx, const OrderBufs& ob, int k);
bool order_sweep(rnmf_ctx* ctx, const OrderBufs& ob, uint64_t seed, int t, float* Wc, int64_t m, float* H, int64_t n,
                 float* Wt, int l, float* S32, double* S64, int k);
bool order_end(rnmf_ctx* ctx, const OrderBufs& ob, float* Wc, int64_t m, float* H, int64_t n, float* Wt, int l,
               float* S32, double* S64, int k);
// init_svd.cu: NNDSVD initial factors (Wc k x m, H k x n) from Q (m x l) and B^T (n x l);
// takes svd_init_bytes(l, k) from the arena; gram_scratch >= gram_scratch_bytes(n, l)
size_t svd_init_bytes(int l, int k);
bool launch_svd_init(rnmf_ctx* ctx, const float* Q, const float* Bt, int64_t m, int64_t n, int l, int k, float* Wc,
                     float* H, double* gram_scratch);
// tiles8.cu: 8 x 8-tile products taken by launch_gemm_atx (out M x N <= 128 x 128)
// and launch_gemm_ax (contraction K <= 128, N <= 128)
bool xty8_fits(int64_t M, int N);
size_t xty8_scratch_bytes(rnmf_ctx* ctx, int64_t M, int N, int64_t K);
bool launch_xty8(rnmf_ctx* ctx, const float* Xr, int64_t sxr, int64_t sxc, int cx, const float* Y, int64_t syr,
                 int64_t syc, int cy, int64_t N, float* out, int64_t so_r, int64_t so_c, double* scratch,
                 bool accumulate);
bool ax8_fits(int N, int64_t K);
bool launch_ax8(rnmf_ctx* ctx, const float* A, int64_t lda, const float* X, int64_t sx_r, int64_t sx_c, float* out,
                int64_t so_r, int64_t so_c, int64_t M, int N, int64_t K, bool accumulate);
bool launch_gemm_atx(rnmf_ctx* ctx, const float* A, int64_t lda, const float* X, int64_t sx_r,
                     int64_t sx_c, float* out, int64_t so_r, int64_t so_c, int64_t M, int N, int64_t K,
                     double* scratch, bool accumulate = false);

// Gram matrices G = X^T X (gram.cu).  X is N x c (c <= 128) with element
// (r, j) at X[r*s_r + j*s_c].  Writes G (c x c, symmetric) as double and, if
// G32 != NULL, as float.  exact: error-free products with float32-pair
// accumulation (for CholeskyQR); otherwise compensated float32.  When
// skip_if_zero != NULL and *skip_if_zero == 0 the launch does nothing.
size_t gram_scratch_bytes(rnmf_ctx* ctx, int64_t N, int c);
// Gp != NULL (not with the column-major non-exact form): also as normalised float pairs hi + lo.
bool launch_gram(rnmf_ctx* ctx, const float* X, int64_t s_r, int64_t s_c, int64_t N, int c, double* G,
                 float* G32, double* scratch, const int* skip_if_zero = nullptr, bool exact = false,
                 float2* Gp = nullptr);

// CholeskyQR (cholqr.cu): Q = Y R^{-1} in place on Y (N x c, row-major, ld c)
// with R = chol(Y^T Y) in double-float arithmetic (df.cuh); two passes (CholeskyQR2), plus a third when
// the first Gram needed a diagonal shift.
size_t cholqr_scratch_bytes(rnmf_ctx* ctx, int64_t N, int c);
bool cholqr2(rnmf_ctx* ctx, float* Y, int64_t N, int c, char* scratch);

// HALS kernels (hals.cu).
//   Row-recurrence update of `count` vectors x (k entries each, element j of
//   vector v at X[v*sv + j*se]) with right-hand side Rhs (element j of vector v
//   at Rhs[v*srv + j*srj]) and Gram S (k x k float, row-major):
//   for j: if S_jj > 0: x_j <- max(0, x_j + (rhs_j - sum_i x_i S_ij) / S_jj).
// alpha, beta: Section 3.4 penalties of the rows (0, 0: the plain rule).
bool launch_hals_rows(rnmf_ctx* ctx, float* X, int64_t sv, int64_t se, const float* Rhs, int64_t srv,
                      int64_t srj, const float* S, int64_t count, int k, float alpha = 0.f, float beta = 0.f);
// hhalf.cu: the products of the H half on column tiles (Bt n x l, Wt l x k, H k x n):
// Rt = (B^T W~)^T (k x n), and Tt = (B H^T)^T (k x l) with V = H H^T (k x k) through
// block partial sums in a scratch of hhalf_scratch_bytes.  hhalf_fits: the
// shared-memory plans fit (else the generic product kernels are used).
bool hhalf_fits(int l, int k);
size_t hhalf_scratch_bytes(rnmf_ctx* ctx, int64_t n, int l, int k);
bool launch_rtile(rnmf_ctx* ctx, const float* Bt, int64_t n, int l, const float* Wt, int k, float* Rt);
bool launch_tv(rnmf_ctx* ctx, const float* Bt, int64_t n, int l, const float* H, int k, float* Tt, float* V,
               float* scratch);
//   Persistent W half-sweep of randomized HALS (Gauss-Seidel over columns j):
//   W~_j += (T_j - W~ V_j)/V_jj; W_j = max(0, Q W~_j); W~_j = Q^T W_j.
//   Qp (m x lp, row-major, lp = l rounded up to 4, zero padded), Wc = W^T (k x m),
//   Wt (l x k), Tt = T^T (k x l), V (k x k).
size_t whalf_scratch_bytes(rnmf_ctx* ctx, int64_t m, int l, int k);
// the fixed-point bound factor of the padded Q into the whalf scratch (once per Q, before launch_whalf)
bool launch_whalf_prepare(rnmf_ctx* ctx, const float* Qp, int64_t m, int l, int lp, char* scratch);
//   With penalties (alpha, beta, Section 3.4): W~_j = (V_jj W~_j + T_j - beta q1 - W~ V_j) / (V_jj + alpha),
//   q1 = Q^T 1 (l floats, from launch_colsum).
// columns [jbeg, jend) of the W half (jend < 0: every column)
bool launch_whalf(rnmf_ctx* ctx, const float* Qp, int64_t m, int l, int lp, int k, float* Wc, float* Wt,
                  const float* Tt, const float* V, char* scratch, long long spin_limit, float alpha = 0.f,
                  float beta = 0.f, const float* q1 = nullptr, int jbeg = 0, int jend = -1);
// interleaved.cu: the interleaved order W_1 -> H_1 -> ... -> W_k -> H_k (Section 3.2) as two
// passes per component; scratch = il_scratch_bytes (a ticket word that il_begin zeroes, then
// block partials).  W pass: column j of W (Wc = W^T) from u = W~ rule(T_row, V_row), then
// W~_:j = Q^T W_j and S_row_out = W^T W_j (gram_mode 1: W~^T W~_j).  H pass: row j of H
// (j < 0: none) from B^T W~_:j and S_row, then T_out = B H_jn^T, V_out = H H_jn^T (jn < 0: none).
size_t il_scratch_bytes(rnmf_ctx* ctx);
bool il_begin(rnmf_ctx* ctx, char* scratch);
bool launch_il_wpass(rnmf_ctx* ctx, const float* Qp, int64_t m, int l, int lp, int k, int j, float* Wc, float* Wt,
                     const float* T_row, const float* V_row, const float* q1, float alpha, float beta, int gram_mode,
                     float* S_row_out, char* scratch);
bool launch_il_hpass(rnmf_ctx* ctx, const float* Bt, int64_t n, int l, int k, int j, int jn, float* H,
                     const float* Wt, const float* S_row, float alpha, float beta, float* T_out, float* V_out,
                     char* scratch);
// Compressed projected gradient (pgrad.cu): partial sums then one float64 total in *out.
size_t pgrad_scratch_bytes(int64_t m, int64_t n);
bool launch_pgrad(rnmf_ctx* ctx, const float* Wc, const float* Q, int64_t m, int l, int lq, int k, const float* V,
                  const float* T, const float* H, const float* Rt, int64_t n, const float* S, double* scratch,
                  double* out);
// q1 = Q^T 1 for Qp (m x lp, rows padded): l column sums in float64, rounded to float.
bool launch_colsum(rnmf_ctx* ctx, const float* Qp, int64_t m, int l, int lp, float* out);
// Copy Q (m x l, ld l) into Qp (m x lp, ld lp) with zero padding (gen.cu).
bool launch_pad_rows(rnmf_ctx* ctx, const float* in, int64_t rows, int cols, int ld_out, float* out);

// Objective (objective.cu): sum (A - W H)^2 and sum A^2 in float64.  W element
// (i, t) at W[i*sw_r + t*sw_c], H row-major k x n.
size_t relerr_scratch_bytes(rnmf_ctx* ctx, int64_t m, int64_t n);
bool launch_relerr(rnmf_ctx* ctx, const float* A, int64_t lda, const float* W, int64_t sw_r, int64_t sw_c,
                   const float* H, int64_t m, int64_t n, int k, double* out2 /* [2] device */,
                   double* scratch);
// Compressed objective (Section 3.2) f~ = ||B - W~ H||_F^2 into out2[0] and ||B||_F^2
// into out2[1] (device), from B^T (n x l), W~ (l x k) and H (k x n); scratch of
// compobj_scratch_bytes.
size_t compobj_scratch_bytes(rnmf_ctx* ctx, int64_t n, int l);
bool launch_compobj(rnmf_ctx* ctx, const float* Bt, int64_t n, int l, const float* Wt, int k, const float* H,
                    double* out2, double* scratch);

// Adjoint of T compressed sweeps (adjoint.cu).  Checkpoint state t holds
// W_t^T (k x m), W~_t (l x k), H_t (k x n).
size_t adjoint_ckpt_floats(int64_t m, int64_t n, int l, int k);
size_t wrev_scratch_bytes(rnmf_ctx* ctx, int64_t m);
bool launch_hrev(rnmf_ctx* ctx, const float* Ho, const float* Hn, const float* dHn, const float* S, int64_t n, int k,
                 float* dHo, float* DA);
bool launch_wrev(rnmf_ctx* ctx, const float* Q, int64_t m, int l, int k, const float* Wn, const float* Wo,
                 const float* Wct, const float* dWct, const float* dWn, const float* T, const float* V, float* dT,
                 float* dV, float* dWo, float* dWpass, char* scratch, long long spin_limit);
bool launch_sym(rnmf_ctx* ctx, const float* P1T, const float* P0T, int k, float* out);
bool launch_outer(rnmf_ctx* ctx, const float* Q, const float* dBt, int64_t m, int64_t n, int l, float* dA);

// Small helpers (gen.cu).
bool launch_transpose(rnmf_ctx* ctx, const float* in, int64_t rows, int64_t cols, float* out);
bool launch_copy(rnmf_ctx* ctx, const float* in, float* out, int64_t count);

// Grid barrier with a bounded wait (device side; sync.cuh).
#define RNMF_DEFAULT_SPIN_LIMIT 2000000000LL

// Bytes of device scratch the context holds now (arena, host staging, batch plan).
size_t scratch_held(rnmf_ctx* ctx);
// True when growing the context's scratch by `extra` bytes stays within its cap.
inline bool scratch_fits(rnmf_ctx* ctx, size_t held_after) {
    return ctx->scratch_limit == 0 || held_after <= ctx->scratch_limit;
}

// Launch of a kernel whose blocks wait on one another (a spin on words other
// blocks write): cooperative, so the driver either makes every block resident
// at once or refuses the launch; a wait can then only run out if a block
// fails, never because its partner was not scheduled.
template <typename... KArgs, typename... Args>
inline bool launch_cooperative(rnmf_ctx* ctx, void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                               Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...) == cudaSuccess;
}

inline bool launch_ok(rnmf_ctx* ctx) {
    ctx->launches++;
    return cudaPeekAtLastError() == cudaSuccess;
}

// After a launch: count it, close its profiling interval, check for errors.
inline bool launch_done(rnmf_ctx* ctx, int cls, double bytes, double flops) {
    if (ctx->prof_on) prof_end(ctx, cls, bytes, flops);
    return launch_ok(ctx);
}
