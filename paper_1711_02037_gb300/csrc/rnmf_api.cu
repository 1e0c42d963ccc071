// rnmf_api.cu - C ABI entry points and the host-side orchestration of
// randomized HALS (Algorithm 1) and deterministic HALS (Section 3.1).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "rnmf_internal.cuh"
#include "tc_gemm.cuh"

// ------------------------------------------------------------------ arena
rnmf_status arena_reserve(rnmf_ctx* ctx, size_t bytes) {
    ctx->arena_used = 0;
    if (bytes <= ctx->arena_size) return RNMF_OK;
    if (!scratch_fits(ctx, scratch_held(ctx) - ctx->arena_size + bytes)) return RNMF_ENOMEM;
    if (ctx->arena) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->arena);
        ctx->arena = nullptr;
        ctx->arena_size = 0;
    }
    size_t want = bytes + (bytes >> 3);
    if (!scratch_fits(ctx, scratch_held(ctx) + want)) want = bytes;
    if (cudaMalloc(&ctx->arena, want) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc(&ctx->arena, bytes) != cudaSuccess) {
            cudaGetLastError();
            ctx->arena = nullptr;
            return RNMF_ENOMEM;
        }
        want = bytes;
    }
    ctx->arena_size = want;
    return RNMF_OK;
}

size_t scratch_held(rnmf_ctx* ctx) { return ctx->arena_size + ctx->stage_A_bytes + rb_plan_bytes(ctx); }

void* arena_take(rnmf_ctx* ctx, size_t bytes) {
    size_t b = arena_round(bytes);
    void* p = ctx->arena + ctx->arena_used;
    ctx->arena_used += b;
    return p;
}

// -------------------------------------------------------------- profiling
static const char* kClassNames[K_COUNT] = {"omega", "uniform_init", "gemm_ax_fp32", "gemm_atx_fp32",
                                           "splitk_reduce", "gram_f64", "chol_inv", "hals_rows", "whalf",
                                           "relerr", "transpose", "tc_gemm_ax", "tc_gemm_atx", "tc_pack",
                                           "tc_reduce", "adjoint", "il_pass", "compobj", "r_tile", "tv_tile",
                                           "r_tc", "tv_tc", "s_tc"};

static cudaEvent_t pool_get(rnmf_ctx* ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(rnmf_ctx* ctx) {
    if (!ctx->prof_on) return;
    ctx->prof_open = pool_get(ctx);
    cudaEventRecord(ctx->prof_open, ctx->stream);
}

void prof_end(rnmf_ctx* ctx, int cls, double bytes, double flops) {
    if (!ctx->prof_on || !ctx->prof_open) return;
    cudaEvent_t b = pool_get(ctx);
    cudaEventRecord(b, ctx->stream);
    ctx->pending.push_back(ProfPending{cls, ctx->prof_open, b, bytes, flops});
    ctx->prof_open = nullptr;
}

void prof_resolve(rnmf_ctx* ctx) {
    if (ctx->pending.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (const ProfPending& p : ctx->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            ctx->prof_launches[p.cls]++;
            ctx->prof_ms[p.cls] += ms;
            ctx->prof_bytes[p.cls] += p.bytes;
            ctx->prof_flops[p.cls] += p.flops;
        }
        ctx->ev_pool.push_back(p.a);
        ctx->ev_pool.push_back(p.b);
    }
    cudaGetLastError();
    ctx->pending.clear();
}

namespace {

rnmf_status fail(rnmf_ctx* ctx, rnmf_status st, const char* msg) {
    if (ctx) ctx->last_error = msg;
    return st;
}

rnmf_status cuda_fail(rnmf_ctx* ctx, const char* where) {
    cudaError_t e = cudaGetLastError();
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    ctx->last_error = buf;
    return RNMF_ECUDA;
}

// Synchronise the stream and turn the device status word into a status.
rnmf_status finish(rnmf_ctx* ctx, const char* what) {
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_fail(ctx, what);
    prof_resolve(ctx);
    int st = 0;
    if (cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_fail(ctx, what);
    if (st == RNMF_DEV_NOTPD)
        return fail(ctx, RNMF_ENOTPD, "Gram matrix of the QR step is not positive definite after the shift");
    if (st == RNMF_DEV_TIMEOUT)
        return fail(ctx, RNMF_ETIMEOUT, "a grid-barrier wait ran out (blocks not co-resident?)");
    if (st != 0) return fail(ctx, RNMF_ECUDA, "unknown device status");
    return RNMF_OK;
}

rnmf_status begin(rnmf_ctx* ctx) {
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, "cudaSetDevice");
    if (cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream) != cudaSuccess)
        return cuda_fail(ctx, "cudaMemsetAsync");
    return RNMF_OK;
}

rnmf_opts opts_or_default(const rnmf_opts* o) {
    rnmf_opts d;
    rnmf_default_opts(&d);
    return o ? *o : d;
}

// Section 3.4 penalties: finite and >= 0.
bool penalties_ok(const rnmf_opts& o) {
    const float v[4] = {o.alpha_W, o.alpha_H, o.beta_W, o.beta_H};
    for (float x : v)
        if (!(x >= 0.f) || !std::isfinite(x)) return false;
    return true;
}

bool has_penalties(const rnmf_opts& o) {
    return o.alpha_W != 0.f || o.alpha_H != 0.f || o.beta_W != 0.f || o.beta_H != 0.f;
}

rnmf_status check_tc(rnmf_ctx* ctx, const float* A, int64_t lda, int precision) {
    if (precision == RNMF_PREC_FP32) return RNMF_OK;
    if (!tc_available()) return fail(ctx, RNMF_ENOTIMPL, "tensor-core forms unavailable (no TMA descriptor entry point)");
    if ((lda & 3) != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0)
        return fail(ctx, RNMF_EINVAL, "tensor-core forms need lda % 4 == 0 and a 16-byte aligned A");
    return RNMF_OK;
}

rnmf_status check_shape(rnmf_ctx* ctx, int64_t m, int64_t n, int64_t lda, int k, int p) {
    if (m < 1 || n < 1 || m >= (1LL << 31) || n >= (1LL << 31)) return fail(ctx, RNMF_EINVAL, "m, n out of range");
    if (lda < n) return fail(ctx, RNMF_EINVAL, "lda < n");
    if (k < 1) return fail(ctx, RNMF_EINVAL, "k < 1");
    if (p < 0) return fail(ctx, RNMF_EINVAL, "p < 0");
    int64_t l = (int64_t)k + p;
    if (l > RNMF_MAX_L) return fail(ctx, RNMF_EINVAL, "l = k + p exceeds 128");
    int64_t mn = m < n ? m : n;
    if (l > mn && !(l == m && m <= n)) return fail(ctx, RNMF_EINVAL, "l = k + p exceeds min(m, n)");
    return RNMF_OK;
}

// ---------------------------------------------------------------- sizes
struct QbBufs {
    float *Omega, *Y, *Z;
    char* cq;      // CholeskyQR scratch
    double* atx;   // split-K scratch (A^T X and A X)
    TcScratch tc;  // tensor-core forms
};

size_t qb_bytes(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int precision) {
    size_t b = arena_round((size_t)n * l * 4) + arena_round((size_t)m * l * 4) + arena_round((size_t)n * l * 4);
    int64_t big = m > n ? m : n;
    b += arena_round(cholqr_scratch_bytes(ctx, big, l));
    size_t a1 = gemm_atx_scratch_bytes(ctx, n, l, m), a2 = gemm_ax_scratch_bytes(ctx, m, l, n);
    if (a2 > a1) a1 = a2;
    b += arena_round(a1 > 0 ? a1 : 8);
    b += tc_scratch_bytes(ctx, m, n, l, precision);
    return b;
}

QbBufs qb_take(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int precision) {
    QbBufs q;
    q.Omega = (float*)arena_take(ctx, (size_t)n * l * 4);
    q.Y = (float*)arena_take(ctx, (size_t)m * l * 4);
    q.Z = (float*)arena_take(ctx, (size_t)n * l * 4);
    int64_t big = m > n ? m : n;
    q.cq = (char*)arena_take(ctx, cholqr_scratch_bytes(ctx, big, l));
    size_t a1 = gemm_atx_scratch_bytes(ctx, n, l, m), a2 = gemm_ax_scratch_bytes(ctx, m, l, n);
    if (a2 > a1) a1 = a2;
    q.atx = (double*)arena_take(ctx, a1 > 0 ? a1 : 8);
    q.tc = tc_scratch_take(ctx, m, n, l, precision);
    return q;
}

// Y (m x l) = A X with X (n x l) row-major; form chosen by `accurate`.
bool product_ax(rnmf_ctx* ctx, const QbBufs& b, int precision, bool accurate, const float* A, int64_t lda,
                const float* X, float* Y, int64_t m, int64_t n, int l) {
    if (precision == RNMF_PREC_FP32) return launch_gemm_ax(ctx, A, lda, X, l, 1, Y, l, 1, m, l, n, false, b.atx);
    return tc_gemm_ax(ctx, b.tc, A, lda, X, Y, m, n, l, accurate ? 3 : 1);
}

// Z (n x l) = A^T X with X (m x l) row-major.
bool product_atx(rnmf_ctx* ctx, const QbBufs& b, int precision, bool accurate, const float* A, int64_t lda,
                 const float* X, float* Z, int64_t m, int64_t n, int l) {
    if (precision == RNMF_PREC_FP32) return launch_gemm_atx(ctx, A, lda, X, l, 1, Z, l, 1, n, l, m, b.atx);
    return tc_gemm_atx(ctx, b.tc, A, lda, X, Z, m, n, l, accurate ? 3 : 1);
}

// Randomized QB (Section 2.3; Algorithm 1 QB part) into Q (m x l) and Bt (n x l).
// Power-iteration products run in the cheap form for RNMF_PREC_BF16; the last
// sketch (which fixes Q) and B always run in an accurate form.
rnmf_status run_qb(rnmf_ctx* ctx, const QbBufs& b, const float* A, int64_t m, int64_t n, int64_t lda, int l, int q,
                   uint64_t seed, const rnmf_opts& o, float* Q, float* Bt) {
    const int prec = o.precision;
    const bool split_all = prec == RNMF_PREC_SPLIT3;
    if (!launch_omega(ctx, b.Omega, n, l, seed, o.omega_dist, l, 1)) return cuda_fail(ctx, "omega");
    // Y = A Omega (accurate when it is also the last sketch)
    if (!product_ax(ctx, b, prec, split_all || q == 0, A, lda, b.Omega, Q, m, n, l)) return cuda_fail(ctx, "A*Omega");
    for (int i = 0; i < q; ++i) {
        if (!cholqr2(ctx, Q, m, l, b.cq)) return cuda_fail(ctx, "cholqr(Y)");
        if (!product_atx(ctx, b, prec, split_all, A, lda, Q, b.Z, m, n, l)) return cuda_fail(ctx, "A^T Q");
        if (!cholqr2(ctx, b.Z, n, l, b.cq)) return cuda_fail(ctx, "cholqr(Z)");
        if (!product_ax(ctx, b, prec, split_all || i == q - 1, A, lda, b.Z, Q, m, n, l))
            return cuda_fail(ctx, "A*Q");
    }
    if (!cholqr2(ctx, Q, m, l, b.cq)) return cuda_fail(ctx, "cholqr(Y)");
    if (!product_atx(ctx, b, prec, true, A, lda, Q, Bt, m, n, l)) return cuda_fail(ctx, "B = Q^T A");
    return RNMF_OK;
}

struct SweepBufs {
    float *Rt, *S32, *T, *V32, *Wt, *Qp, *q1;
    double *S64, *V64, *gram, *atx, *relerr, *hist;
    // compressed objective (Section 3.2) per sweep: (f~ after the H half, ||B||^2,
    // f~ after the sweep, ||B||^2) for sweep t at obj[4 t]; objpart: tile partials
    double *obj, *objpart;
    float* hh;  // block partial sums of the one-pass H half
    char* wh;
    // projected-gradient measure (Section 3.3): R^T, T, V, S of the current state
    float *pgRt, *pgT, *pgV, *pgS;
    double *pgV64, *pgS64, *pgpart, *pgout;
    TcHhalf tch;  // the H half on tensor cores (sweep_products = RNMF_SWEEP_SPLIT3), else empty
};

// Scratch of the tensor-core H half: taken when the option asks for it and the
// tensor-core path exists (run_sweeps checks the remaining conditions per call).
bool tch_wanted(const rnmf_opts& o, int l, int k) {
    return o.sweep_products == RNMF_SWEEP_SPLIT3 && l <= 128 && k <= 128 && tc_available();
}
size_t tch_reserve(rnmf_ctx* ctx, const rnmf_opts& o, int64_t m, int64_t n, int l, int k) {
    return tch_wanted(o, l, k) ? tc_hhalf_bytes(ctx, m, n, l, k) : 0;
}
void tch_take(rnmf_ctx* ctx, const rnmf_opts& o, int64_t m, int64_t n, int l, int k, SweepBufs& s) {
    if (tch_wanted(o, l, k)) s.tch = tc_hhalf_take(ctx, m, n, l, k);
}
bool sweep_products_ok(const rnmf_opts& o) {
    return o.sweep_products == RNMF_SWEEP_FP32 || o.sweep_products == RNMF_SWEEP_SPLIT3;
}

size_t sweep_bytes(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int k, int iters, bool track) {
    int64_t big = m > n ? m : n;
    size_t b = arena_round((size_t)k * n * 4) + 2 * arena_round((size_t)k * k * 4) + 2 * arena_round((size_t)l * k * 4);
    b += 2 * arena_round((size_t)k * k * 8);
    b += arena_round(gram_scratch_bytes(ctx, big, k));
    size_t a1 = gemm_atx_scratch_bytes(ctx, l, k, n), a2 = gemm_atx_scratch_bytes(ctx, l, k, m);
    b += arena_round((a1 > a2 ? a1 : a2) + 8);
    b += arena_round(track ? relerr_scratch_bytes(ctx, m, n) : 8);
    b += arena_round((size_t)(iters + 1) * 2 * 8);
    b += arena_round((size_t)(iters + 1) * 4 * 8) + arena_round(compobj_scratch_bytes(ctx, n, l));
    b += arena_round(hhalf_fits(l, k) ? hhalf_scratch_bytes(ctx, n, l, k) : 8);
    b += arena_round(whalf_scratch_bytes(ctx, m, l, k));
    b += arena_round((size_t)m * ((l + 3) / 4 * 4) * 4);
    b += arena_round((size_t)RNMF_MAX_L * 4);
    b += arena_round((size_t)k * n * 4) + arena_round((size_t)l * k * 4) + 2 * arena_round((size_t)k * k * 4) +
         2 * arena_round((size_t)k * k * 8) + arena_round(pgrad_scratch_bytes(m, n)) + arena_round(8);
    return b;
}

SweepBufs sweep_take(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int k, int iters, bool track) {
    SweepBufs s;
    int64_t big = m > n ? m : n;
    s.Rt = (float*)arena_take(ctx, (size_t)k * n * 4);
    s.S32 = (float*)arena_take(ctx, (size_t)k * k * 4);
    s.V32 = (float*)arena_take(ctx, (size_t)k * k * 4);
    s.T = (float*)arena_take(ctx, (size_t)l * k * 4);
    s.Wt = (float*)arena_take(ctx, (size_t)l * k * 4);
    s.S64 = (double*)arena_take(ctx, (size_t)k * k * 8);
    s.V64 = (double*)arena_take(ctx, (size_t)k * k * 8);
    s.gram = (double*)arena_take(ctx, gram_scratch_bytes(ctx, big, k));
    size_t a1 = gemm_atx_scratch_bytes(ctx, l, k, n), a2 = gemm_atx_scratch_bytes(ctx, l, k, m);
    s.atx = (double*)arena_take(ctx, (a1 > a2 ? a1 : a2) + 8);
    s.relerr = (double*)arena_take(ctx, track ? relerr_scratch_bytes(ctx, m, n) : 8);
    s.hist = (double*)arena_take(ctx, (size_t)(iters + 1) * 2 * 8);
    s.obj = (double*)arena_take(ctx, (size_t)(iters + 1) * 4 * 8);
    s.objpart = (double*)arena_take(ctx, compobj_scratch_bytes(ctx, n, l));
    s.hh = (float*)arena_take(ctx, hhalf_fits(l, k) ? hhalf_scratch_bytes(ctx, n, l, k) : 8);
    s.wh = (char*)arena_take(ctx, whalf_scratch_bytes(ctx, m, l, k));
    s.Qp = (float*)arena_take(ctx, (size_t)m * ((l + 3) / 4 * 4) * 4);
    s.q1 = (float*)arena_take(ctx, (size_t)RNMF_MAX_L * 4);
    s.pgRt = (float*)arena_take(ctx, (size_t)k * n * 4);
    s.pgT = (float*)arena_take(ctx, (size_t)l * k * 4);
    s.pgV = (float*)arena_take(ctx, (size_t)k * k * 4);
    s.pgS = (float*)arena_take(ctx, (size_t)k * k * 4);
    s.pgV64 = (double*)arena_take(ctx, (size_t)k * k * 8);
    s.pgS64 = (double*)arena_take(ctx, (size_t)k * k * 8);
    s.pgpart = (double*)arena_take(ctx, pgrad_scratch_bytes(m, n));
    s.pgout = (double*)arena_take(ctx, 8);
    return s;
}

// ||grad^P||_F^2 of the compressed problem at (W = Wc^T, W~ = s.Wt, H) (Section 3.3);
// s.Qp must hold Q with rows padded to lp.  Synchronises (host read).
bool pg_measure(rnmf_ctx* ctx, const SweepBufs& s, const float* Bt, int64_t m, int64_t n, int l, int lp, int k,
                const float* Wc, const float* H, double* out) {
    if (!launch_gemm_ax(ctx, Bt, l, s.Wt, k, 1, s.pgRt, 1, n, n, k, l)) return false;
    if (!launch_gemm_atx(ctx, Bt, l, H, 1, n, s.pgT, k, 1, l, k, n, s.atx)) return false;
    if (!launch_gram(ctx, H, 1, n, n, k, s.pgV64, s.pgV, s.gram)) return false;
    if (!launch_gram(ctx, Wc, 1, m, m, k, s.pgS64, s.pgS, s.gram)) return false;
    if (!launch_pgrad(ctx, Wc, s.Qp, m, l, lp, k, s.pgV, s.pgT, H, s.pgRt, n, s.pgS, s.pgpart, s.pgout))
        return false;
    return cudaMemcpyAsync(out, s.pgout, 8, cudaMemcpyDeviceToHost, ctx->stream) == cudaSuccess &&
           cudaStreamSynchronize(ctx->stream) == cudaSuccess;
}

// Gram S for the H update: W^T W (gram_mode 0, W held transposed as Wc k x m) or W~^T W~.
bool gram_S(rnmf_ctx* ctx, const SweepBufs& s, int gram_mode, const float* Wc, int64_t m, int l, int k) {
    if (gram_mode == 0) return launch_gram(ctx, Wc, 1, m, m, k, s.S64, s.S32, s.gram);
    return launch_gram(ctx, s.Wt, k, 1, l, k, s.S64, s.S32, s.gram);
}

// S from an arbitrary state (W^T, W~) into (S64, S32).
bool gram_S_from(rnmf_ctx* ctx, int gram_mode, const float* Wc, const float* Wt, int64_t m, int l, int k, double* S64,
                 float* S32, double* scratch) {
    if (gram_mode == 0) return launch_gram(ctx, Wc, 1, m, m, k, S64, S32, scratch);
    return launch_gram(ctx, Wt, k, 1, l, k, S64, S32, scratch);
}

// `iters` sweeps of Algorithm 1's loop from Wc (= W^T, k x m), H, W~ (in s.Wt), S (in s.S32).
// Copy the sweep state (W^T, W~, H) into checkpoint slot `slot` (adjoint.cu layout).
bool save_state(rnmf_ctx* ctx, float* ckpt, int slot, const float* Wc, const float* Wt, const float* H, int64_t m,
                int64_t n, int l, int k) {
    float* base = ckpt + (size_t)slot * adjoint_ckpt_floats(m, n, l, k);
    return cudaMemcpyAsync(base, Wc, (size_t)k * m * 4, cudaMemcpyDeviceToDevice, ctx->stream) == cudaSuccess &&
           cudaMemcpyAsync(base + (size_t)k * m, Wt, (size_t)l * k * 4, cudaMemcpyDeviceToDevice, ctx->stream) ==
               cudaSuccess &&
           cudaMemcpyAsync(base + (size_t)k * m + (size_t)l * k, H, (size_t)k * n * 4, cudaMemcpyDeviceToDevice,
                           ctx->stream) == cudaSuccess;
}

// S = W^T W of sweep t on the side stream: it reads W (the W half's output) and
// writes S, which only the next sweep's H rows read, so it runs next to the
// next sweep's W~ pack and R (they read W~ and B^T).  The join comes before
// the H rows.
bool side_ready(rnmf_ctx* ctx) {
    if (ctx->side_stream) return true;
    if (cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking) != cudaSuccess) return false;
    for (auto& e : ctx->side_events)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
    return true;
}
bool gram_S_side(rnmf_ctx* ctx, const SweepBufs& s, const float* Wc, int64_t m, int k) {
    if (cudaEventRecord(ctx->side_events[0], ctx->stream) != cudaSuccess ||
        cudaStreamWaitEvent(ctx->side_stream, ctx->side_events[0], 0) != cudaSuccess)
        return false;
    cudaStream_t main = ctx->stream;
    ctx->stream = ctx->side_stream;  // the launch helpers (and the profiler's events) follow ctx->stream
    const bool ok = tc_hhalf_gram(ctx, s.tch, Wc, m, k, s.S32);
    ctx->stream = main;
    return ok && cudaEventRecord(ctx->side_events[1], ctx->side_stream) == cudaSuccess;
}
bool side_join(rnmf_ctx* ctx, bool* pending) {
    if (!*pending) return true;
    *pending = false;
    return cudaStreamWaitEvent(ctx->stream, ctx->side_events[1], 0) == cudaSuccess;
}

rnmf_status run_sweeps(rnmf_ctx* ctx, const SweepBufs& s, const float* Q, const float* Bt, int64_t m, int64_t n, int l,
                       int k, int iters, const rnmf_opts& o, float* Wc, float* H, const float* A, int64_t lda,
                       int* ntracked, float* ckpt = nullptr, int* done = nullptr, double* pg_ratio = nullptr,
                       const OrderBufs* ob = nullptr, bool obj = false) {
    *ntracked = 0;
    // shuffled order: the components are gathered into sweep t's visiting order before it
    const bool shuffled = o.order == RNMF_ORDER_SHUFFLED && iters > 0;
    if (shuffled && (!ob || !order_begin(ctx, *ob, k))) return cuda_fail(ctx, "order");
    if (done) *done = iters;
    if (pg_ratio) *pg_ratio = -1.0;
    const int lp = (l + 3) / 4 * 4;
    // the H half's products on tensor cores: B^T's operand tiles once for all sweeps
    const bool tch = s.tch.part && o.order != RNMF_ORDER_INTERLEAVED && iters > 0 && tc_hhalf_fits(n, l, k, Bt, H);
    if (tch && !tc_hhalf_pack_b(ctx, s.tch, Bt, n, l)) return cuda_fail(ctx, "pack B^T");
    const bool tch_s = s.tch.part && o.order == RNMF_ORDER_CYCLIC && o.gram_mode == 0 && tc_gram_fits(m, k, Wc);
    if (tch_s && !side_ready(ctx)) return cuda_fail(ctx, "side stream");
    bool s_pending = false;  // S of the last sweep still running on the side stream
    struct JoinAtExit {      // every return (the last sweep, a stop, an error) orders the side work first
        rnmf_ctx* ctx;
        bool* pending;
        ~JoinAtExit() { side_join(ctx, pending); }
    } join_at_exit{ctx, &s_pending};
    if (iters > 0 && !launch_pad_rows(ctx, Q, m, l, lp, s.Qp)) return cuda_fail(ctx, "pad Q");
    if (iters > 0 && !launch_whalf_prepare(ctx, s.Qp, m, l, lp, s.wh)) return cuda_fail(ctx, "Q row norms");
    if (iters > 0 && o.beta_W != 0.f && !launch_colsum(ctx, s.Qp, m, l, lp, s.q1)) return cuda_fail(ctx, "Q^T 1");
    // Section 3.3 stopping rule: ||grad^P||^2 <= pg_tol ||grad^P(W0, H0)||^2, checked every pg_every sweeps
    const bool pg = o.pg_tol > 0.0 && iters > 0;
    const int every = o.pg_every > 0 ? o.pg_every : 10;
    double pg0 = 0.0;
    if (pg && !pg_measure(ctx, s, Bt, m, n, l, lp, k, Wc, H, &pg0)) return cuda_fail(ctx, "projected gradient");
    for (int it = 0; it < iters; ++it) {
        if (o.order == RNMF_ORDER_INTERLEAVED) {
            // W_1 -> H_1 -> ... -> W_k -> H_k, every block update from the current values: the
            // H pass of component j also forms T_:jn, V_:jn for the next W update
            if (!ob || !ob->il) return cuda_fail(ctx, "interleaved scratch");
            if (it == 0 && (!il_begin(ctx, ob->il) ||
                            !launch_il_hpass(ctx, Bt, n, l, k, -1, 0, H, s.Wt, nullptr, 0.f, 0.f, s.T, s.V32, ob->il)))
                return cuda_fail(ctx, "T_1, V_1");
            for (int j = 0; j < k; ++j) {
                if (!launch_il_wpass(ctx, s.Qp, m, l, lp, k, j, Wc, s.Wt, s.T + (size_t)j * l, s.V32 + (size_t)j * k,
                                     s.q1, o.alpha_W, o.beta_W, o.gram_mode, s.S32 + (size_t)j * k, ob->il))
                    return cuda_fail(ctx, "W column");
                const int jn = j + 1 < k ? j + 1 : (it + 1 < iters ? 0 : -1);
                float* Tn = jn >= 0 ? s.T + (size_t)jn * l : nullptr;
                float* Vn = jn >= 0 ? s.V32 + (size_t)jn * k : nullptr;
                if (!launch_il_hpass(ctx, Bt, n, l, k, j, jn, H, s.Wt, s.S32 + (size_t)j * k, o.alpha_H, o.beta_H, Tn,
                                     Vn, ob->il))
                    return cuda_fail(ctx, "H row");
            }
        } else {
        if (shuffled && !order_sweep(ctx, *ob, o.order_seed, it, Wc, m, H, n, s.Wt, l, s.S32, s.S64, k))
            return cuda_fail(ctx, "shuffled order");
        // R^T (k x n) = (B^T W~)^T; H rows (Gauss-Seidel, clamp); T^T (k x l) = (B H^T)^T and
        // V = H H^T of the new H - on column tiles when their shared-memory plans fit
        const bool tiles = hhalf_fits(l, k);
        if (!(tch     ? tc_hhalf_r(ctx, s.tch, Bt, n, l, s.Wt, k, s.Rt)
              : tiles ? launch_rtile(ctx, Bt, n, l, s.Wt, k, s.Rt)
                      : launch_gemm_ax(ctx, Bt, l, s.Wt, k, 1, s.Rt, 1, n, n, k, l)))
            return cuda_fail(ctx, "R = B^T W~");
        if (!side_join(ctx, &s_pending)) return cuda_fail(ctx, "join S");
        if (!launch_hals_rows(ctx, H, 1, n, s.Rt, 1, n, s.S32, n, k, o.alpha_H, o.beta_H))
            return cuda_fail(ctx, "H update");
        if (tch) {
            if (!tc_hhalf_tv(ctx, s.tch, H, n, l, k, s.T, s.V32)) return cuda_fail(ctx, "T = B H^T, V = H H^T");
        } else if (tiles) {
            if (!launch_tv(ctx, Bt, n, l, H, k, s.T, s.V32, s.hh)) return cuda_fail(ctx, "T = B H^T, V = H H^T");
        } else {
            if (!launch_gemm_atx(ctx, Bt, l, H, 1, n, s.T, 1, l, l, k, n, s.atx)) return cuda_fail(ctx, "T = B H^T");
            if (!launch_gram(ctx, H, 1, n, n, k, s.V64, s.V32, s.gram)) return cuda_fail(ctx, "V = H H^T");
        }
        // f~ after the H half (W~ not yet updated)
        if (obj && !launch_compobj(ctx, Bt, n, l, s.Wt, k, H, s.obj + 4 * (size_t)it, s.objpart))
            return cuda_fail(ctx, "compressed objective");
        // W~ columns, reprojection W = max(0, Q W~), W~ = Q^T W
        if (!launch_whalf(ctx, s.Qp, m, l, lp, k, Wc, s.Wt, s.T, s.V32, s.wh, o.spin_limit, o.alpha_W, o.beta_W,
                          s.q1))
            return cuda_fail(ctx, "W half");
        // S for the next sweep (the shuffled order also permutes S's float64 copy: float32 products there)
        if (tch_s) {
            if (!gram_S_side(ctx, s, Wc, m, k)) return cuda_fail(ctx, "S = W^T W");
            s_pending = true;
        } else if (!gram_S(ctx, s, o.gram_mode, Wc, m, l, k)) {
            return cuda_fail(ctx, "S = W^T W");
        }
        }
        if (obj && !launch_compobj(ctx, Bt, n, l, s.Wt, k, H, s.obj + 4 * (size_t)it + 2, s.objpart))
            return cuda_fail(ctx, "compressed objective");
        if (ckpt && !save_state(ctx, ckpt, it + 1, Wc, s.Wt, H, m, n, l, k)) return cuda_fail(ctx, "checkpoint");
        if (o.track_every > 0 && A && ((it + 1) % o.track_every == 0 || it + 1 == iters)) {
            if (!launch_relerr(ctx, A, lda, Wc, 1, m, H, m, n, k, s.hist + 2 * (*ntracked), s.relerr))
                return cuda_fail(ctx, "relerr");
            ++*ntracked;
        }
        if (pg && ((it + 1) % every == 0 || it + 1 == iters)) {
            double v = 0.0;
            if (!pg_measure(ctx, s, Bt, m, n, l, lp, k, Wc, H, &v)) return cuda_fail(ctx, "projected gradient");
            if (pg_ratio) *pg_ratio = pg0 > 0.0 ? v / pg0 : 0.0;
            if (v <= o.pg_tol * pg0) {
                if (done) *done = it + 1;
                break;
            }
        }
    }
    if (shuffled && !order_end(ctx, *ob, Wc, m, H, n, s.Wt, l, s.S32, s.S64, k))
        return cuda_fail(ctx, "index order");
    return RNMF_OK;
}

bool order_ok(const rnmf_opts& o) {
    return o.order == RNMF_ORDER_CYCLIC || o.order == RNMF_ORDER_SHUFFLED || o.order == RNMF_ORDER_INTERLEAVED;
}
size_t order_reserve(rnmf_ctx* ctx, const rnmf_opts& o, int64_t m, int64_t n, int l, int k) {
    if (o.order == RNMF_ORDER_SHUFFLED) return arena_round(order_bytes(m, n, l, k));
    return o.order == RNMF_ORDER_INTERLEAVED ? arena_round(il_scratch_bytes(ctx)) : 0;
}

// the update order's buffers (none for the cyclic order)
OrderBufs order_bufs(rnmf_ctx* ctx, const rnmf_opts& o, int64_t m, int64_t n, int l, int k) {
    OrderBufs ob{};
    if (o.order == RNMF_ORDER_SHUFFLED) ob = order_take(ctx, m, n, l, k);
    if (o.order == RNMF_ORDER_INTERLEAVED) ob.il = (char*)arena_take(ctx, il_scratch_bytes(ctx));
    return ob;
}

void fill_hist(rnmf_ctx* ctx, const SweepBufs& s, int ntracked, int track_every, int iters, rnmf_stats* stats) {
    if (!stats) return;
    stats->final_rel_err = -1.0;
    if (ntracked <= 0) return;
    std::vector<double> h((size_t)ntracked * 2);
    cudaMemcpy(h.data(), s.hist, h.size() * 8, cudaMemcpyDeviceToHost);
    int nfull = iters / track_every;
    for (int i = 0; i < ntracked; ++i) {
        double r = h[2 * i + 1] > 0 ? std::sqrt(h[2 * i] / h[2 * i + 1]) : 0.0;
        if (stats->rel_err_hist && i < nfull) stats->rel_err_hist[i] = r;
        if (i == ntracked - 1) stats->final_rel_err = r;
    }
    (void)ctx;
}

bool wants_obj(const rnmf_stats* stats) { return stats && (stats->obj_hist || stats->obj_half_hist); }

// Per-sweep compressed objective into the caller's host arrays (sweeps [0, done)).
// The interleaved order has no H half: its obj_half_hist entries are NaN.
void fill_obj(const SweepBufs& s, int done, bool halves, rnmf_stats* stats) {
    if (!wants_obj(stats) || done <= 0) return;
    std::vector<double> h((size_t)done * 4);
    cudaMemcpy(h.data(), s.obj, h.size() * 8, cudaMemcpyDeviceToHost);
    for (int t = 0; t < done; ++t) {
        if (stats->obj_half_hist) stats->obj_half_hist[t] = halves ? h[4 * t] : std::nan("");
        if (stats->obj_hist) stats->obj_hist[t] = h[4 * t + 2];
    }
}

rnmf_status rnmf_device(rnmf_ctx* ctx, const float* A, int64_t m, int64_t n, int64_t lda, int k, int p, int q,
                        int iters, uint64_t seed, const rnmf_opts& o, float* W, float* H, rnmf_stats* stats) {
    const int l = k + p;
    const bool track = o.track_every > 0;
    size_t need = qb_bytes(ctx, m, n, l, o.precision) + arena_round((size_t)m * l * 4) +
                  arena_round((size_t)n * l * 4) + arena_round((size_t)k * m * 4) +
                  sweep_bytes(ctx, m, n, l, k, iters, track) + order_reserve(ctx, o, m, n, l, k) +
                  tch_reserve(ctx, o, m, n, l, k) + (o.init == RNMF_INIT_SVD ? svd_init_bytes(l, k) : 0);
    rnmf_status st = arena_reserve(ctx, need);
    if (st != RNMF_OK) return fail(ctx, st, "scratch allocation failed");
    if ((st = begin(ctx)) != RNMF_OK) return st;
    QbBufs qb = qb_take(ctx, m, n, l, o.precision);
    float* Q = (float*)arena_take(ctx, (size_t)m * l * 4);
    float* Bt = (float*)arena_take(ctx, (size_t)n * l * 4);
    float* Wc = (float*)arena_take(ctx, (size_t)k * m * 4);
    SweepBufs sb = sweep_take(ctx, m, n, l, k, iters, track);
    OrderBufs ob = order_bufs(ctx, o, m, n, l, k);
    tch_take(ctx, o, m, n, l, k, sb);

    cudaEventRecord(ctx->ev0, ctx->stream);
    if ((st = run_qb(ctx, qb, A, m, n, lda, l, q, seed, o, Q, Bt)) != RNMF_OK) return st;
    cudaEventRecord(ctx->ev1, ctx->stream);
    if (o.init == RNMF_INIT_SVD) {
        // NNDSVD of the randomized SVD (the QB's Gram scratch is free now)
        if (!launch_svd_init(ctx, Q, Bt, m, n, l, k, Wc, H, reinterpret_cast<double*>(qb.cq)))
            return cuda_fail(ctx, "SVD init");
    } else {
        // W_init (stored transposed) and H_init ~ U[0,1) from key seed + 1
        if (!launch_uniform_matrix(ctx, Wc, m, k, seed + 1, 2, 1, m)) return cuda_fail(ctx, "W_init");
        if (!launch_uniform_matrix(ctx, H, k, n, seed + 1, 3, n, 1)) return cuda_fail(ctx, "H_init");
    }
    // W~ = Q^T W_init; S from W_init
    if (!launch_gemm_atx(ctx, Q, l, Wc, 1, m, sb.Wt, k, 1, l, k, m, sb.atx)) return cuda_fail(ctx, "W~ = Q^T W");
    if (!gram_S(ctx, sb, o.gram_mode, Wc, m, l, k)) return cuda_fail(ctx, "S");
    int ntracked = 0, done = iters;
    double pgr = -1.0;
    if ((st = run_sweeps(ctx, sb, Q, Bt, m, n, l, k, iters, o, Wc, H, A, lda, &ntracked, nullptr, &done, &pgr,
                         &ob, wants_obj(stats))) != RNMF_OK)
        return st;
    if (!launch_transpose(ctx, Wc, k, m, W)) return cuda_fail(ctx, "transpose W");
    cudaEventRecord(ctx->ev2, ctx->stream);
    if ((st = finish(ctx, "rnmf")) != RNMF_OK) return st;
    if (stats) {
        cudaEventElapsedTime(&stats->ms_qb, ctx->ev0, ctx->ev1);
        cudaEventElapsedTime(&stats->ms_sweeps, ctx->ev1, ctx->ev2);
        stats->sweeps_done = done;
        stats->pg_ratio = pgr;
        fill_hist(ctx, sb, ntracked, o.track_every, done, stats);
        fill_obj(sb, done, o.order != RNMF_ORDER_INTERLEAVED, stats);
    }
    return RNMF_OK;
}

}  // namespace

// ===================================================================== ABI
extern "C" {

void rnmf_default_opts(rnmf_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = RNMF_PREC_FP32;
    o->gram_mode = 0;
    o->omega_dist = 0;
    o->track_every = 0;
    o->spin_limit = 0;
}

rnmf_status rnmf_create(rnmf_ctx** out, int device, void* cuda_stream) {
    if (!out) return RNMF_EINVAL;
    *out = nullptr;
    rnmf_ctx* ctx = new rnmf_ctx();
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return RNMF_ECUDA;
    }
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return RNMF_ECUDA;
        }
        ctx->own_stream = true;
    }
    if (cudaMalloc(&ctx->d_status, 256) != cudaSuccess || cudaMalloc(&ctx->d_bar, 256) != cudaSuccess ||
        cudaMalloc(&ctx->d_flags, 256) != cudaSuccess) {
        cudaGetLastError();
        rnmf_destroy(ctx);
        return RNMF_ENOMEM;
    }
    cudaMemset(ctx->d_status, 0, 256);
    cudaMemset(ctx->d_bar, 0, 256);
    cudaMemset(ctx->d_flags, 0, 256);
    cudaEventCreate(&ctx->ev0);
    cudaEventCreate(&ctx->ev1);
    cudaEventCreate(&ctx->ev2);
    *out = ctx;
    return RNMF_OK;
}

rnmf_status rnmf_destroy(rnmf_ctx* ctx) {
    if (!ctx) return RNMF_EINVAL;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    rb_plan_release(ctx);
    if (ctx->copy_stream) {
        cudaStreamSynchronize(ctx->copy_stream);
        cudaStreamDestroy(ctx->copy_stream);
    }
    for (auto e : ctx->copy_events)
        if (e) cudaEventDestroy(e);
    if (ctx->side_stream) {
        cudaStreamSynchronize(ctx->side_stream);
        cudaStreamDestroy(ctx->side_stream);
    }
    for (auto e : ctx->side_events)
        if (e) cudaEventDestroy(e);
    if (ctx->arena) cudaFree(ctx->arena);
    if (ctx->stage_A) cudaFree(ctx->stage_A);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->d_bar) cudaFree(ctx->d_bar);
    if (ctx->d_flags) cudaFree(ctx->d_flags);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->ev2) cudaEventDestroy(ctx->ev2);
    for (const ProfPending& p : ctx->pending) {
        ctx->ev_pool.push_back(p.a);
        ctx->ev_pool.push_back(p.b);
    }
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return RNMF_OK;
}

rnmf_status rnmf_set_scratch_limit(rnmf_ctx* ctx, size_t bytes) {
    if (!ctx) return RNMF_EINVAL;
    ctx->scratch_limit = bytes;
    return RNMF_OK;
}

size_t rnmf_scratch_bytes(rnmf_ctx* ctx) { return ctx ? scratch_held(ctx) : 0; }

const char* rnmf_last_error(rnmf_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

long long rnmf_kernel_launches(rnmf_ctx* ctx) { return ctx ? ctx->launches : 0; }

rnmf_status rnmf_profile(rnmf_ctx* ctx, int on) {
    if (!ctx) return RNMF_EINVAL;
    prof_resolve(ctx);
    if (on) {
        for (int c = 0; c < K_COUNT; ++c) {
            ctx->prof_launches[c] = 0;
            ctx->prof_ms[c] = ctx->prof_bytes[c] = ctx->prof_flops[c] = 0.0;
        }
    }
    ctx->prof_on = on != 0;
    return RNMF_OK;
}

int rnmf_profile_read(rnmf_ctx* ctx, rnmf_kernel_prof* out, int max) {
    if (!ctx || !out) return 0;
    prof_resolve(ctx);
    int n = 0;
    for (int c = 0; c < K_COUNT && n < max; ++c) {
        if (ctx->prof_launches[c] == 0) continue;
        out[n].name = kClassNames[c];
        out[n].launches = ctx->prof_launches[c];
        out[n].ms = ctx->prof_ms[c];
        out[n].bytes = ctx->prof_bytes[c];
        out[n].flops = ctx->prof_flops[c];
        ++n;
    }
    return n;
}

rnmf_status rnmf(rnmf_ctx* ctx, const float* A, int64_t m, int64_t n, int64_t lda, int k, int p, int q, int iters,
                 uint64_t seed, const rnmf_opts* opts, float* W, float* H, rnmf_stats* stats) {
    if (!ctx) return RNMF_EINVAL;
    rnmf_status st = check_shape(ctx, m, n, lda, k, p);
    if (st != RNMF_OK) return st;
    if (!A || !W || !H) return fail(ctx, RNMF_EINVAL, "null pointer");
    if (q < 0 || iters < 0) return fail(ctx, RNMF_EINVAL, "q < 0 or iters < 0");
    rnmf_opts o = opts_or_default(opts);
    if (o.precision < 0 || o.precision > 2 || o.gram_mode < 0 || o.gram_mode > 1 || o.omega_dist < 0 ||
        o.omega_dist > 1 || o.track_every < 0 || !penalties_ok(o) || !order_ok(o) || o.init < 0 || o.init > 1 ||
        !sweep_products_ok(o))
        return fail(ctx, RNMF_EINVAL, "bad option");
    if ((st = check_tc(ctx, A, lda, o.precision)) != RNMF_OK) return st;
    return rnmf_device(ctx, A, m, n, lda, k, p, q, iters, seed, o, W, H, stats);
}

rnmf_status rnmf_host(rnmf_ctx* ctx, const float* A_host, int64_t m, int64_t n, int64_t lda, int k, int p, int q,
                      int iters, uint64_t seed, const rnmf_opts* opts, float* W_host, float* H_host,
                      rnmf_stats* stats) {
    if (!ctx) return RNMF_EINVAL;
    rnmf_status st = check_shape(ctx, m, n, lda, k, p);
    if (st != RNMF_OK) return st;
    if (!A_host || !W_host || !H_host) return fail(ctx, RNMF_EINVAL, "null pointer");
    if (q < 0 || iters < 0) return fail(ctx, RNMF_EINVAL, "q < 0 or iters < 0");
    rnmf_opts o = opts_or_default(opts);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, "cudaSetDevice");
    size_t abytes = (size_t)m * n * 4, wbytes = (size_t)m * k * 4, hbytes = (size_t)k * n * 4;
    size_t need = arena_round(abytes) + arena_round(wbytes) + arena_round(hbytes);
    if (ctx->stage_A_bytes < need) {
        if (!scratch_fits(ctx, scratch_held(ctx) - ctx->stage_A_bytes + need))
            return fail(ctx, RNMF_ENOMEM, "staging of A exceeds the context's scratch limit");
        if (ctx->stage_A) cudaFree(ctx->stage_A);
        ctx->stage_A = nullptr;
        ctx->stage_A_bytes = 0;
        if (cudaMalloc(&ctx->stage_A, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, RNMF_ENOMEM, "staging allocation failed");
        }
        ctx->stage_A_bytes = need;
    }
    float* dA = ctx->stage_A;
    float* dW = (float*)((char*)ctx->stage_A + arena_round(abytes));
    float* dH = (float*)((char*)dW + arena_round(wbytes));
    // pinned host memory: the GPU pulls A itself (many loads in flight over the
    // host link); pageable memory: the copy engine
    if (const float* Adev = host_device_view(A_host)) {
        if (!launch_pull_rows(ctx, ctx->stream, Adev, lda, m, n, dA)) return cuda_fail(ctx, "pull A to device");
    } else if (cudaMemcpy2DAsync(dA, n * 4, A_host, lda * 4, n * 4, m, cudaMemcpyHostToDevice, ctx->stream) !=
               cudaSuccess) {
        return cuda_fail(ctx, "copy A to device");
    }
    st = rnmf(ctx, dA, m, n, n, k, p, q, iters, seed, &o, dW, dH, stats);
    if (st != RNMF_OK) return st;
    if (cudaMemcpyAsync(W_host, dW, wbytes, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(H_host, dH, hbytes, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
        return cuda_fail(ctx, "copy W, H to host");
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_fail(ctx, "rnmf_host");
    return RNMF_OK;
}

rnmf_status rnmf_qb(rnmf_ctx* ctx, const float* A, int64_t m, int64_t n, int64_t lda, int l, int q, uint64_t seed,
                    const rnmf_opts* opts, float* Q, float* Bt) {
    if (!ctx) return RNMF_EINVAL;
    rnmf_status st = check_shape(ctx, m, n, lda, l, 0);
    if (st != RNMF_OK) return st;
    if (!A || !Q || !Bt) return fail(ctx, RNMF_EINVAL, "null pointer");
    if (q < 0) return fail(ctx, RNMF_EINVAL, "q < 0");
    rnmf_opts o = opts_or_default(opts);
    if (o.precision < 0 || o.precision > 2 || o.omega_dist < 0 || o.omega_dist > 1)
        return fail(ctx, RNMF_EINVAL, "bad option");
    if ((st = check_tc(ctx, A, lda, o.precision)) != RNMF_OK) return st;
    if ((st = arena_reserve(ctx, qb_bytes(ctx, m, n, l, o.precision))) != RNMF_OK)
        return fail(ctx, st, "scratch allocation failed");
    if ((st = begin(ctx)) != RNMF_OK) return st;
    QbBufs qb = qb_take(ctx, m, n, l, o.precision);
    if ((st = run_qb(ctx, qb, A, m, n, lda, l, q, seed, o, Q, Bt)) != RNMF_OK) return st;
    return finish(ctx, "rnmf_qb");
}

rnmf_status rnmf_sweeps(rnmf_ctx* ctx, const float* Q, const float* Bt, int64_t m, int64_t n, int l, int k,
                        int iters, const rnmf_opts* opts, float* W, float* H, float* Wt, const float* A, int64_t lda,
                        rnmf_stats* stats) {
    if (!ctx) return RNMF_EINVAL;
    if (m < 1 || n < 1 || k < 1 || l < k || l > RNMF_MAX_L || iters < 0)
        return fail(ctx, RNMF_EINVAL, "bad sizes");
    if (!Q || !Bt || !W || !H) return fail(ctx, RNMF_EINVAL, "null pointer");
    rnmf_opts o = opts_or_default(opts);
    if (!penalties_ok(o)) return fail(ctx, RNMF_EINVAL, "penalties must be finite and >= 0");
    if (!order_ok(o)) return fail(ctx, RNMF_EINVAL, "bad update order");
    if (!sweep_products_ok(o)) return fail(ctx, RNMF_EINVAL, "bad sweep_products");
    if (o.track_every > 0 && (!A || lda < n)) return fail(ctx, RNMF_EINVAL, "tracking needs A");
    const bool track = o.track_every > 0;
    size_t need = arena_round((size_t)k * m * 4) + sweep_bytes(ctx, m, n, l, k, iters, track) +
                  order_reserve(ctx, o, m, n, l, k) + tch_reserve(ctx, o, m, n, l, k);
    rnmf_status st = arena_reserve(ctx, need);
    if (st != RNMF_OK) return fail(ctx, st, "scratch allocation failed");
    if ((st = begin(ctx)) != RNMF_OK) return st;
    float* Wc = (float*)arena_take(ctx, (size_t)k * m * 4);
    SweepBufs sb = sweep_take(ctx, m, n, l, k, iters, track);
    OrderBufs ob = order_bufs(ctx, o, m, n, l, k);
    tch_take(ctx, o, m, n, l, k, sb);
    if (!launch_transpose(ctx, W, m, k, Wc)) return cuda_fail(ctx, "transpose W");
    if (Wt) {
        if (cudaMemcpyAsync(sb.Wt, Wt, (size_t)l * k * 4, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
            return cuda_fail(ctx, "copy Wt");
    } else if (!launch_gemm_atx(ctx, Q, l, Wc, 1, m, sb.Wt, k, 1, l, k, m, sb.atx)) {
        return cuda_fail(ctx, "W~ = Q^T W");
    }
    if (!gram_S(ctx, sb, o.gram_mode, Wc, m, l, k)) return cuda_fail(ctx, "S");
    cudaEventRecord(ctx->ev1, ctx->stream);
    int ntracked = 0, done = iters;
    double pgr = -1.0;
    if ((st = run_sweeps(ctx, sb, Q, Bt, m, n, l, k, iters, o, Wc, H, A, lda, &ntracked, nullptr, &done, &pgr,
                         &ob, wants_obj(stats))) != RNMF_OK)
        return st;
    if (!launch_transpose(ctx, Wc, k, m, W)) return cuda_fail(ctx, "transpose W");
    if (Wt && cudaMemcpyAsync(Wt, sb.Wt, (size_t)l * k * 4, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
        return cuda_fail(ctx, "copy Wt");
    cudaEventRecord(ctx->ev2, ctx->stream);
    if ((st = finish(ctx, "rnmf_sweeps")) != RNMF_OK) return st;
    if (stats) {
        stats->ms_qb = 0.f;
        cudaEventElapsedTime(&stats->ms_sweeps, ctx->ev1, ctx->ev2);
        stats->sweeps_done = done;
        stats->pg_ratio = pgr;
        fill_hist(ctx, sb, ntracked, o.track_every, done, stats);
        fill_obj(sb, done, o.order != RNMF_ORDER_INTERLEAVED, stats);
    }
    return RNMF_OK;
}

rnmf_status rnmf_qb_streamed(rnmf_ctx* ctx, const float* A_host, int64_t m, int64_t n, int64_t lda, int l, int q,
                             uint64_t seed, const rnmf_opts* opts, int64_t block_cols, float* Q, float* Bt) {
    if (!ctx) return RNMF_EINVAL;
    if (m < 1 || n < 1 || lda < n || l < 1 || l > RNMF_MAX_L || l > m || l > n || q < 0 || !A_host || !Q || !Bt)
        return fail(ctx, RNMF_EINVAL, "bad argument");
    rnmf_opts o = opts_or_default(opts);
    if (o.omega_dist < 0 || o.omega_dist > 1 || o.precision < 0 || o.precision > 2)
        return fail(ctx, RNMF_EINVAL, "bad option");
    if (o.precision != RNMF_PREC_FP32 && !tc_available())
        return fail(ctx, RNMF_ENOTIMPL, "tensor-core forms unavailable (no TMA descriptor entry point)");
    const int64_t bc = streamed_block_cols(m, n, block_cols);
    rnmf_status st = arena_reserve(ctx, streamed_qb_bytes(ctx, m, n, l, bc, o.precision));
    if (st != RNMF_OK) return fail(ctx, st, "scratch allocation failed");
    if ((st = begin(ctx)) != RNMF_OK) return st;
    if ((st = run_qb_streamed(ctx, A_host, m, n, lda, l, q, seed, o.omega_dist, bc, o.precision, Q, Bt)) != RNMF_OK)
        return st;
    return finish(ctx, "rnmf_qb_streamed");
}

rnmf_status rnmf_streamed(rnmf_ctx* ctx, const float* A_host, int64_t m, int64_t n, int64_t lda, int k, int p, int q,
                          int iters, uint64_t seed, const rnmf_opts* opts, int64_t block_cols, float* W, float* H,
                          rnmf_stats* stats) {
    if (!ctx) return RNMF_EINVAL;
    const int64_t l = (int64_t)k + p;
    if (m < 1 || n < 1 || lda < n || k < 1 || p < 0 || q < 0 || iters < 0 || l > RNMF_MAX_L || l > m || l > n ||
        !A_host || !W || !H)
        return fail(ctx, RNMF_EINVAL, "bad argument");
    rnmf_opts o = opts_or_default(opts);
    if (o.precision < 0 || o.precision > 2 || o.track_every != 0 || o.gram_mode < 0 || o.gram_mode > 1 ||
        o.omega_dist < 0 || o.omega_dist > 1 || !penalties_ok(o) || !order_ok(o) || o.init != RNMF_INIT_UNIFORM ||
        !sweep_products_ok(o))
        return fail(ctx, RNMF_EINVAL, "bad option (the streamed path cannot track the error; uniform init)");
    if (o.precision != RNMF_PREC_FP32 && !tc_available())
        return fail(ctx, RNMF_ENOTIMPL, "tensor-core forms unavailable (no TMA descriptor entry point)");
    const int64_t bc = streamed_block_cols(m, n, block_cols);
    size_t need = streamed_qb_bytes(ctx, m, n, (int)l, bc, o.precision) + arena_round((size_t)m * l * 4) +
                  arena_round((size_t)n * l * 4) + arena_round((size_t)k * m * 4) +
                  sweep_bytes(ctx, m, n, (int)l, k, iters, false) + order_reserve(ctx, o, m, n, (int)l, k) +
                  tch_reserve(ctx, o, m, n, (int)l, k);
    rnmf_status st = arena_reserve(ctx, need);
    if (st != RNMF_OK) return fail(ctx, st, "scratch allocation failed");
    if ((st = begin(ctx)) != RNMF_OK) return st;
    float* Q = (float*)arena_take(ctx, (size_t)m * l * 4);
    float* Bt = (float*)arena_take(ctx, (size_t)n * l * 4);
    float* Wc = (float*)arena_take(ctx, (size_t)k * m * 4);
    SweepBufs sb = sweep_take(ctx, m, n, (int)l, k, iters, false);
    OrderBufs ob = order_bufs(ctx, o, m, n, (int)l, k);
    tch_take(ctx, o, m, n, (int)l, k, sb);
    cudaEventRecord(ctx->ev0, ctx->stream);
    if ((st = run_qb_streamed(ctx, A_host, m, n, lda, (int)l, q, seed, o.omega_dist, bc, o.precision, Q, Bt)) !=
        RNMF_OK)
        return st;
    cudaEventRecord(ctx->ev1, ctx->stream);
    if (!launch_uniform_matrix(ctx, Wc, m, k, seed + 1, 2, 1, m)) return cuda_fail(ctx, "W_init");
    if (!launch_uniform_matrix(ctx, H, k, n, seed + 1, 3, n, 1)) return cuda_fail(ctx, "H_init");
    if (!launch_gemm_atx(ctx, Q, l, Wc, 1, m, sb.Wt, k, 1, l, k, m, sb.atx)) return cuda_fail(ctx, "W~ = Q^T W");
    if (!gram_S(ctx, sb, o.gram_mode, Wc, m, (int)l, k)) return cuda_fail(ctx, "S");
    int ntracked = 0, done = iters;
    double pgr = -1.0;
    if ((st = run_sweeps(ctx, sb, Q, Bt, m, n, (int)l, k, iters, o, Wc, H, nullptr, n, &ntracked, nullptr, &done,
                         &pgr, &ob, wants_obj(stats))) != RNMF_OK)
        return st;
    if (!launch_transpose(ctx, Wc, k, m, W)) return cuda_fail(ctx, "transpose W");
    cudaEventRecord(ctx->ev2, ctx->stream);
    if ((st = finish(ctx, "rnmf_streamed")) != RNMF_OK) return st;
    if (stats) {
        cudaEventElapsedTime(&stats->ms_qb, ctx->ev0, ctx->ev1);
        cudaEventElapsedTime(&stats->ms_sweeps, ctx->ev1, ctx->ev2);
        stats->sweeps_done = done;
        stats->pg_ratio = pgr;
        stats->final_rel_err = -1.0;
        fill_obj(sb, done, o.order != RNMF_ORDER_INTERLEAVED, stats);
    }
    return RNMF_OK;
}

rnmf_status rnmf_projected_gradient(rnmf_ctx* ctx, const float* Q, const float* Bt, int64_t m, int64_t n, int l,
                                    int k, const float* W, const float* H, double* out) {
    if (!ctx) return RNMF_EINVAL;
    if (m < 1 || n < 1 || k < 1 || l < k || l > RNMF_MAX_L || !Q || !Bt || !W || !H || !out)
        return fail(ctx, RNMF_EINVAL, "bad argument");
    size_t need = arena_round((size_t)k * m * 4) + sweep_bytes(ctx, m, n, l, k, 0, false);
    rnmf_status st = arena_reserve(ctx, need);
    if (st != RNMF_OK) return fail(ctx, st, "scratch allocation failed");
    if ((st = begin(ctx)) != RNMF_OK) return st;
    float* Wc = (float*)arena_take(ctx, (size_t)k * m * 4);
    SweepBufs sb = sweep_take(ctx, m, n, l, k, 0, false);
    const int lp = (l + 3) / 4 * 4;
    if (!launch_transpose(ctx, W, m, k, Wc)) return cuda_fail(ctx, "transpose W");
    if (!launch_gemm_atx(ctx, Q, l, Wc, 1, m, sb.Wt, k, 1, l, k, m, sb.atx)) return cuda_fail(ctx, "W~ = Q^T W");
    if (!launch_pad_rows(ctx, Q, m, l, lp, sb.Qp)) return cuda_fail(ctx, "pad Q");
    if (!pg_measure(ctx, sb, Bt, m, n, l, lp, k, Wc, H, out)) return cuda_fail(ctx, "projected gradient");
    return finish(ctx, "rnmf_projected_gradient");
}

size_t rnmf_ckpt_floats(int64_t m, int64_t n, int l, int k, int T) {
    return (size_t)(T + 1) * adjoint_ckpt_floats(m, n, l, k);
}

rnmf_status rnmf_sweeps_fwd(rnmf_ctx* ctx, const float* Q, const float* Bt, int64_t m, int64_t n, int l, int k, int T,
                            const rnmf_opts* opts, float* W, float* H, float* ckpt) {
    if (!ctx) return RNMF_EINVAL;
    if (m < 1 || n < 1 || k < 1 || l < k || l > RNMF_MAX_L || T < 0) return fail(ctx, RNMF_EINVAL, "bad sizes");
    if (!Q || !Bt || !W || !H) return fail(ctx, RNMF_EINVAL, "null pointer");
    rnmf_opts o = opts_or_default(opts);
    o.track_every = 0;
    if (has_penalties(o) || o.order != RNMF_ORDER_CYCLIC)
        return fail(ctx, RNMF_EINVAL, "the adjoint differentiates the unpenalised cyclic sweeps");
    size_t need = arena_round((size_t)k * m * 4) + sweep_bytes(ctx, m, n, l, k, T, false);
    rnmf_status st = arena_reserve(ctx, need);
    if (st != RNMF_OK) return fail(ctx, st, "scratch allocation failed");
    if ((st = begin(ctx)) != RNMF_OK) return st;
    float* Wc = (float*)arena_take(ctx, (size_t)k * m * 4);
    SweepBufs sb = sweep_take(ctx, m, n, l, k, T, false);
    if (!launch_transpose(ctx, W, m, k, Wc)) return cuda_fail(ctx, "transpose W");
    if (!launch_gemm_atx(ctx, Q, l, Wc, 1, m, sb.Wt, k, 1, l, k, m, sb.atx)) return cuda_fail(ctx, "W~ = Q^T W");
    if (!gram_S(ctx, sb, o.gram_mode, Wc, m, l, k)) return cuda_fail(ctx, "S");
    if (ckpt && !save_state(ctx, ckpt, 0, Wc, sb.Wt, H, m, n, l, k)) return cuda_fail(ctx, "checkpoint");
    int ntracked = 0;
    if ((st = run_sweeps(ctx, sb, Q, Bt, m, n, l, k, T, o, Wc, H, nullptr, n, &ntracked, ckpt)) != RNMF_OK) return st;
    if (!launch_transpose(ctx, Wc, k, m, W)) return cuda_fail(ctx, "transpose W");
    return finish(ctx, "rnmf_sweeps_fwd");
}

rnmf_status rnmf_sweeps_bwd(rnmf_ctx* ctx, const float* Q, const float* Bt, int64_t m, int64_t n, int l, int k, int T,
                            const rnmf_opts* opts, const float* ckpt, const float* dW_T, const float* dH_T, float* dBt,
                            float* dW_init, float* dH_init) {
    if (!ctx) return RNMF_EINVAL;
    if (m < 1 || n < 1 || k < 1 || l < k || l > RNMF_MAX_L || T < 0) return fail(ctx, RNMF_EINVAL, "bad sizes");
    if (5LL * l * k + 2LL * k * k > 56000) return fail(ctx, RNMF_EINVAL, "adjoint needs 5 l k + 2 k^2 <= 56000");
    if (!Q || !Bt || !ckpt || !dW_T || !dH_T || !dBt || !dW_init || !dH_init) return fail(ctx, RNMF_EINVAL, "null pointer");
    rnmf_opts o = opts_or_default(opts);
    if (has_penalties(o) || o.order != RNMF_ORDER_CYCLIC)
        return fail(ctx, RNMF_EINVAL, "the adjoint differentiates the unpenalised cyclic sweeps");
    const int64_t big = m > n ? m : n;
    size_t atx = 0;
    const int64_t shapes[][3] = {{l, k, n}, {n, k, k}, {n, l, k}, {k, k, n}, {l, k, n}, {m, k, k}};
    for (auto& sh : shapes) {
        size_t b = gemm_atx_scratch_bytes(ctx, sh[0], (int)sh[1], sh[2]);
        if (b > atx) atx = b;
    }
    const size_t fk = (size_t)k * k * 4;
    size_t need = 2 * arena_round((size_t)k * m * 4) + 2 * arena_round((size_t)l * k * 4) +
                  2 * arena_round((size_t)k * n * 4) + 3 * arena_round((size_t)l * k * 4) + 8 * arena_round(fk) +
                  2 * arena_round(fk * 2) + arena_round((size_t)n * k * 4) + arena_round(gram_scratch_bytes(ctx, big, k)) +
                  arena_round(atx + 8) + arena_round(wrev_scratch_bytes(ctx, m));
    rnmf_status st = arena_reserve(ctx, need);
    if (st != RNMF_OK) return fail(ctx, st, "scratch allocation failed");
    if ((st = begin(ctx)) != RNMF_OK) return st;
    float* dWc[2] = {(float*)arena_take(ctx, (size_t)k * m * 4), (float*)arena_take(ctx, (size_t)k * m * 4)};
    float* dWt[2] = {(float*)arena_take(ctx, (size_t)l * k * 4), (float*)arena_take(ctx, (size_t)l * k * 4)};
    float* dH[2] = {(float*)arena_take(ctx, (size_t)k * n * 4), (float*)arena_take(ctx, (size_t)k * n * 4)};
    float* Tm = (float*)arena_take(ctx, (size_t)l * k * 4);
    float* dT = (float*)arena_take(ctx, (size_t)l * k * 4);
    float* spare = (float*)arena_take(ctx, (size_t)l * k * 4);
    (void)spare;
    float* V32 = (float*)arena_take(ctx, fk);
    float* S32 = (float*)arena_take(ctx, fk);
    float* dV = (float*)arena_take(ctx, fk);
    float* dVsym = (float*)arena_take(ctx, fk);
    float* P1T = (float*)arena_take(ctx, fk);
    float* P0T = (float*)arena_take(ctx, fk);
    float* dSsym = (float*)arena_take(ctx, fk);
    (void)arena_take(ctx, fk);
    double* V64 = (double*)arena_take(ctx, fk * 2);
    double* S64 = (double*)arena_take(ctx, fk * 2);
    float* DA = (float*)arena_take(ctx, (size_t)n * k * 4);
    double* gram = (double*)arena_take(ctx, gram_scratch_bytes(ctx, big, k));
    double* atxs = (double*)arena_take(ctx, atx + 8);
    char* wrs = (char*)arena_take(ctx, wrev_scratch_bytes(ctx, m));
    const size_t SZ = adjoint_ckpt_floats(m, n, l, k);
    int cur = 0;
    // seeds: dW_T (stored transposed), dW~_T = 0, dH_T; dB^T = 0
    if (!launch_transpose(ctx, dW_T, m, k, dWc[cur])) return cuda_fail(ctx, "transpose dW");
    if (cudaMemsetAsync(dWt[cur], 0, (size_t)l * k * 4, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(dH[cur], dH_T, (size_t)k * n * 4, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess ||
        cudaMemsetAsync(dBt, 0, (size_t)n * l * 4, ctx->stream) != cudaSuccess)
        return cuda_fail(ctx, "init adjoint");
    for (int t = T; t >= 1; --t) {
        const float* Wc_o = ckpt + (size_t)(t - 1) * SZ;
        const float* Wt_o = Wc_o + (size_t)k * m;
        const float* H_o = Wt_o + (size_t)l * k;
        const float* Wc_n = ckpt + (size_t)t * SZ;
        const float* Wt_n = Wc_n + (size_t)k * m;
        const float* H_n = Wt_n + (size_t)l * k;
        const int nx = cur ^ 1;
        // --- W half (reverse): T = B H_t^T, V = H_t H_t^T recomputed
        if (!launch_gemm_atx(ctx, Bt, l, H_n, 1, n, Tm, k, 1, l, k, n, atxs)) return cuda_fail(ctx, "T");
        if (!launch_gram(ctx, H_n, 1, n, n, k, V64, V32, gram)) return cuda_fail(ctx, "V");
        if (!launch_wrev(ctx, Q, m, l, k, Wt_n, Wt_o, Wc_n, dWc[cur], dWt[cur], Tm, V32, dT, dV, dWt[nx], dWc[nx], wrs,
                         o.spin_limit))
            return cuda_fail(ctx, "W half reverse");
        // dH_t += B^T dT (as (n x k) = Bt dT) and += H_t^T (dV + dV^T)
        if (!launch_gemm_ax(ctx, Bt, l, dT, k, 1, dH[cur], 1, n, n, k, l, true)) return cuda_fail(ctx, "dH += B^T dT");
        if (!launch_sym(ctx, dV, nullptr, k, dVsym)) return cuda_fail(ctx, "dV sym");
        if (!launch_gemm_atx(ctx, H_n, n, dVsym, k, 1, dH[cur], 1, n, n, k, k, atxs, true)) return cuda_fail(ctx, "dH += dV H");
        // dB^T += H_t^T dT^T
        if (!launch_gemm_atx(ctx, H_n, n, dT, 1, k, dBt, l, 1, n, l, k, atxs, true)) return cuda_fail(ctx, "dB += dT H");
        // --- H half (reverse): S from the state before the sweep
        if (!gram_S_from(ctx, o.gram_mode, Wc_o, Wt_o, m, l, k, S64, S32, gram)) return cuda_fail(ctx, "S");
        if (!launch_hrev(ctx, H_o, H_n, dH[cur], S32, n, k, dH[nx], DA)) return cuda_fail(ctx, "H half reverse");
        // dS from DA: P1 = H_t DA, P0 = H_{t-1} DA (transposed products)
        if (!launch_gemm_atx(ctx, DA, k, H_n, 1, n, P1T, k, 1, k, k, n, atxs)) return cuda_fail(ctx, "P1");
        if (!launch_gemm_atx(ctx, DA, k, H_o, 1, n, P0T, k, 1, k, k, n, atxs)) return cuda_fail(ctx, "P0");
        if (!launch_sym(ctx, P1T, P0T, k, dSsym)) return cuda_fail(ctx, "dS");
        // R = B^T W~_{t-1}: dW~_{t-1} += B dR = Bt^T DA; dB^T += DA W~_{t-1}^T
        if (!launch_gemm_atx(ctx, Bt, l, DA, k, 1, dWt[nx], k, 1, l, k, n, atxs, true)) return cuda_fail(ctx, "dW~ += B dR");
        if (!launch_gemm_ax(ctx, DA, k, Wt_o, 1, k, dBt, l, 1, n, l, k, true)) return cuda_fail(ctx, "dB += dR W~");
        // S = W^T W: dW_{t-1} += W (dS + dS^T) (stored transposed); or S = W~^T W~
        if (o.gram_mode == 0) {
            if (!launch_gemm_atx(ctx, Wc_o, m, dSsym, k, 1, dWc[nx], 1, m, m, k, k, atxs, true))
                return cuda_fail(ctx, "dW += W dS");
        } else {
            if (!launch_gemm_ax(ctx, Wt_o, k, dSsym, k, 1, dWt[nx], k, 1, l, k, k, true))
                return cuda_fail(ctx, "dW~ += W~ dS");
        }
        cur = nx;
    }
    // W~_0 = Q^T W_init: dW_init += Q dW~_0
    if (!launch_gemm_ax(ctx, Q, l, dWt[cur], k, 1, dWc[cur], 1, m, m, k, l, true)) return cuda_fail(ctx, "dW0 += Q dW~0");
    if (!launch_transpose(ctx, dWc[cur], k, m, dW_init)) return cuda_fail(ctx, "transpose dW0");
    if (cudaMemcpyAsync(dH_init, dH[cur], (size_t)k * n * 4, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
        return cuda_fail(ctx, "copy dH0");
    return finish(ctx, "rnmf_sweeps_bwd");
}

rnmf_status rnmf_dA(rnmf_ctx* ctx, const float* Q, const float* dBt, int64_t m, int64_t n, int l, float* dA) {
    if (!ctx) return RNMF_EINVAL;
    if (m < 1 || n < 1 || l < 1 || !Q || !dBt || !dA) return fail(ctx, RNMF_EINVAL, "bad argument");
    rnmf_status st = begin(ctx);
    if (st != RNMF_OK) return st;
    if (!launch_outer(ctx, Q, dBt, m, n, l, dA)) return cuda_fail(ctx, "dA = Q dB");
    return finish(ctx, "rnmf_dA");
}

rnmf_status rnmf_hals(rnmf_ctx* ctx, const float* A, int64_t m, int64_t n, int64_t lda, int k, int iters,
                      uint64_t seed, const rnmf_opts* opts, float* W, float* H, rnmf_stats* stats) {
    if (!ctx) return RNMF_EINVAL;
    rnmf_status st = check_shape(ctx, m, n, lda, k, 0);
    if (st != RNMF_OK) return st;
    if (!A || !W || !H) return fail(ctx, RNMF_EINVAL, "null pointer");
    if (iters < 0) return fail(ctx, RNMF_EINVAL, "iters < 0");
    rnmf_opts o = opts_or_default(opts);
    if (!penalties_ok(o)) return fail(ctx, RNMF_EINVAL, "penalties must be finite and >= 0");
    if (o.order != RNMF_ORDER_CYCLIC || o.init != RNMF_INIT_UNIFORM)
        return fail(ctx, RNMF_EINVAL, "deterministic HALS runs the cyclic order from uniform factors");
    const bool track = o.track_every > 0;
    int64_t big = m > n ? m : n;
    size_t a1 = gemm_atx_scratch_bytes(ctx, n, k, m), a2 = gemm_ax_scratch_bytes(ctx, m, k, n);
    if (a2 > a1) a1 = a2;
    size_t need = arena_round((size_t)k * n * 4) + arena_round((size_t)m * k * 4) + 2 * arena_round((size_t)k * k * 4) +
                  2 * arena_round((size_t)k * k * 8) + arena_round(gram_scratch_bytes(ctx, big, k)) +
                  arena_round(a1 + 8) + arena_round(track ? relerr_scratch_bytes(ctx, m, n) : 8) +
                  arena_round((size_t)(iters + 1) * 16);
    if ((st = arena_reserve(ctx, need)) != RNMF_OK) return fail(ctx, st, "scratch allocation failed");
    if ((st = begin(ctx)) != RNMF_OK) return st;
    float* Rt = (float*)arena_take(ctx, (size_t)k * n * 4);
    float* P = (float*)arena_take(ctx, (size_t)m * k * 4);
    float* S32 = (float*)arena_take(ctx, (size_t)k * k * 4);
    float* V32 = (float*)arena_take(ctx, (size_t)k * k * 4);
    double* S64 = (double*)arena_take(ctx, (size_t)k * k * 8);
    double* V64 = (double*)arena_take(ctx, (size_t)k * k * 8);
    double* gram = (double*)arena_take(ctx, gram_scratch_bytes(ctx, big, k));
    double* atx = (double*)arena_take(ctx, a1 + 8);
    double* rel = (double*)arena_take(ctx, track ? relerr_scratch_bytes(ctx, m, n) : 8);
    double* hist = (double*)arena_take(ctx, (size_t)(iters + 1) * 16);

    cudaEventRecord(ctx->ev1, ctx->stream);
    if (!launch_uniform_matrix(ctx, W, m, k, seed + 1, 2, k, 1)) return cuda_fail(ctx, "W_init");
    if (!launch_uniform_matrix(ctx, H, k, n, seed + 1, 3, n, 1)) return cuda_fail(ctx, "H_init");
    int ntracked = 0;
    for (int it = 0; it < iters; ++it) {
        // H rows: R = A^T W, S = W^T W
        if (!launch_gemm_atx(ctx, A, lda, W, k, 1, Rt, 1, n, n, k, m, atx)) return cuda_fail(ctx, "A^T W");
        if (!launch_gram(ctx, W, k, 1, m, k, S64, S32, gram)) return cuda_fail(ctx, "W^T W");
        if (!launch_hals_rows(ctx, H, 1, n, Rt, 1, n, S32, n, k, o.alpha_H, o.beta_H))
            return cuda_fail(ctx, "H update");
        // W columns: P = A H^T, V = H H^T; rows of W are independent
        if (!launch_gemm_ax(ctx, A, lda, H, 1, n, P, k, 1, m, k, n, false, atx)) return cuda_fail(ctx, "A H^T");
        if (!launch_gram(ctx, H, 1, n, n, k, V64, V32, gram)) return cuda_fail(ctx, "H H^T");
        if (!launch_hals_rows(ctx, W, k, 1, P, k, 1, V32, m, k, o.alpha_W, o.beta_W))
            return cuda_fail(ctx, "W update");
        if (track && ((it + 1) % o.track_every == 0 || it + 1 == iters)) {
            if (!launch_relerr(ctx, A, lda, W, k, 1, H, m, n, k, hist + 2 * ntracked, rel))
                return cuda_fail(ctx, "relerr");
            ++ntracked;
        }
    }
    cudaEventRecord(ctx->ev2, ctx->stream);
    if ((st = finish(ctx, "rnmf_hals")) != RNMF_OK) return st;
    if (stats) {
        stats->ms_qb = 0.f;
        cudaEventElapsedTime(&stats->ms_sweeps, ctx->ev1, ctx->ev2);
        stats->sweeps_done = iters;
        stats->pg_ratio = -1.0;
        SweepBufs sb{};
        sb.hist = hist;
        fill_hist(ctx, sb, ntracked, o.track_every, iters, stats);
    }
    return RNMF_OK;
}

rnmf_status rnmf_sketch(rnmf_ctx* ctx, const float* A, int64_t m, int64_t n, int64_t lda, const float* X, int l,
                        int transpose, int form, float* out) {
    if (!ctx) return RNMF_EINVAL;
    if (m < 1 || n < 1 || lda < n || l < 1 || l > RNMF_MAX_L || !A || !X || !out || transpose < 0 || transpose > 1 ||
        form < 0 || form > 2)
        return fail(ctx, RNMF_EINVAL, "bad argument");
    rnmf_status st = check_tc(ctx, A, lda, form);
    if (st != RNMF_OK) return st;
    size_t a1 = gemm_atx_scratch_bytes(ctx, n, l, m), a2 = gemm_ax_scratch_bytes(ctx, m, l, n);
    if (a2 > a1) a1 = a2;
    if ((st = arena_reserve(ctx, arena_round(a1 + 8) + tc_scratch_bytes(ctx, m, n, l, form))) != RNMF_OK)
        return fail(ctx, st, "scratch allocation failed");
    if ((st = begin(ctx)) != RNMF_OK) return st;
    QbBufs b{};
    b.atx = (double*)arena_take(ctx, a1 + 8);
    b.tc = tc_scratch_take(ctx, m, n, l, form);
    const bool accurate = form == RNMF_PREC_SPLIT3;
    const int prec = form == RNMF_PREC_FP32 ? RNMF_PREC_FP32 : RNMF_PREC_BF16;
    bool ok = transpose ? product_atx(ctx, b, prec, accurate, A, lda, X, out, m, n, l)
                        : product_ax(ctx, b, prec, accurate, A, lda, X, out, m, n, l);
    if (!ok) return cuda_fail(ctx, "sketch product");
    return finish(ctx, "rnmf_sketch");
}

rnmf_status rnmf_omega(rnmf_ctx* ctx, int64_t n, int l, uint64_t seed, int dist, float* Omega) {
    if (!ctx) return RNMF_EINVAL;
    if (n < 1 || l < 1 || !Omega || dist < 0 || dist > 1) return fail(ctx, RNMF_EINVAL, "bad argument");
    rnmf_status st = begin(ctx);
    if (st != RNMF_OK) return st;
    if (!launch_omega(ctx, Omega, n, l, seed, dist, l, 1)) return cuda_fail(ctx, "omega");
    return finish(ctx, "rnmf_omega");
}

rnmf_status rnmf_init_factors(rnmf_ctx* ctx, int64_t m, int64_t n, int k, uint64_t seed, float* W, float* H) {
    if (!ctx) return RNMF_EINVAL;
    if (m < 1 || n < 1 || k < 1 || !W || !H) return fail(ctx, RNMF_EINVAL, "bad argument");
    rnmf_status st = begin(ctx);
    if (st != RNMF_OK) return st;
    if (!launch_uniform_matrix(ctx, W, m, k, seed + 1, 2, k, 1)) return cuda_fail(ctx, "W_init");
    if (!launch_uniform_matrix(ctx, H, k, n, seed + 1, 3, n, 1)) return cuda_fail(ctx, "H_init");
    return finish(ctx, "rnmf_init_factors");
}

rnmf_status rnmf_rel_err(rnmf_ctx* ctx, const float* A, int64_t m, int64_t n, int64_t lda, const float* W,
                         const float* H, int k, double* out) {
    if (!ctx) return RNMF_EINVAL;
    if (m < 1 || n < 1 || lda < n || k < 1 || !A || !W || !H || !out) return fail(ctx, RNMF_EINVAL, "bad argument");
    rnmf_status st = arena_reserve(ctx, arena_round(relerr_scratch_bytes(ctx, m, n)) + 256);
    if (st != RNMF_OK) return fail(ctx, st, "scratch allocation failed");
    if ((st = begin(ctx)) != RNMF_OK) return st;
    double* scratch = (double*)arena_take(ctx, relerr_scratch_bytes(ctx, m, n));
    double* out2 = (double*)arena_take(ctx, 16);
    if (!launch_relerr(ctx, A, lda, W, k, 1, H, m, n, k, out2, scratch)) return cuda_fail(ctx, "relerr");
    if ((st = finish(ctx, "rnmf_rel_err")) != RNMF_OK) return st;
    double h[2];
    if (cudaMemcpy(h, out2, 16, cudaMemcpyDeviceToHost) != cudaSuccess) return cuda_fail(ctx, "copy");
    *out = h[1] > 0 ? std::sqrt(h[0] / h[1]) : 0.0;
    return RNMF_OK;
}

}  // extern "C"
