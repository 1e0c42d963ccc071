/*
 * rnmf.h - C ABI of the GB300 (sm_103a) randomized HALS NMF library (librnmf.so).
 *
 * Method: Erichson, Mendible, Wihlborn, Kutz, "Randomized Nonnegative Matrix
 * Factorization", arXiv:1711.02037.  The library computes nonnegative factors
 * W (m x k) and H (k x n) with A ~ W H (Section 2.1, Eq. for X ~ W H; NMF
 * objective of Section 2.2) by
 *   1. the randomized QB decomposition of Section 2.3 / Algorithm 1: Gaussian
 *      test matrix Omega (n x l, l = k + p), Y = A Omega, q subspace
 *      iterations with re-orthonormalisation, Q = qr(Y), B = Q^T A;
 *   2. the compressed HALS sweeps of Section 3.2 / Algorithm 1: H rows
 *      H_j <- max(0, H_j + (R_:j - H^T S_:j)/S_jj) with R = B^T W~ and
 *      S = W^T W; W~ columns W~_j <- W~_j + (T_:j - W~ V_:j)/V_jj with
 *      T = B H^T, V = H H^T; reprojection W_j = max(0, Q W~_j), W~_j = Q^T W_j.
 * Deterministic HALS (Section 3.1, residual-free rules) is provided on the full
 * A for comparison.
 *
 * Conventions for every call:
 *   - Matrices are float32, row-major, in DEVICE memory, unless a call says
 *     otherwise.  A is m x n with leading dimension lda >= n and is read only.
 *     W is m x k and H is k x n (dense, leading dimensions k and n).
 *   - All buffers are owned by the caller; the library never frees them.  The
 *     context owns all scratch memory (grown on demand, kept until destroy).
 *   - Work is issued on the context's stream.  Every compute call returns after
 *     synchronising that stream and reading the device status word, so a
 *     returned RNMF_OK means the outputs are complete.
 *   - Argument errors return RNMF_EINVAL before any work is issued and leave the
 *     outputs untouched.  Any other error leaves the outputs unspecified;
 *     rnmf_last_error() returns a message.
 *   - Limits of this GPU path: 1 <= k, l = k + p <= 128, l <= min(m, n)
 *     (l == m <= n is accepted: Q is then square), m, n < 2^31.
 *   - Random draws use Philox4x32-10 (Salmon et al., SC'11) with key
 *     (lo32(seed), hi32(seed)) and counter (lo32(b), hi32(b), stream, 0):
 *     Omega from key seed, stream 1 (Gaussian: Box-Muller on a block, element
 *     2b <- cos branch, 2b+1 <- sin branch; uniform: word e&3 of block e>>2,
 *     (word >> 8) 2^-24); W_init (stream 2) and H_init (stream 3) uniform
 *     [0,1) from key seed + 1, both indexed by the row-major element number.
 *   - One context per host thread.  Calls on one context must not overlap.
 */
#ifndef RNMF_H
#define RNMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rnmf_ctx rnmf_ctx;

typedef enum {
    RNMF_OK = 0,
    RNMF_EINVAL = 1,    /* bad argument (checked on the host before any work) */
    RNMF_ENOMEM = 2,    /* device allocation of scratch failed */
    RNMF_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
    RNMF_ENOTPD = 4,    /* Gram matrix of the QR step not positive definite even after the shift */
    RNMF_ETIMEOUT = 5,  /* a bounded device-side wait (grid barrier) ran out */
    RNMF_ENOTIMPL = 6   /* option combination not built */
} rnmf_status;

/* Arithmetic form of the QB products (Y = A X, Z = A^T X, B = Q^T A). */
enum {
    RNMF_PREC_FP32 = 0,      /* FP32 CUDA-core products, compensated accumulation */
    RNMF_PREC_BF16 = 1,      /* power-iteration products in BF16 on tcgen05 tensor cores
                                (FP32 accumulate); the final sketch and B in 3-term split
                                BF16 (FP32-accurate to ~2^-16) */
    RNMF_PREC_SPLIT3 = 2     /* every QB product in 3-term split BF16 on tcgen05 */
};

typedef struct {
    int precision;        /* RNMF_PREC_*; default RNMF_PREC_FP32 */
    int gram_mode;        /* 0: S = W^T W (Algorithm 1); 1: S = W~^T W~ (Section 3.2 H rule) */
    int omega_dist;       /* 0: standard Gaussian Omega; 1: uniform [0,1) Omega */
    int track_every;      /* > 0: relative error ||A - W H||_F/||A||_F after every
                             track_every-th sweep is written to stats->rel_err_hist */
    long long spin_limit; /* grid-barrier wait limit in SM clock cycles; 0 = default (~2e9) */
    /* Section 3.4 penalties (elastic net, all >= 0; 0 = plain HALS): the sweeps
     * minimise ||A - W H||^2 + alpha_W ||W||^2 + alpha_H ||H||^2
     *           + 2 beta_W sum(W) + 2 beta_H sum(H)
     * component by component (the printed l1 rules take the l1 weight once
     * against the halved quadratic term).  Compressed form: the W~ column rule
     * subtracts beta_W Q^T 1 and divides by V_jj + alpha_W. */
    float alpha_W, alpha_H, beta_W, beta_H;
    /* Section 3.3 stopping rule (0 = off): stop after the first checked sweep with
     * ||grad^P f(W, H)||_F^2 <= pg_tol ||grad^P f(W0, H0)||_F^2, f = ||A - W H||^2
     * on the compressed problem (A replaced by Q B); checked every pg_every sweeps
     * (0: 10).  stats->sweeps_done and stats->pg_ratio report the outcome. */
    double pg_tol;
    int pg_every;
    /* Update order of the components within a sweep (Section 3.2 lists the
     * cyclic orders and a shuffled one):
     *   RNMF_ORDER_CYCLIC (default): every sweep updates the k rows of H, then
     *     the k columns of W~ / W, each in index order 1..k (Algorithm 1);
     *   RNMF_ORDER_SHUFFLED: sweep t of a call (t = 0, 1, ...) visits the
     *     components in the order pi_t in both halves; pi_t sorts j = 0..k-1 by
     *     (u_j, j) ascending, u_j = word (j mod 4) of Philox4x32-10 block
     *     t ceil(k/4) + floor(j/4) with key order_seed and counter stream 4;
     *   RNMF_ORDER_INTERLEAVED: the cyclic order W_1 -> H_1 -> ... -> W_k -> H_k
     *     (the first of Section 3.2's two cyclic orders): column j of W~ / W is
     *     updated from T_:j = B H_j^T and V_:j = H H_j^T of the current H, then
     *     row j of H from B^T W~_j and S_:j of the current W.  Runs as two
     *     passes per component: one over Q and W^T, one over B^T and H.
     * The shuffled and interleaved orders are taken by rnmf, rnmf_host,
     * rnmf_sweeps and rnmf_streamed; rnmf_hals, rnmf_batched, rnmf_sweeps_fwd
     * and rnmf_sweeps_bwd reject them (RNMF_EINVAL); the QB entries ignore them. */
    int order;
    unsigned long long order_seed;
    /* Initial factors: RNMF_INIT_UNIFORM (default: W, H ~ U[0,1) from key
     * seed + 1, Algorithm 1) or RNMF_INIT_SVD: nonnegative double SVD (NNDSVD)
     * of the randomized SVD A ~ Q B = (Q U_B) diag(s) V^T (the initialisation
     * remark after Algorithm 1; Section 4): component 1 from |u_1|, |v_1|, every
     * other from the larger (by |u.| |v.|) of its positive and negative part
     * pairs, scaled by sqrt(s_j |u.| |v.|).  Taken by rnmf and rnmf_host;
     * rnmf_hals, rnmf_batched and rnmf_streamed reject RNMF_INIT_SVD. */
    int init;
    /* Arithmetic of the sweeps' products in the cyclic and shuffled orders
     * (R = B^T W~, T = B H^T, V = H H^T and, in the cyclic order with
     * gram_mode 0, S = W^T W; Algorithm 1's loop body):
     *   RNMF_SWEEP_FP32 (default): float32 CUDA-core products summed in index
     *     order;
     *   RNMF_SWEEP_SPLIT3: 3-term split BF16 on tcgen05 tensor cores (relative
     *     product error ~2^-16, float32 accumulation, unit sums as two-sum
     *     pairs).  R, T, V are taken where n and l are multiples of 4; S where
     *     m is; l, k <= 128 and the operands 16-byte aligned (device
     *     allocations are); elsewhere the float32 products run.  The H rows and
     *     the W half stay float32.
     * Taken by rnmf, rnmf_host, rnmf_sweeps and rnmf_streamed. */
    int sweep_products;
} rnmf_opts;

enum { RNMF_INIT_UNIFORM = 0, RNMF_INIT_SVD = 1 };

enum { RNMF_SWEEP_FP32 = 0, RNMF_SWEEP_SPLIT3 = 1 };

enum { RNMF_ORDER_CYCLIC = 0, RNMF_ORDER_SHUFFLED = 1, RNMF_ORDER_INTERLEAVED = 2 };

/* Statistics of a call.  The pointer fields are inputs (host arrays the call
 * fills, or NULL): zero-initialise the struct before setting them. */
typedef struct {
    double *rel_err_hist;   /* HOST array of length >= iters / track_every, or NULL */
    double final_rel_err;   /* relative error after the last sweep (if track_every > 0), else -1 */
    float ms_qb;            /* device time of the QB stage (ms) */
    float ms_sweeps;        /* device time of the sweeps (ms) */
    int sweeps_done;
    double pg_ratio;        /* last checked ||grad^P||^2 / ||grad^P(W0, H0)||^2, or -1 */
    /* Compressed objective f~(W~, H) = ||B - W~ H||_F^2 of Section 3.2 (the
     * problem the sweeps minimise, B = Q^T A), per sweep, in float64 from
     * float32 residual entries (one pass over B^T and H, none over A).  Set
     * either pointer to a HOST array of length >= iters to request it (NULL:
     * not computed); entries [0, sweeps_done) are written.
     *   obj_hist[t]: after sweep t (W~ = Q^T W, so f~ <= ||A - W H||_F^2);
     *   obj_half_hist[t]: after the H half of sweep t, W~ not yet updated.
     *     With gram_mode 1 the H half is exact block coordinate descent on f~,
     *     so obj_half_hist[t] <= obj_hist[t - 1] up to rounding.  The
     *     interleaved order has no H half: NaN.
     * Taken by rnmf, rnmf_host, rnmf_sweeps and rnmf_streamed. */
    double *obj_hist;
    double *obj_half_hist;
} rnmf_stats;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * owned by the caller, cudaStreamLegacy or cudaStreamPerThread included; every
 * call of the context launches on it, so inputs written earlier on that stream
 * are ordered before the call.  NULL: the context creates and owns a
 * non-blocking stream, not ordered with any other stream (the caller must
 * finish writing the inputs before the call).
 * Errors: RNMF_EINVAL (ctx NULL), RNMF_ECUDA. */
rnmf_status rnmf_create(rnmf_ctx **ctx, int device, void *cuda_stream);

/* Release the context and its scratch memory (the stream too if it owns it). */
rnmf_status rnmf_destroy(rnmf_ctx *ctx);

/* Fill `opts` with the defaults. */
void rnmf_default_opts(rnmf_opts *opts);

/* Randomized HALS NMF (Algorithm 1): randomized QB with l = k + p, q subspace
 * iterations, Omega from `seed`, W_init/H_init ~ U[0,1) from seed + 1, then
 * `iters` compressed sweeps.  A (m x n, lda), W (m x k), H (k x n): device.
 * opts may be NULL (defaults); stats may be NULL. */
rnmf_status rnmf(rnmf_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, int k, int p, int q,
                 int iters, uint64_t seed, const rnmf_opts *opts, float *W, float *H, rnmf_stats *stats);

/* Same computation with A, W, H in HOST memory (pinned or pageable).  The
 * host-to-device copy of A and the device-to-host copies of W and H are part
 * of the call; A is staged in context scratch. */
rnmf_status rnmf_host(rnmf_ctx *ctx, const float *A_host, int64_t m, int64_t n, int64_t lda, int k, int p,
                      int q, int iters, uint64_t seed, const rnmf_opts *opts, float *W_host, float *H_host,
                      rnmf_stats *stats);

/* Deterministic HALS (Section 3.1 residual-free rules, Algorithm 1's order: all
 * H rows, then all W columns) on the full A, from the same W_init/H_init as
 * rnmf(seed).  Two passes over A per sweep.  Only opts->track_every and
 * opts->spin_limit are used. */
rnmf_status rnmf_hals(rnmf_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, int k, int iters,
                      uint64_t seed, const rnmf_opts *opts, float *W, float *H, rnmf_stats *stats);

/* Randomized QB decomposition (Section 2.3; Algorithm 1 QB part): writes
 * Q (m x l, orthonormal columns) and Bt = B^T = A^T Q (n x l).  Device memory.
 * Uses opts->precision and opts->omega_dist. */
rnmf_status rnmf_qb(rnmf_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, int l, int q,
                    uint64_t seed, const rnmf_opts *opts, float *Q, float *Bt);

/* `iters` compressed HALS sweeps (Section 3.2, Algorithm 1 repeat loop) from a
 * given Q (m x l), Bt (n x l), W (m x k, in: W_init, out: result), H (k x n,
 * in/out) and optional Wt (l x k, in/out; NULL: W~ = Q^T W is formed first and
 * discarded at the end).  A (m x n, lda) is only read when
 * opts->track_every > 0 (may be NULL otherwise).  Device memory. */
rnmf_status rnmf_sweeps(rnmf_ctx *ctx, const float *Q, const float *Bt, int64_t m, int64_t n, int l, int k,
                        int iters, const rnmf_opts *opts, float *W, float *H, float *Wt, const float *A,
                        int64_t lda, rnmf_stats *stats);

/* One product of the randomized QB (Section 2.3; Algorithm 1 steps that form
 * Y = A Omega, Y = A Q and B = Q^T A): transpose = 0 computes Y = A X with
 * X (n x l) and Y (m x l); transpose = 1 computes Z = A^T X with X (m x l) and
 * Z (n x l).  X and the output are row-major (leading dimension l), device
 * memory, l <= 128.  form: RNMF_PREC_FP32 (CUDA cores), RNMF_PREC_BF16 (one
 * bf16 product on tensor cores), RNMF_PREC_SPLIT3 (hi/lo split, 3 products).
 * The tensor-core forms need lda % 4 == 0 and a 16-byte aligned A. */
rnmf_status rnmf_sketch(rnmf_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *X, int l,
                        int transpose, int form, float *out);

/* ---- Batched ragged problems.  Many independent problems of different sizes
 * run through Algorithm 1 together (FP32 form): the randomized QB steps are
 * shared launches over tiles of all problems, the sweeps give each problem one
 * thread-block cluster (1, 2, 4 or 8 CTAs, chosen by an autotuner that times
 * candidate configurations on the batch itself the first time its sizes are
 * seen), and the whole pipeline is captured into one CUDA graph that later
 * calls with the same sizes replay.  Each problem is what rnmf() computes for
 * it, with the Philox instance word `instance` in every random draw (Omega,
 * W_init, H_init), so rnmf(seed) equals instance 0. */
typedef struct {
    const float *A;   /* m x n, row-major, lda >= n; device */
    int64_t m, n, lda;
    int k, p, q, iters; /* 1 <= k <= 32, p >= 0, k + p <= min(m, n, 64), q >= 0 */
    uint64_t seed;
    uint32_t instance;
    float *W;         /* m x k output; device */
    float *H;         /* k x n output; device */
} rnmf_problem;

typedef struct {
    float ms;              /* device time of the graph replay of this call */
    int tuned;             /* 1: this call built the plan (autotuning, capture) */
    int graph_kernels;     /* kernel launches in one replay */
    int cluster_count[4];  /* problems swept by clusters of 1, 2, 4, 8 CTAs */
    int threads_small;     /* threads per CTA chosen for l <= 32 */
    int failed;            /* problems with a non-OK status */
    float tune_ms[8];      /* autotuner: time of each candidate (4 sweeps) */
} rnmf_batch_stats;

/* Runs every problem of `probs` (host array of `count`).  opts: gram_mode and
 * omega_dist are used (precision must be RNMF_PREC_FP32).  status_out (host,
 * may be NULL) receives each problem's status.  The first call for a list of
 * sizes allocates the plan's device workspace and captures the graph; the
 * plan is kept in the context until a call with other sizes or
 * rnmf_destroy.  Errors: RNMF_EINVAL (a problem out of range, named in
 * rnmf_last_error), RNMF_ENOMEM, RNMF_ENOTPD (a CholeskyQR factorisation
 * failed; other problems are still computed), RNMF_ECUDA. */
rnmf_status rnmf_batched(rnmf_ctx *ctx, const rnmf_problem *probs, int count, const rnmf_opts *opts,
                         int *status_out, rnmf_batch_stats *stats);

/* Fixes what the autotuner of later plans may choose: max_cluster (1, 2, 4 or
 * 8: the largest problem gets clusters of that size and smaller ones
 * proportionally fewer CTAs; 0: tune) and threads_small (256 or 512 threads
 * per CTA for l <= 32; 0: tune).  Drops the current plan. */
rnmf_status rnmf_batched_config(rnmf_ctx *ctx, int max_cluster, int threads_small);

/* ||A_i - W_i H_i||_F / ||A_i||_F of every problem (host output, count). */
rnmf_status rnmf_batched_rel_err(rnmf_ctx *ctx, const rnmf_problem *probs, int count, double *out);

/* ---- A in host memory, read in column blocks (Algorithm 2, Appendix A): for
 * matrices larger than device memory.  Each pass copies blocks of block_cols
 * columns (0: blocks of about 1 GiB) into two device staging buffers, the next
 * block's copy overlapping the current block's products (opts->precision
 * selects the product form as in rnmf: FP32 CUDA cores, or tcgen05 tensor
 * cores - BF16 power passes, 3-term split elsewhere, or the split everywhere;
 * a block whose width is not a multiple of 4 floats uses the CUDA cores):
 *   Y = sum_J A(:, J) Omega(J, :);
 *   q times: Q = qr(Y), Y = sum_J A(:, J) (A(:, J)^T Q)   (one pass each);
 *   Q = qr(Y);  B^T(J, :) = A(:, J)^T Q.
 * q + 2 passes over A (Algorithm 1's in-memory scheme takes 2 q + 2).  A is a
 * HOST pointer (pinned memory overlaps the copies; pageable memory works but
 * each copy blocks the host); Q (m x l) and Bt (n x l) are device outputs. */
rnmf_status rnmf_qb_streamed(rnmf_ctx *ctx, const float *A_host, int64_t m, int64_t n, int64_t lda, int l, int q,
                             uint64_t seed, const rnmf_opts *opts, int64_t block_cols, float *Q, float *Bt);

/* rnmf() with the streamed QB above: A in host memory, W (m x k) and H (k x n)
 * device outputs.  opts->track_every must be 0 (the error needs A on the
 * device; use rnmf_rel_err on a device copy if it fits). */
rnmf_status rnmf_streamed(rnmf_ctx *ctx, const float *A_host, int64_t m, int64_t n, int64_t lda, int k, int p, int q,
                          int iters, uint64_t seed, const rnmf_opts *opts, int64_t block_cols, float *W, float *H,
                          rnmf_stats *stats);

/* Projected-gradient measure of Section 3.3 on the compressed problem,
 * ||grad^P f(W, H)||_F^2 with f = ||Q B - W H||_F^2 evaluated as
 * G_W = 2 (W H H^T - Q B H^T), G_H = 2 (W^T W H - (Q^T W)^T B), projected
 * (G where the entry is > 0, min(0, G) where it is 0), summed in float64.
 * Q (m x l), Bt (n x l), W (m x k), H (k x n); device memory, host output. */
rnmf_status rnmf_projected_gradient(rnmf_ctx *ctx, const float *Q, const float *Bt, int64_t m, int64_t n, int l,
                                    int k, const float *W, const float *H, double *out);

/* ---- Differentiation of T unrolled compressed sweeps (loss L = <G, W_T H_T>
 * is formed by the caller).  Not a step of the paper: reverse mode through the
 * Section 3.2 update rules (Algorithm 1 loop), with Q held fixed so that
 * dL/dA = Q dL/dB.  The adjoint needs 5 l k + 2 k^2 <= 56000. */

/* Floats of the checkpoint buffer for T sweeps: (T + 1) states of
 * W^T (k x m), W~ (l x k), H (k x n). */
size_t rnmf_ckpt_floats(int64_t m, int64_t n, int l, int k, int T);

/* T sweeps from W (m x k, in: W_init, out: W_T) and H (k x n, in/out), with
 * W~ = Q^T W_init; if ckpt != NULL it receives every sweep-boundary state.
 * Q (m x l), Bt (n x l).  Device memory. */
rnmf_status rnmf_sweeps_fwd(rnmf_ctx *ctx, const float *Q, const float *Bt, int64_t m, int64_t n, int l, int k,
                            int T, const rnmf_opts *opts, float *W, float *H, float *ckpt);

/* Reverse pass: from dL/dW_T (m x k) and dL/dH_T (k x n) and the checkpoints
 * of rnmf_sweeps_fwd, writes dL/dB^T (n x l), dL/dW_init (m x k) and
 * dL/dH_init (k x n).  Every sweep is recomputed from its checkpoints.
 * Subgradient 0 at every clamp argument equal to 0.  Device memory. */
rnmf_status rnmf_sweeps_bwd(rnmf_ctx *ctx, const float *Q, const float *Bt, int64_t m, int64_t n, int l, int k,
                            int T, const rnmf_opts *opts, const float *ckpt, const float *dW_T, const float *dH_T,
                            float *dBt, float *dW_init, float *dH_init);

/* dL/dA = Q dL/dB = Q dBt^T (m x n, row-major).  Device memory. */
rnmf_status rnmf_dA(rnmf_ctx *ctx, const float *Q, const float *dBt, int64_t m, int64_t n, int l, float *dA);

/* The test matrix Omega (n x l, row-major) of rnmf(seed): dist 0 Gaussian,
 * 1 uniform.  Device memory.  Bit-identical to the library's internal draw. */
rnmf_status rnmf_omega(rnmf_ctx *ctx, int64_t n, int l, uint64_t seed, int dist, float *Omega);

/* The initial factors of rnmf(seed) / rnmf_hals(seed): W_init (m x k) and
 * H_init (k x n), uniform [0,1) from key seed + 1.  Device memory. */
rnmf_status rnmf_init_factors(rnmf_ctx *ctx, int64_t m, int64_t n, int k, uint64_t seed, float *W, float *H);

/* Relative error ||A - W H||_F / ||A||_F (the "Error" column of Section 4),
 * W H formed in float32, squares accumulated in float64.  Device inputs, host
 * output. */
rnmf_status rnmf_rel_err(rnmf_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *W,
                         const float *H, int k, double *out);

/* rnmf_rel_err without any device allocation.  The paper has no counterpart:
 * this is for callers that cannot let the library call cudaMalloc/cudaFree - a
 * process that has given all free device memory to its own pool, or one that
 * keeps other streams busy and cannot take the device-wide synchronisation of
 * those calls.  Same kernels and result as rnmf_rel_err; the per-tile partial
 * sums live in a fixed 4 MiB device array compiled into the library.
 *   Limit: ceil(m/64) * ceil(n/64) <= 262144 (RNMF_EINVAL beyond it), and
 *   per-kernel profiling must be off (RNMF_EINVAL otherwise).
 *   Nothing in the array needs to start at zero.
 *   The array is shared by all contexts on a device: calls on one device
 *   whose work overlaps in time race on it; the caller serialises them.
 *   The first call on a device looks the array up (cudaGetSymbolAddress);
 *   make it before any stream capture begins.
 * Device inputs, host output. */
rnmf_status rnmf_rel_err_noalloc(rnmf_ctx *ctx, const float *A, int64_t m, int64_t n, int64_t lda, const float *W,
                                 const float *H, int k, double *out);

/* Caps the device scratch the context may hold at `bytes` (its arena, the
 * staging of rnmf_host and the workspace of a batched plan; 0: no cap, the
 * default).  Not a step of the paper: for callers that share the device with
 * other work and must bound the library's memory.  A call that would need more
 * returns RNMF_ENOMEM before any work is issued and leaves the outputs
 * untouched; scratch already held is kept (rnmf_destroy frees it).
 * Errors: RNMF_EINVAL (ctx NULL). */
rnmf_status rnmf_set_scratch_limit(rnmf_ctx *ctx, size_t bytes);

/* Bytes of device scratch the context holds now (0 for a NULL ctx). */
size_t rnmf_scratch_bytes(rnmf_ctx *ctx);

/* Message for the last non-OK status on this context (static storage). */
const char *rnmf_last_error(rnmf_ctx *ctx);

/* Number of kernels this context has launched since creation (diagnostics). */
long long rnmf_kernel_launches(rnmf_ctx *ctx);

/* Per-kernel-class device time of the launches issued while profiling is on:
 * CUDA events are recorded on the context stream around every launch, and
 * each launch adds its algorithmic bytes (compulsory DRAM traffic of the
 * operation) and flops.  rnmf_profile(ctx, 1) resets the counters and starts,
 * rnmf_profile(ctx, 0) stops.  rnmf_profile_read() fills at most `max` entries
 * (classes with launches only) and returns how many it filled; names are
 * static strings.  Reading synchronises the context stream. */
typedef struct {
    const char *name;
    long long launches;
    double ms;      /* total device time of the class (sum over launches) */
    double bytes;   /* total algorithmic bytes */
    double flops;   /* total algorithmic flops */
} rnmf_kernel_prof;

rnmf_status rnmf_profile(rnmf_ctx *ctx, int on);
int rnmf_profile_read(rnmf_ctx *ctx, rnmf_kernel_prof *out, int max);

#ifdef __cplusplus
}
#endif

#endif /* RNMF_H */
