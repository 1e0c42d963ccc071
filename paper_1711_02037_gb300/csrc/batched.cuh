// batched.cuh - shared layout of the batched ragged randomized HALS path.
//
// Many independent problems (A_i, k_i, p_i, q_i, iters_i) run through the same
// steps as the single-problem path (Algorithm 1): Gaussian Omega_i, sketch,
// q subspace iterations with CholeskyQR2, B_i = Q_i^T A_i, then the compressed
// sweeps.  Every step is one launch over all problems: the products and
// CholeskyQR steps walk a list of row or column tiles of every problem (a
// persistent grid takes tiles from an atomic counter), and the sweeps give each
// problem one thread-block cluster that keeps W~, S, T, V replicated in every
// member's shared memory and combines partial sums over distributed shared
// memory.
#pragma once

#include "rnmf_internal.cuh"

constexpr int RB_MAX_L = 64;    // l = k + p
constexpr int RB_MAX_K = 32;    // k
constexpr int RB_GR = 512;      // rows per partial Gram matrix
constexpr int RB_BMAX = 256;    // rows (columns) per product tile
constexpr int RB_MAX_CLUSTER = 8;

// One problem of a batch (device copy; the caller's pointers are refreshed
// before every run, everything else is fixed by the plan).
struct __align__(16) RbInst {
    const float* A;  // m x n, row-major, leading dimension lda
    float* W;        // m x k (output)
    float* H;        // k x n (output)
    float* Y;        // m x ldq: sketch, then Q
    float* Z;        // n x ldq: Omega, then A^T Q, finally B^T
    float* Wc;       // k x m: W stored transposed during the sweeps
    double* gpart;   // ceil(max(m, n) / RB_GR) partial Gram matrices, l x l each
    float* Rinv;     // l x l: inverse Cholesky factor of the current CholeskyQR pass
    int64_t lda;
    int m, n, k, l, ldq, iters, q;
    int gram_mode, omega_dist;
    int bm;          // rows (columns) per product tile
    int shifted;     // CholeskyQR pass 1 used the shift (a third pass follows)
    int status;      // RNMF_DEV_* of this problem
    uint64_t seed;
    uint32_t inst;   // Philox instance word of this problem
    uint32_t pad2_;
};

// A contiguous range [r0, r1) of rows (or columns) of problem `inst`.
struct RbTile {
    int inst, r0, r1, pad;
};

// Launchers (batched.cu).  All take device arrays built by the plan; `grid` is
// the persistent grid of the tile kernels; `gate` skips problems with q < gate
// (the power iteration a launch belongs to; 0 for steps every problem takes).
bool rb_launch_omega(cudaStream_t s, RbInst* I, int count);
bool rb_launch_init(cudaStream_t s, RbInst* I, int count);
// mode 0: Y = A Z (tiles over rows of A); 1: Y = Y Rinv (rows of Y); 2: Z = Z Rinv (rows of Z).
// only_shifted: skip problems whose first CholeskyQR pass did not shift.
bool rb_launch_rows(cudaStream_t s, int grid, RbInst* I, const RbTile* tiles, int ntiles, int* counter, int mode,
                    int only_shifted, int gate);
// Z = A^T Y (tiles over columns of A).
bool rb_launch_atx(cudaStream_t s, int grid, RbInst* I, const RbTile* tiles, int ntiles, int* counter, int gate);
// Partial Gram matrices of Y (which 0) or Z (which 1) over RB_GR-row chunks.
bool rb_launch_gram(cudaStream_t s, int grid, RbInst* I, const RbTile* tiles, int ntiles, int* counter, int which,
                    int only_shifted, int gate);
// Cholesky + inverse per problem; pass 0 may shift, pass 2 runs only after a shift.
bool rb_launch_chol(cudaStream_t s, RbInst* I, int count, int which, int pass, int gate);
// Compressed sweeps: one cluster of `csize` CTAs per problem in `list` (count
// problems), `nt` threads per CTA, register blocks of lq >= l columns and
// km >= k rows (16 or 32).
// iters_override >= 0 replaces every problem's sweep count (autotuning runs).
bool rb_launch_sweeps(cudaStream_t s, RbInst* I, const int* list, int count, int csize, int lq, int km, int nt,
                      int iters_override);
// Rows (columns) per product tile for a problem with l columns.
int rb_tile_rows(int l);
// Register-block width of the sweeps for l columns (16, 32 or 64) and k (16, 32).
int rb_lq(int l);
int rb_km(int k);
