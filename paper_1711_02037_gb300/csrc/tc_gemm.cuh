// tc_gemm.cuh - tcgen05 (5th-generation tensor core) forms of the QB products.
#pragma once
#include "rnmf_internal.cuh"

struct TcScratch {
    void* xhi = nullptr;      // packed BF16 operand X (K-major, swizzled tiles), hi part
    void* xlo = nullptr;      // lo part (3-term form)
    void* partial = nullptr;  // split-K partials (float)
    size_t xpack_bytes = 0, partial_bytes = 0;
};

bool tc_available();
size_t tc_scratch_bytes(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int precision);
TcScratch tc_scratch_take(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int precision);
// Y (m x l) = A (m x n, lda) X (n x l); nterms = 1 (BF16) or 3 (split BF16 hi/lo);
// accumulate: Y += A X (the old Y and the partials summed as a two-sum pair, rounded once).
bool tc_gemm_ax(rnmf_ctx* ctx, const TcScratch& s, const float* A, int64_t lda, const float* X, float* Y, int64_t m,
                int64_t n, int l, int nterms, bool accumulate = false);
// Z (n x l) = A^T (n x m) X (m x l) (accumulate: Z += A^T X).
bool tc_gemm_atx(rnmf_ctx* ctx, const TcScratch& s, const float* A, int64_t lda, const float* X, float* Z, int64_t m,
                 int64_t n, int l, int nterms, bool accumulate = false);

// The products of a randomized HALS sweep on tensor cores, every one in the 3-term
// split (Bt n x l, Wt l x k, H k x n, Wc = W^T k x m, all row-major float32;
// l, k <= 128; n, m and l multiples of 4, the matrices 16-byte aligned -
// tc_hhalf_fits, tc_gram_fits):
//   tc_hhalf_pack_b: B^T's bf16 hi/lo operand tiles, once per solve (B is fixed);
//   tc_hhalf_r:      R^T (k x n) = (B^T W~)^T;
//   tc_hhalf_tv:     T^T (k x l) = (B H^T)^T and V (k x k) = H H^T from one pass over H
//                    (H's tile is the A operand of both products and V's B operand);
//   tc_hhalf_gram:   S (k x k) = W^T W from one pass over W^T.
struct TcHhalf {
    void *bhi = nullptr, *blo = nullptr;  // packed B^T (K = n)
    void *whi = nullptr, *wlo = nullptr;  // packed W~ (K = l), per sweep
    float* part = nullptr;                // per-unit partials of T^T and V, or of S
};
bool tc_hhalf_fits(int64_t n, int l, int k, const float* Bt, const float* H);
bool tc_gram_fits(int64_t m, int k, const float* Wc);
size_t tc_hhalf_bytes(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int k);
TcHhalf tc_hhalf_take(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int k);
bool tc_hhalf_pack_b(rnmf_ctx* ctx, const TcHhalf& h, const float* Bt, int64_t n, int l);
bool tc_hhalf_r(rnmf_ctx* ctx, const TcHhalf& h, const float* Bt, int64_t n, int l, const float* Wt, int k, float* Rt);
bool tc_hhalf_tv(rnmf_ctx* ctx, const TcHhalf& h, const float* H, int64_t n, int l, int k, float* Tt, float* V);
bool tc_hhalf_gram(rnmf_ctx* ctx, const TcHhalf& h, const float* Wc, int64_t m, int k, float* S);
