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
// accumulate: Y += A X (the sum formed in float64 with the old Y, rounded once).
bool tc_gemm_ax(rnmf_ctx* ctx, const TcScratch& s, const float* A, int64_t lda, const float* X, float* Y, int64_t m,
                int64_t n, int l, int nterms, bool accumulate = false);
// Z (n x l) = A^T (n x m) X (m x l) (accumulate: Z += A^T X).
bool tc_gemm_atx(rnmf_ctx* ctx, const TcScratch& s, const float* A, int64_t lda, const float* X, float* Z, int64_t m,
                 int64_t n, int l, int nterms, bool accumulate = false);
