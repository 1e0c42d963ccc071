// tc_gemm.cu - placeholder until the tcgen05 engine lands.
#include "tc_gemm.cuh"

bool tc_available() { return false; }
size_t tc_scratch_bytes(rnmf_ctx*, int64_t, int64_t, int, int) { return 0; }
TcScratch tc_scratch_take(rnmf_ctx*, int64_t, int64_t, int, int) { return TcScratch{}; }
bool tc_gemm_ax(rnmf_ctx*, const TcScratch&, const float*, int64_t, const float*, float*, int64_t, int64_t, int, int) {
    return false;
}
bool tc_gemm_atx(rnmf_ctx*, const TcScratch&, const float*, int64_t, const float*, float*, int64_t, int64_t, int, int) {
    return false;
}
