// tc_gemm.cu - the skinny QB products on 5th-generation tensor cores (tcgen05).
//
//   AX : Y (M = m rows) = A (m x n) X (n x l)        contraction over n
//   ATX: Z (M = n rows) = A^T (n x m) X (m x l)      contraction over m
// (Y = A Omega and Y = A Q of the power scheme, Z = A^T Q, B^T = A^T Q;
// Section 2.3 / Algorithm 1.)  A stays float32 in HBM and is read once per
// product; X is small (l <= 128 columns).
// The same kernel forms the sweeps' products (Algorithm 1's loop body):
//   AX with a transposed output: R^T = (B^T W~)^T;
//   mode 2 (pair): the A tile (rows of H, or of W^T) against X and against its
//     own first rows, two accumulators side by side in tensor memory:
//     T^T = H B^T^T and V = H H^T from one pass over H, or S = W^T W alone.
//     One unit per CTA; the unit's partial block is staged in shared memory and
//     written with one bulk copy, and hv_reduce_kernel adds the units.
//
// Precision forms: nterms = 1 multiplies bf16(A) bf16(X); nterms = 3 splits
// every float32 value into hi = bf16(x) and lo = bf16(x - hi) and accumulates
// hi*hi + hi*lo + lo*hi (relative product error ~2^-16).  Accumulation is float32
// in tensor memory.
//
// Kernel structure (one persistent CTA per SM, 10 warps):
//   warp 0  TMA producer: A tiles (128 x 64 float32) with cp.async.bulk.tensor
//           into a float32 staging ring; the pre-packed bf16 X tile for the same
//           k-step with cp.async.bulk into the MMA operand ring.
//   warp 1  MMA issuer: tcgen05.mma.cta_group::1.kind::f16, M = 128, N = lpad,
//           K = 16, accumulator in TMEM; tcgen05.commit frees operand slots.
//   warps 2-5 converters: float32 staging -> bf16 hi (/lo) in the 128-byte
//           swizzled K-major layout the MMA reads (AX: row-contiguous tile;
//           ATX: column-contiguous tile, transposed while converting).
//   warps 6-9 epilogue: tcgen05.ld of the accumulator rows -> global float32;
//           two TMEM accumulators, so a unit drains while the next one runs.
// Work units are (128-row tile, contraction chunk).  The tensor core's float32
// accumulation is not exactly rounded, so its error grows with the number of
// chained MMAs; a unit therefore spans at most 4096 contraction elements in the
// 3-term form (and 16384 in the 1-term form, whose operand rounding dominates),
// and the per-unit partials are summed as two-sum pairs in a fixed order by a
// separate reduction (deterministic results).
// Every mbarrier wait is bounded: on a timeout the CTA records RNMF_ETIMEOUT,
// waits (bounded) for its own bulk copies and MMAs in flight, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>

#include "pair_sum.cuh"
#include "tc_gemm.cuh"
#include "tma.cuh"

namespace {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int NTHREADS = 320;
constexpr int F32_STAGE = BM * BK * 4;       // 32 KB float32 staging
constexpr int BF_TILE = BM * BK * 2;         // 16 KB bf16 operand tile (also max B tile: 128 x 64)
constexpr uint32_t TMEM_COLS = 256;   // two 128-column accumulators

template <int NTERMS>
struct Cfg {
    static constexpr int NF = NTERMS == 3 ? 3 : 4;                        // float32 staging stages
    static constexpr int NM = NTERMS == 3 ? 2 : 3;                        // MMA operand stages
    static constexpr int M_STAGE = (NTERMS == 3 ? 4 : 2) * BF_TILE;       // A hi(,lo) + B hi(,lo)
    static constexpr int OFF_M = NF * F32_STAGE;
    static constexpr int OFF_BAR = OFF_M + NM * M_STAGE;
    static constexpr int NBAR = 2 * NF + 3 * NM + 6;
    static constexpr size_t SMEM = 1024 + OFF_BAR + NBAR * 8 + 16;
};

struct TcParams {
    int mode;  // 0 = AX, 1 = ATX, 2 = the H-half pair (mode 0's A tile times X, and times itself)
    int64_t Mdim, Kdim;
    int l, lpad, ksteps, tiles, splits, ksp, units;
    int direct;     // 1: one split and no accumulation - the tile goes straight to out
    int trans_out;  // direct only: out is l x Mdim (entry (row, c) at out[c * Mdim + row])
    int vcols, vpad;  // mode 2: columns of the second product (its A tile's first vcols rows), padded to 16
    const uint8_t* xhi;
    const uint8_t* xlo;
    float* out;
    float* partial;
    int* status;
    long long spin_limit;
};

// ---------------------------------------------------------------- PTX (mbarrier and TMA: tma.cuh)
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                           // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset
    d |= (uint64_t)1 << 46;                           // descriptor version (tcgen05)
    d |= (uint64_t)2 << 61;                           // SWIZZLE_128B
    return d;
}
// Instruction descriptor: kind::f16, A = B = bf16, D = f32, both K-major, M x N.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// W = 32 or 64 consecutive accumulator columns of this thread's lane with one load and
// one wait (the epilogues: fewer load-to-use round trips than 16-column loads).  The
// wait names the loaded registers, so no use of them can move above it.
#define TC_O4(b) "=r"(r[b]), "=r"(r[b + 1]), "=r"(r[b + 2]), "=r"(r[b + 3])
#define TC_O16(b) TC_O4(b), TC_O4(b + 4), TC_O4(b + 8), TC_O4(b + 12)
#define TC_P4(b) "+r"(r[b]), "+r"(r[b + 1]), "+r"(r[b + 2]), "+r"(r[b + 3])
#define TC_P16(b) TC_P4(b), TC_P4(b + 4), TC_P4(b + 8), TC_P4(b + 12)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : TC_O16(0), TC_O16(16)
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : TC_P16(0), TC_P16(16)::"memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, "
        "%36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, "
        "%57, %58, %59, %60, %61, %62, %63}, [%64];"
        : TC_O16(0), TC_O16(16), TC_O16(32), TC_O16(48)
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : TC_P16(0), TC_P16(16), TC_P16(32), TC_P16(48)::"memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}
#undef TC_O4
#undef TC_O16
#undef TC_P4
#undef TC_P16
__device__ __forceinline__ void tmem_ldw(uint32_t taddr, float (&v)[16]) { tmem_ld16(taddr, v); }
__device__ __forceinline__ void tmem_ldw(uint32_t taddr, float (&v)[32]) { tmem_ld32(taddr, v); }
__device__ __forceinline__ void tmem_ldw(uint32_t taddr, float (&v)[64]) { tmem_ld64(taddr, v); }

// W accumulator columns c0 .. c0 + W - 1 of this lane to dst[c * stride] for c < lim
// (every lane of the warp takes part in the load; `ok` guards the stores).
template <int W>
__device__ __forceinline__ void epi_cols(uint32_t taddr, float* dst, int64_t stride, int c0, int lim, bool ok) {
    float v[W];
    tmem_ldw(taddr, v);
    if (ok) {
#pragma unroll
        for (int j = 0; j < W; ++j)
            if (c0 + j < lim) dst[(int64_t)(c0 + j) * stride] = v[j];
    }
}
// W accumulator columns c0 .. of this lane into its row `row` (16-byte aligned) as
// float4s: columns from c0 up to lim rounded up to 4 (the row's pad takes the rest).
template <int W>
__device__ __forceinline__ void epi_row(uint32_t taddr, float* row, int c0, int lim, bool ok) {
    float v[W];
    tmem_ldw(taddr, v);
    if (ok) {
#pragma unroll
        for (int j = 0; j < W; j += 4)
            if (c0 + j < lim) *reinterpret_cast<float4*>(row + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    }
}
__device__ __forceinline__ void epi_row_span(uint32_t tbase, int pad, float* row, int lim, bool ok) {
    for (int c0 = 0; c0 < pad;) {
        const int rem = pad - c0;
        if (rem >= 64) {
            epi_row<64>(tbase + (uint32_t)c0, row, c0, lim, ok);
            c0 += 64;
        } else if (rem >= 32) {
            epi_row<32>(tbase + (uint32_t)c0, row, c0, lim, ok);
            c0 += 32;
        } else {
            epi_row<16>(tbase + (uint32_t)c0, row, c0, lim, ok);
            c0 += 16;
        }
    }
}
// Row pitch (floats) of a pair-mode partial block of w columns: a multiple of 4 with an
// odd number of 16-byte chunks, so eight consecutive rows' float4s hit distinct banks.
__host__ __device__ __forceinline__ int pair_pitch(int w) {
    const int p4 = (w + 3) / 4 * 4;
    return (p4 / 4) % 2 ? p4 : p4 + 4;
}

// Columns [0, pad) (pad a multiple of 16) in chunks of 64, 32 and 16.
__device__ __forceinline__ void epi_span(uint32_t tbase, int pad, float* dst, int64_t stride, int lim, bool ok) {
    for (int c0 = 0; c0 < pad;) {
        const int rem = pad - c0;
        if (rem >= 64) {
            epi_cols<64>(tbase + (uint32_t)c0, dst, stride, c0, lim, ok);
            c0 += 64;
        } else if (rem >= 32) {
            epi_cols<32>(tbase + (uint32_t)c0, dst, stride, c0, lim, ok);
            c0 += 32;
        } else {
            epi_cols<16>(tbase + (uint32_t)c0, dst, stride, c0, lim, ok);
            c0 += 16;
        }
    }
}

// Bounded wait: false on timeout (recorded in *status and in the CTA abort flag) or abort.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status,
                                         long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > limit) {
            *abort_flag = 1;
            atomicCAS(status, RNMF_DEV_OK, RNMF_DEV_TIMEOUT);
            return false;
        }
    }
}
// Bounded wait used on the way out (ignores the abort flag).
__device__ __forceinline__ void drain_bar(uint32_t bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) break;
    }
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

template <int NTERMS>
__global__ void __launch_bounds__(NTHREADS, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, TcParams p) {
    using C = Cfg<NTERMS>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
    const uint32_t bar0 = smem_u32(bars);
    // barrier index layout
    auto F_full = [&](int s) { return bar0 + 8u * s; };
    auto F_empty = [&](int s) { return bar0 + 8u * (C::NF + s); };
    auto M_afull = [&](int s) { return bar0 + 8u * (2 * C::NF + s); };
    auto M_bfull = [&](int s) { return bar0 + 8u * (2 * C::NF + C::NM + s); };
    auto M_empty = [&](int s) { return bar0 + 8u * (2 * C::NF + 2 * C::NM + s); };
    const uint32_t ACC_full0 = bar0 + 8u * (2 * C::NF + 3 * C::NM);   // [2]
    const uint32_t ACC_empty0 = ACC_full0 + 16u;                       // [2]
    const uint32_t DRAIN = ACC_full0 + 32u;
    const uint32_t EPI = ACC_full0 + 40u;  // mode 2: the four epilogue warps have staged their rows
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + C::OFF_BAR + C::NBAR * 8);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + C::OFF_BAR + C::NBAR * 8 + 8);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (threadIdx.x == 0) {
        // fetch A's tensor map while the barriers are set up (the first TMA load needs it)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        for (int s = 0; s < C::NF; ++s) {
            mbar_init(F_full(s), 1);
            mbar_init(F_empty(s), 4);
        }
        for (int s = 0; s < C::NM; ++s) {
            mbar_init(M_afull(s), 4);
            mbar_init(M_bfull(s), 1);
            mbar_init(M_empty(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(ACC_full0 + 8u * b, 1);
            mbar_init(ACC_empty0 + 8u * b, 4);
        }
        mbar_init(DRAIN, 1);
        mbar_init(EPI, 4);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const long long lim = p.spin_limit;
    const uint32_t b_bytes = (uint32_t)p.lpad * 128u;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------------ producer
            int issuedF[C::NF] = {}, issuedB[C::NM] = {};
            uint32_t g = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
                const int tile = u / p.splits, split = u % p.splits;
                const int kb0 = split * p.ksp;
                const int kb1 = min(kb0 + p.ksp, p.ksteps);
                for (int kb = kb0; kb < kb1; ++kb, ++g) {
                    const int sf = g % C::NF, sm = g % C::NM;
                    if (!wait_bar(F_empty(sf), ((g / C::NF) & 1) ^ 1, abort_flag, p.status, lim)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fdst = smem_u32(smem + sf * F32_STAGE);
                    mbar_expect_tx(F_full(sf), F32_STAGE);
                    if (p.mode != 1) {
                        tma_load_2d(fdst, &tmA, kb * BK, tile * BM, F_full(sf));
                        tma_load_2d(fdst + F32_STAGE / 2, &tmA, kb * BK + 32, tile * BM, F_full(sf));
                    } else {
                        tma_load_2d(fdst, &tmA, tile * BM, kb * BK, F_full(sf));
                    }
                    ++issuedF[sf];
                    if (!wait_bar(M_empty(sm), ((g / C::NM) & 1) ^ 1, abort_flag, p.status, lim)) {
                        ok = false;
                        break;
                    }
                    uint8_t* mst = smem + C::OFF_M + sm * C::M_STAGE;
                    const size_t xoff = (size_t)kb * b_bytes;
                    mbar_expect_tx(M_bfull(sm), (NTERMS == 3 ? 2u : 1u) * b_bytes);
                    if (b_bytes > 0) {  // mode 2 with no X (the self product alone): a plain arrival
                        bulk_load(smem_u32(mst + (NTERMS == 3 ? 2 : 1) * BF_TILE), p.xhi + xoff, b_bytes,
                                  M_bfull(sm));
                        if (NTERMS == 3) bulk_load(smem_u32(mst + 3 * BF_TILE), p.xlo + xoff, b_bytes, M_bfull(sm));
                    }
                    ++issuedB[sm];
                }
            }
            // wait (bounded) for every bulk copy this CTA issued before leaving
            for (int s = 0; s < C::NF; ++s)
                if (issuedF[s]) drain_bar(F_full(s), (issuedF[s] - 1) & 1, lim);
            for (int s = 0; s < C::NM; ++s)
                if (issuedB[s]) drain_bar(M_bfull(s), (issuedB[s] - 1) & 1, lim);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------------- MMA
            const uint32_t idesc = idesc_bf16(BM, p.lpad);
            const uint32_t idesc_v = idesc_bf16(BM, p.mode == 2 ? p.vpad : 16);
            uint32_t g = 0, ucount = 0;
            bool ok = true, issued = false;
            for (int u = blockIdx.x; u < p.units && ok; u += gridDim.x, ++ucount) {
                const int split = u % p.splits;
                const int kb0 = split * p.ksp;
                const int kb1 = min(kb0 + p.ksp, p.ksteps);
                // mode 2 holds both products of a unit in the two accumulators: one unit in flight
                const uint32_t buf = p.mode == 2 ? 0u : (ucount & 1), use = p.mode == 2 ? ucount : (ucount >> 1);
                if (use > 0 && !wait_bar(ACC_empty0 + 8u * buf, (use - 1) & 1, abort_flag, p.status, lim)) break;
                tc_fence_after();
                const uint32_t acc_tmem = tmem + buf * 128u;
                for (int kb = kb0; kb < kb1; ++kb, ++g) {
                    const int sm = g % C::NM;
                    const uint32_t par = (g / C::NM) & 1;
                    if (!wait_bar(M_afull(sm), par, abort_flag, p.status, lim) ||
                        !wait_bar(M_bfull(sm), par, abort_flag, p.status, lim)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = smem_u32(smem + C::OFF_M + sm * C::M_STAGE);
                    const uint32_t a_hi = st, a_lo = st + BF_TILE;
                    const uint32_t b_hi = st + (NTERMS == 3 ? 2 : 1) * BF_TILE, b_lo = st + 3 * BF_TILE;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint32_t acc = (kb > kb0 || kk > 0) ? 1u : 0u;
                        if (p.lpad > 0) {
                            mma_bf16(acc_tmem, desc_sw128(a_hi + kk * 32), desc_sw128(b_hi + kk * 32), idesc, acc);
                            if (NTERMS == 3) {
                                mma_bf16(acc_tmem, desc_sw128(a_hi + kk * 32), desc_sw128(b_lo + kk * 32), idesc,
                                         1u);
                                mma_bf16(acc_tmem, desc_sw128(a_lo + kk * 32), desc_sw128(b_hi + kk * 32), idesc,
                                         1u);
                            }
                        }
                        if (p.mode == 2) {
                            // the A tile against its own first vpad rows (K-major, the same swizzle)
                            const uint32_t acc_v = tmem + 128u;
                            mma_bf16(acc_v, desc_sw128(a_hi + kk * 32), desc_sw128(a_hi + kk * 32), idesc_v, acc);
                            if (NTERMS == 3) {
                                mma_bf16(acc_v, desc_sw128(a_hi + kk * 32), desc_sw128(a_lo + kk * 32), idesc_v, 1u);
                                mma_bf16(acc_v, desc_sw128(a_lo + kk * 32), desc_sw128(a_hi + kk * 32), idesc_v, 1u);
                            }
                        }
                    }
                    issued = true;
                    mma_commit(M_empty(sm));
                }
                if (!ok) break;
                mma_commit(ACC_full0 + 8u * buf);
            }
            if (issued) {
                mma_commit(DRAIN);
                drain_bar(DRAIN, 0, lim);
            }
        }
    } else if (warp < 6) {
        // ------------------------------------------------------- converters
        const int r = (warp - 2) * 32 + lane;   // tile row converted by this thread
        uint32_t g = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < p.units && ok; u += gridDim.x) {
            const int split = u % p.splits;
            const int kb0 = split * p.ksp;
            const int kb1 = min(kb0 + p.ksp, p.ksteps);
            for (int kb = kb0; kb < kb1; ++kb, ++g) {
                const int sf = g % C::NF, sm = g % C::NM;
                if (!wait_bar(F_full(sf), (g / C::NF) & 1, abort_flag, p.status, lim) ||
                    !wait_bar(M_empty(sm), ((g / C::NM) & 1) ^ 1, abort_flag, p.status, lim)) {
                    ok = false;
                    break;
                }
                const uint8_t* F = smem + sf * F32_STAGE;
                uint8_t* Ahi = smem + C::OFF_M + sm * C::M_STAGE;
                uint8_t* Alo = Ahi + BF_TILE;
                const uint32_t rbase = (uint32_t)(r >> 3) * 1024u + (uint32_t)(r & 7) * 128u;
#pragma unroll
                for (int oc = 0; oc < 8; ++oc) {
                    float x[8];
                    if (p.mode != 1) {
                        // staging: two 128 x 32 float32 sub-tiles, 128-byte swizzled rows
                        const uint8_t* sub = F + (oc >> 2) * (F32_STAGE / 2) + r * 128;
                        const int c0 = 2 * (oc & 3);
                        const float4 v0 = *reinterpret_cast<const float4*>(sub + ((c0 ^ (r & 7)) << 4));
                        const float4 v1 = *reinterpret_cast<const float4*>(sub + (((c0 + 1) ^ (r & 7)) << 4));
                        x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
                        x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
                    } else {
                        // staging: 64 x 128 float32 (rows = contraction index, columns = tile rows)
                        const float* Fs = reinterpret_cast<const float*>(F);
#pragma unroll
                        for (int e = 0; e < 8; ++e) x[e] = Fs[(oc * 8 + e) * BM + r];
                    }
                    uint4 hi;
                    hi.x = pack_bf16(x[0], x[1]);
                    hi.y = pack_bf16(x[2], x[3]);
                    hi.z = pack_bf16(x[4], x[5]);
                    hi.w = pack_bf16(x[6], x[7]);
                    const uint32_t off = rbase + (uint32_t)((oc ^ (r & 7)) << 4);
                    *reinterpret_cast<uint4*>(Ahi + off) = hi;
                    if (NTERMS == 3) {
                        const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&hi);
                        float y[8];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float2 f = __bfloat1622float2(h2[e]);
                            y[2 * e] = x[2 * e] - f.x;
                            y[2 * e + 1] = x[2 * e + 1] - f.y;
                        }
                        uint4 lo;
                        lo.x = pack_bf16(y[0], y[1]);
                        lo.y = pack_bf16(y[2], y[3]);
                        lo.z = pack_bf16(y[4], y[5]);
                        lo.w = pack_bf16(y[6], y[7]);
                        *reinterpret_cast<uint4*>(Alo + off) = lo;
                    }
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(F_empty(sf));
                    mbar_arrive(M_afull(sm));
                }
            }
        }
    } else {
        // --------------------------------------------------------- epilogue
        const int q = warp & 3;                 // TMEM lane quarter of this warp
        const int r = q * 32 + lane;            // tile row owned by this thread
        uint32_t ucount = 0;
        for (int u = blockIdx.x; u < p.units; u += gridDim.x, ++ucount) {
            const int tile = u / p.splits, split = u % p.splits;
            const uint32_t buf = p.mode == 2 ? 0u : (ucount & 1), use = p.mode == 2 ? ucount : (ucount >> 1);
            if (!wait_bar(ACC_full0 + 8u * buf, use & 1, abort_flag, p.status, lim)) break;
            tc_fence_after();
            const int64_t grow = (int64_t)tile * BM + r;
            if (p.mode == 2) {
                // partial of unit `split`, column-major: the first product's l columns, then
                // the second's vcols
                // row-major, Mdim rows of pitch pair_pitch(w); l is a multiple of 4, so the
                // second product's columns start 16-byte aligned.  One unit per CTA: the
                // unit's block is staged in the shared memory of the operand rings (free
                // once its MMAs have completed) and written with one bulk copy.
                const int w = p.l + p.vcols;
                const int wp = pair_pitch(w);
                const uint32_t lanes = (uint32_t)(q * 32) << 16;
                const bool ok = grow < p.Mdim;
                float* gdst = p.partial + (int64_t)split * p.Mdim * wp;
                if (p.units <= (int)gridDim.x) {
                    float* row = reinterpret_cast<float*>(smem) + (int64_t)r * wp;
                    epi_row_span(tmem + lanes, p.lpad, row, p.l, ok);
                    epi_row_span(tmem + 128u + lanes, p.vpad, row + p.l, p.vcols, ok);
                    fence_proxy_async();  // the staged block is read by the bulk copy (async proxy)
                    __syncwarp();
                    if (lane == 0) mbar_arrive(EPI);
                    if (warp == 6 && lane == 0) {
                        if (wait_bar(EPI, 0, abort_flag, p.status, lim)) {
                            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                                         "r"(smem_u32(smem)), "r"((uint32_t)(p.Mdim * wp * 4))
                                         : "memory");
                            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                            asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
                        }
                    }
                } else {
                    float* row = gdst + grow * wp;
                    epi_row_span(tmem + lanes, p.lpad, row, p.l, ok);
                    epi_row_span(tmem + 128u + lanes, p.vpad, row + p.l, p.vcols, ok);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(ACC_empty0);
                continue;
            }
            if (p.direct && p.trans_out) {
                // out is l x Mdim: for each column the warp's 32 rows are 32 consecutive floats
                epi_span(tmem + buf * 128u + ((uint32_t)(q * 32) << 16), p.lpad, p.out + grow, p.Mdim, p.l,
                         grow < p.Mdim);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(ACC_empty0 + 8u * buf);
                continue;
            }
            float* dst = p.direct ? p.out + grow * p.l : p.partial + ((int64_t)split * p.Mdim + grow) * p.l;
            const bool vec = (p.l & 3) == 0;
            for (int c0 = 0; c0 < p.lpad; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + buf * 128u + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                if (grow < p.Mdim) {
                    if (vec && c0 + 16 <= p.l) {
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            *reinterpret_cast<float4*>(dst + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0 + j < p.l) dst[c0 + j] = v[j];
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(ACC_empty0 + 8u * buf);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// X (K x l float32, row-major) -> bf16 hi (and lo) in the swizzled K-major tile
// layout [ceil(K/64)][lpad rows][128 B]; every byte of every tile is written
// (zero past K and past l), so no uninitialised value reaches the MMA.
__global__ void pack_x_kernel(const float* __restrict__ X, int64_t K, int l, int lpad, int nterms,
                              uint8_t* __restrict__ xhi, uint8_t* __restrict__ xlo) {
    const int64_t groups = (K + BK - 1) / BK * (BK / 8);
    const int64_t total = groups * lpad;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(t % lpad);
        const int64_t k0 = (t / lpad) * 8;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = (j < l && k0 + e < K) ? X[(k0 + e) * l + j] : 0.f;
        uint4 hi;
        hi.x = pack_bf16(x[0], x[1]);
        hi.y = pack_bf16(x[2], x[3]);
        hi.z = pack_bf16(x[4], x[5]);
        hi.w = pack_bf16(x[6], x[7]);
        const int64_t kb = k0 / BK;
        const int oc = (int)((k0 % BK) / 8);
        const size_t off = (size_t)kb * lpad * 128 + (size_t)(j >> 3) * 1024 + (size_t)(j & 7) * 128 +
                           (size_t)((oc ^ (j & 7)) << 4);
        *reinterpret_cast<uint4*>(xhi + off) = hi;
        if (nterms == 3) {
            const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&hi);
            float y[8];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(h2[e]);
                y[2 * e] = x[2 * e] - f.x;
                y[2 * e + 1] = x[2 * e + 1] - f.y;
            }
            uint4 lo;
            lo.x = pack_bf16(y[0], y[1]);
            lo.y = pack_bf16(y[2], y[3]);
            lo.z = pack_bf16(y[4], y[5]);
            lo.w = pack_bf16(y[6], y[7]);
            *reinterpret_cast<uint4*>(xlo + off) = lo;
        }
    }
}

// out = sum of the partials (accumulate: out + sum) in split order as a two-sum
// pair (pair_sum.cuh: about twice float32's precision, off the slow float64
// pipe), rounded once.
__global__ void split_sum_kernel(const float* __restrict__ partial, int splits, int64_t count, float* __restrict__ out,
                                 int accumulate) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        float2 s = make_float2(accumulate ? out[e] : 0.f, 0.f);
        int q = 0;
        for (; q + 4 <= splits; q += 4) {
            float x[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) x[t] = partial[(int64_t)(q + t) * count + e];
#pragma unroll
            for (int t = 0; t < 4; ++t) two_sum_add(s, x[t]);
        }
        for (; q < splits; ++q) two_sum_add(s, partial[(int64_t)q * count + e]);
        out[e] = pair_value(s);
    }
}

// T^T (k x l) and V (k x k) from the mode-2 unit partials (row-major, k rows of
// pitch pair_pitch(l + k) each): entry e summed over the units as two-sum pairs (pair_sum.cuh), eight
// slices of units per entry combined in slice order (a fixed order: bit-identical
// from run to run).  V's entry (r, c) is taken from the unit sums with r <= c and
// written to both halves, so V is exactly symmetric.
constexpr int HV_SLICES = 8;
__global__ void __launch_bounds__(256) hv_reduce_kernel(const float* __restrict__ part, int units, int k, int l,
                                                        float* __restrict__ Tt, float* __restrict__ V) {
    __shared__ float2 acc_s[HV_SLICES][32];
    const int slice = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int w = l + k;
    const int64_t cnt = (int64_t)k * w;
    const int wp = pair_pitch(w);
    const int64_t ustride = (int64_t)k * wp;
    const int64_t e = (int64_t)blockIdx.x * 32 + lane;
    const int64_t ep = e / w * wp + e % w;  // entry e = (row e / w, column e % w) in a unit's block
    float2 acc = make_float2(0.f, 0.f);
    if (e < cnt) {
        int u = slice;
        for (; u + 3 * HV_SLICES < units; u += 4 * HV_SLICES) {
            float x[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) x[t] = part[(int64_t)(u + t * HV_SLICES) * ustride + ep];
#pragma unroll
            for (int t = 0; t < 4; ++t) two_sum_add(acc, x[t]);
        }
        for (; u < units; u += HV_SLICES) two_sum_add(acc, part[(int64_t)u * ustride + ep]);
    }
    acc_s[slice][lane] = acc;
    __syncthreads();
    if (slice != 0 || e >= cnt) return;
    for (int t = 1; t < HV_SLICES; ++t) acc = pair_add(acc, acc_s[t][lane]);
    const float f = pair_value(acc);
    const int r = (int)(e / w), c = (int)(e % w);
    if (c < l) {
        Tt[(int64_t)r * l + c] = f;
    } else {
        const int cv = c - l;
        if (r <= cv) {
            V[(int64_t)r * k + cv] = f;
            V[(int64_t)cv * k + r] = f;
        }
    }
}

// ---------------------------------------------------------------- host
int lpad_of(int l) { return (l + 15) / 16 * 16; }

// Work units: (tile, contraction chunk of at most kmax k-steps); the chunk count
// is raised further when that evens out the last wave over the SMs.
void choose_splits(int tiles, int ksteps, int sms, int kmax, int* splits, int* ksp) {
    int s0 = (ksteps + kmax - 1) / kmax;
    int best = s0;
    double best_eff = 0.0;
    for (int s = s0; s <= 4 * s0 + 8; ++s) {
        if (s > 1 && ksteps / s < 4) break;
        const double units = (double)tiles * s;
        const double waves = std::ceil(units / sms);
        const double eff = units / (waves * sms);
        if (eff > best_eff + 0.02) {
            best_eff = eff;
            best = s;
        }
        if (eff > 0.95) break;
    }
    *ksp = (ksteps + best - 1) / best;
    *splits = (ksteps + *ksp - 1) / *ksp;
}

bool run_tc(rnmf_ctx* ctx, const TcScratch& s, int mode, const float* A, int64_t lda, int64_t m, int64_t n,
            const float* X, float* out, int l, int nterms, bool accumulate, bool trans_out = false,
            int cls = -1) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const int64_t Mdim = mode == 0 ? m : n;
    const int64_t Kdim = mode == 0 ? n : m;
    const int lpad = lpad_of(l);
    const int ksteps = (int)((Kdim + BK - 1) / BK);
    const int tiles = (int)((Mdim + BM - 1) / BM);
    int splits, ksp;
    choose_splits(tiles, ksteps, ctx->num_sms, nterms == 3 ? 64 : 256, &splits, &ksp);
    // pack X
    {
        const int64_t total = (int64_t)ksteps * (BK / 8) * lpad;
        int g = (int)((total + 255) / 256);
        if (g > ctx->num_sms * 8) g = ctx->num_sms * 8;
        prof_begin(ctx);
        pack_x_kernel<<<g, 256, 0, ctx->stream>>>(X, Kdim, l, lpad, nterms, (uint8_t*)s.xhi, (uint8_t*)s.xlo);
        if (!launch_done(ctx, K_TC_PACK, 4.0 * Kdim * l + 2.0 * nterms / 1.5 * ksteps * lpad * 64, 0)) return false;
    }
    // tensor map of A (float32, dims {n, m}, row pitch lda)
    CUtensorMap tm;
    memset(&tm, 0, sizeof tm);
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
    cuuint64_t strides[1] = {(cuuint64_t)lda * 4};
    cuuint32_t box[2], estr[2] = {1, 1};
    CUtensorMapSwizzle sw;
    if (mode == 0) {
        box[0] = 32;
        box[1] = BM;
        sw = CU_TENSOR_MAP_SWIZZLE_128B;
    } else {
        box[0] = BM;
        box[1] = BK;
        sw = CU_TENSOR_MAP_SWIZZLE_NONE;
    }
    CUresult cr = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return false;
    TcParams p;
    p.mode = mode;
    p.Mdim = Mdim;
    p.Kdim = Kdim;
    p.l = l;
    p.lpad = lpad;
    p.ksteps = ksteps;
    p.tiles = tiles;
    p.splits = splits;
    p.ksp = ksp;
    p.units = tiles * splits;
    p.direct = splits == 1 && !accumulate;
    p.trans_out = trans_out ? 1 : 0;
    if (trans_out && !p.direct) return false;
    p.vcols = 0;
    p.vpad = 16;
    p.xhi = (const uint8_t*)s.xhi;
    p.xlo = (const uint8_t*)s.xlo;
    p.out = out;
    p.partial = (float*)s.partial;
    p.status = ctx->d_status;
    p.spin_limit = RNMF_DEFAULT_SPIN_LIMIT;
    const int grid = p.units < ctx->num_sms ? p.units : ctx->num_sms;
    const double bytes = 4.0 * (double)m * n + 4.0 * (double)Mdim * l * splits;
    const double flops = 2.0 * (double)m * n * l * nterms;
    prof_begin(ctx);
    if (nterms == 3) {
        cudaFuncSetAttribute(tc_gemm_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<3>::SMEM);
        tc_gemm_kernel<3><<<grid, NTHREADS, Cfg<3>::SMEM, ctx->stream>>>(tm, p);
    } else {
        cudaFuncSetAttribute(tc_gemm_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<1>::SMEM);
        tc_gemm_kernel<1><<<grid, NTHREADS, Cfg<1>::SMEM, ctx->stream>>>(tm, p);
    }
    if (!launch_done(ctx, cls >= 0 ? cls : (mode == 0 ? K_TC_AX : K_TC_ATX), bytes, flops)) return false;
    if (!p.direct) {
        const int64_t count = Mdim * l;
        int g = (int)((count + 255) / 256);
        if (g > ctx->num_sms * 8) g = ctx->num_sms * 8;
        prof_begin(ctx);
        split_sum_kernel<<<g, 256, 0, ctx->stream>>>(p.partial, splits, count, out, accumulate ? 1 : 0);
        if (!launch_done(ctx, K_TC_REDUCE, 4.0 * count * (splits + 1 + (accumulate ? 1 : 0)), (double)count * splits))
            return false;
    }
    return true;
}

// Largest split-K partial buffer either product can need (float32).
size_t tc_partial_bytes(int64_t m, int64_t n, int l) {
    size_t worst = 0;
    for (int mode = 0; mode < 2; ++mode) {
        const int64_t Mdim = mode == 0 ? m : n, Kdim = mode == 0 ? n : m;
        const int ksteps = (int)((Kdim + BK - 1) / BK);
        const int s_max = 4 * ((ksteps + 63) / 64) + 8;
        const size_t b = (size_t)(s_max < ksteps ? s_max : ksteps) * Mdim * l * 4;
        if (b > worst) worst = b;
    }
    return worst;
}

}  // namespace

bool tc_available() { return encode_fn() != nullptr; }

size_t tc_scratch_bytes(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int precision) {
    (void)ctx;
    if (precision == RNMF_PREC_FP32) return 0;
    const int64_t big = m > n ? m : n;
    const size_t pack = (size_t)((big + BK - 1) / BK) * lpad_of(l) * 128;
    return 2 * arena_round(pack) + arena_round(tc_partial_bytes(m, n, l));
}

TcScratch tc_scratch_take(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int precision) {
    TcScratch s;
    if (precision == RNMF_PREC_FP32) return s;
    const int64_t big = m > n ? m : n;
    s.xpack_bytes = (size_t)((big + BK - 1) / BK) * lpad_of(l) * 128;
    s.xhi = arena_take(ctx, s.xpack_bytes);
    s.xlo = arena_take(ctx, s.xpack_bytes);
    s.partial_bytes = tc_partial_bytes(m, n, l);
    s.partial = arena_take(ctx, s.partial_bytes);
    return s;
}

bool tc_gemm_ax(rnmf_ctx* ctx, const TcScratch& s, const float* A, int64_t lda, const float* X, float* Y, int64_t m,
                int64_t n, int l, int nterms, bool accumulate) {
    return run_tc(ctx, s, 0, A, lda, m, n, X, Y, l, nterms, accumulate);
}

bool tc_gemm_atx(rnmf_ctx* ctx, const TcScratch& s, const float* A, int64_t lda, const float* X, float* Z, int64_t m,
                 int64_t n, int l, int nterms, bool accumulate) {
    return run_tc(ctx, s, 1, A, lda, m, n, X, Z, l, nterms, accumulate);
}

// ------------------------------------------------ the H half of a sweep on tensor cores
namespace {
size_t hh_bpack_bytes(int64_t n, int l) { return (size_t)((n + BK - 1) / BK) * lpad_of(l) * 128; }
size_t hh_wpack_bytes(int l, int k) { return (size_t)((l + BK - 1) / BK) * lpad_of(k) * 128; }
int hh_units(rnmf_ctx* ctx, int64_t n, int* ksp) {
    const int ksteps = (int)((n + BK - 1) / BK);
    *ksp = (ksteps + ctx->num_sms - 1) / ctx->num_sms;
    return (ksteps + *ksp - 1) / *ksp;
}
}  // namespace

bool tc_hhalf_fits(int64_t n, int l, int k, const float* Bt, const float* H) {
    return tc_available() && n > 0 && l >= 1 && l <= BM && k >= 1 && k <= BM && l % 4 == 0 && n % 4 == 0 &&
           (reinterpret_cast<uintptr_t>(Bt) & 15) == 0 && (reinterpret_cast<uintptr_t>(H) & 15) == 0;
}

bool tc_gram_fits(int64_t m, int k, const float* Wc) {
    return tc_available() && m > 0 && k >= 1 && k <= BM && m % 4 == 0 && (reinterpret_cast<uintptr_t>(Wc) & 15) == 0;
}

namespace {
size_t hh_part_bytes(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int k) {
    int ksp;
    const size_t pn = (size_t)hh_units(ctx, n, &ksp) * k * pair_pitch(l + k) * 4;
    const size_t pm = (size_t)hh_units(ctx, m, &ksp) * k * pair_pitch(k) * 4;
    return pn > pm ? pn : pm;
}
}  // namespace

size_t tc_hhalf_bytes(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int k) {
    return 2 * arena_round(hh_bpack_bytes(n, l)) + 2 * arena_round(hh_wpack_bytes(l, k)) +
           arena_round(hh_part_bytes(ctx, m, n, l, k));
}

TcHhalf tc_hhalf_take(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int k) {
    TcHhalf h;
    h.bhi = arena_take(ctx, hh_bpack_bytes(n, l));
    h.blo = arena_take(ctx, hh_bpack_bytes(n, l));
    h.whi = arena_take(ctx, hh_wpack_bytes(l, k));
    h.wlo = arena_take(ctx, hh_wpack_bytes(l, k));
    h.part = (float*)arena_take(ctx, hh_part_bytes(ctx, m, n, l, k));
    return h;
}

bool tc_hhalf_pack_b(rnmf_ctx* ctx, const TcHhalf& h, const float* Bt, int64_t n, int l) {
    const int lpad = lpad_of(l);
    const int64_t total = (n + BK - 1) / BK * (BK / 8) * lpad;
    int g = (int)((total + 255) / 256);
    if (g > ctx->num_sms * 8) g = ctx->num_sms * 8;
    prof_begin(ctx);
    pack_x_kernel<<<g, 256, 0, ctx->stream>>>(Bt, n, l, lpad, 3, (uint8_t*)h.bhi, (uint8_t*)h.blo);
    return launch_done(ctx, K_TC_PACK, 4.0 * n * l + 4.0 * total * 8, 0);
}

bool tc_hhalf_r(rnmf_ctx* ctx, const TcHhalf& h, const float* Bt, int64_t n, int l, const float* Wt, int k,
                float* Rt) {
    TcScratch s;
    s.xhi = h.whi;
    s.xlo = h.wlo;
    return run_tc(ctx, s, 0, Bt, l, n, l, Wt, Rt, k, 3, false, true, K_R_TC);
}

namespace {
// Mode 2 over the rows of X (c x N, row-major, pitch N): out1 (c x l) = X Y with Y
// (N x l) pre-packed in (yhi, ylo) (l = 0: none), out2 (c x c) = X X^T.
bool run_pair(rnmf_ctx* ctx, float* part, const float* X, int64_t N, int c, const void* yhi, const void* ylo, int l,
              float* out1, float* out2, int cls) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    // tensor map of X (float32 c x N, row pitch N): mode 0's 128-row x 32-column boxes
    CUtensorMap tm;
    memset(&tm, 0, sizeof tm);
    cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)c};
    cuuint64_t strides[1] = {(cuuint64_t)N * 4};
    cuuint32_t box[2] = {32, BM}, estr[2] = {1, 1};
    if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    int ksp;
    const int units = hh_units(ctx, N, &ksp);
    TcParams p;
    p.mode = 2;
    p.Mdim = c;
    p.Kdim = N;
    p.l = l;
    p.lpad = l > 0 ? lpad_of(l) : 0;
    p.ksteps = (int)((N + BK - 1) / BK);
    p.tiles = 1;
    p.splits = units;
    p.ksp = ksp;
    p.units = units;
    p.direct = 0;
    p.trans_out = 0;
    p.vcols = c;
    p.vpad = lpad_of(c);
    p.xhi = (const uint8_t*)yhi;
    p.xlo = (const uint8_t*)ylo;
    p.out = nullptr;
    p.partial = part;
    p.status = ctx->d_status;
    p.spin_limit = RNMF_DEFAULT_SPIN_LIMIT;
    const int grid = units < ctx->num_sms ? units : ctx->num_sms;
    cudaFuncSetAttribute(tc_gemm_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<3>::SMEM);
    prof_begin(ctx);
    tc_gemm_kernel<3><<<grid, NTHREADS, Cfg<3>::SMEM, ctx->stream>>>(tm, p);
    const double w = (double)l + c;
    if (!launch_done(ctx, cls, 4.0 * N * c + 4.0 * (double)p.ksteps * p.lpad * 64 + 4.0 * units * c * w,
                     2.0 * 3 * N * c * w))
        return false;
    const int64_t cnt = (int64_t)c * (l + c);
    prof_begin(ctx);
    hv_reduce_kernel<<<(unsigned)((cnt + 31) / 32), 256, 0, ctx->stream>>>(part, units, c, l, out1, out2);
    return launch_done(ctx, cls, 4.0 * cnt * units + 4.0 * (l * c + c * c), (double)cnt * units);
}
}  // namespace

bool tc_hhalf_tv(rnmf_ctx* ctx, const TcHhalf& h, const float* H, int64_t n, int l, int k, float* Tt, float* V) {
    return run_pair(ctx, h.part, H, n, k, h.bhi, h.blo, l, Tt, V, K_TV_TC);
}

bool tc_hhalf_gram(rnmf_ctx* ctx, const TcHhalf& h, const float* Wc, int64_t m, int k, float* S) {
    return run_pair(ctx, h.part, Wc, m, k, nullptr, nullptr, 0, nullptr, S, K_S_TC);
}
