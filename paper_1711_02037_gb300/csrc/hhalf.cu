// hhalf.cu - the products of the H half of a randomized HALS sweep, on tiles
// of columns held in shared memory.
//
// Section 3.2 H rule (Algorithm 1's loop body): the H rows need R = B^T W~
// (n x k), and the W half that follows needs T = B H^T (l x k) and V = H H^T
// (k x k) of the new H.  Two persistent kernels take tiles of HH_NC columns:
//   rtile: R^T for the tile from the tile's rows of B^T and W~ (held in shared
//     memory for the whole launch); each thread owns 4 x 8 entries of R and sums
//     the l products in index order.  Two blocks per SM (about 110 KB of shared
//     memory each): one block's loads overlap the other's products.
//   tv: the tile's rows of B^T and columns of the new H (transposed) are added
//     into the block's partial sums of T and V, held in registers across tiles
//     (32 x 32 warp tiles; V's upper tiles only); a second launch adds the
//     blocks' partial sums in block order (two-sum pairs) and writes T^T and V.
// The H rows themselves (the Gauss-Seidel recurrence) run between the two in
// hals_rows_kernel (hals.cu).  B^T is read twice and H once more than the
// recurrence needs, against a generic product kernel for each of R, T and V.
#include "async_copy.cuh"
#include "pair_sum.cuh"
#include "rnmf_internal.cuh"

namespace {

constexpr int HH_NT = 256;
constexpr int HH_NC = 64;           // columns per tile
constexpr int HH_WT = 4;            // warp tiles (32 x 32 entries of T or V) per warp at most

// Tile geometry for l, k: kp = k to 8, l4 = l to 4; pb = pitch of a B^T tile (l to 32,
// + 4: = 4 (mod 32), so the 4 x 8 blocks of R read 16 rows 4 banks apart, and a
// warp tile's 32 columns stay inside a row); ph = pitch of an H^T tile (k to 32,
// + 4); na, nb = 32-blocks of l and k; nt, nv = T and V warp tiles, jobs = both.
struct HhLayout {
    int kp, l4, l8, pb, ph;
    int nb, na, nt, nv, jobs;
};

__host__ __device__ inline HhLayout hh_layout(int l, int k) {
    HhLayout L;
    L.kp = (k + 7) / 8 * 8;
    L.l4 = (l + 3) / 4 * 4;
    L.l8 = (l + 7) / 8 * 8;
    L.pb = (l + 31) / 32 * 32 + 4;
    L.ph = (k + 31) / 32 * 32 + 4;
    L.nb = (k + 31) / 32;
    L.na = (l + 31) / 32;
    L.nt = L.na * L.nb;
    L.nv = L.nb * (L.nb + 1) / 2;
    L.jobs = L.nt + L.nv;
    return L;
}

// rtile shared memory (floats): W~ (l4 x kp), a B^T tile (HH_NC x pb), an R tile (HH_NC x kp)
__host__ __device__ inline size_t rt_floats(const HhLayout& L) {
    return (size_t)L.l4 * L.kp + (size_t)HH_NC * L.pb + (size_t)HH_NC * L.kp;
}
// tv shared memory (floats): two (B^T tile HH_NC x pb, H^T tile HH_NC x ph) pairs
__host__ __device__ inline size_t tv_floats(const HhLayout& L) { return 2 * (size_t)HH_NC * (L.pb + L.ph); }

// rows c0.. of B^T into a tile (rows past nc zero; columns past l stay as they are)
__device__ __forceinline__ void hh_load_bt(float* Bs, const float* __restrict__ Bt, int64_t c0, int nc, int l, int pb,
                                           int vec4) {
    if (vec4) {
        const int l4 = l / 4;
        for (int e = threadIdx.x; e < HH_NC * l4; e += HH_NT) {
            const int c = e / l4, i4 = e % l4;
            cp_async16(Bs + c * pb + 4 * i4, c < nc ? Bt + (c0 + c) * l + 4 * i4 : Bt, c < nc);
        }
    } else {
        for (int e = threadIdx.x; e < HH_NC * l; e += HH_NT) {
            const int c = e / l, i = e % l;
            cp_async4(Bs + c * pb + i, c < nc ? Bt + (c0 + c) * l + i : Bt, c < nc);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ int hh_tile_cols(int64_t n, int64_t t) {
    return (int)(n - t * HH_NC < HH_NC ? n - t * HH_NC : HH_NC);
}

// R^T (k x n) = (B^T W~)^T, tile by tile.
__global__ void __launch_bounds__(HH_NT, 2) rtile_kernel(const float* __restrict__ Bt, int64_t n, int l,
                                                         const float* __restrict__ Wt, int k, float* __restrict__ Rt,
                                                         int vec4) {
    extern __shared__ __align__(16) float sm[];
    const HhLayout L = hh_layout(l, k);
    const int kp = L.kp, pb = L.pb;
    float* Ws = sm;
    float* const Bs0 = sm + (size_t)L.l4 * kp;
    float* Rs = Bs0 + (size_t)HH_NC * pb;
    const int tid = threadIdx.x;
    for (int e = tid; e < L.l4 * kp; e += HH_NT) {
        const int i = e / kp, j = e % kp;
        Ws[e] = (i < l && j < k) ? Wt[(int64_t)i * k + j] : 0.f;
    }
    for (int e = tid; e < HH_NC * pb; e += HH_NT) Bs0[e] = 0.f;  // columns past l stay zero
    __syncthreads();
    const int64_t ntiles = (n + HH_NC - 1) / HH_NC;
    const int tc = tid & 15, tj = tid >> 4;  // rows tc + 16 a of the tile, entries 8 tj..
    const bool active = tj < kp / 8;
    if ((int64_t)blockIdx.x < ntiles)
        hh_load_bt(Bs0, Bt, (int64_t)blockIdx.x * HH_NC, hh_tile_cols(n, blockIdx.x), l, pb, vec4);
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t c0 = tile * HH_NC;
        const int nc = hh_tile_cols(n, tile);
        if (tile != blockIdx.x) hh_load_bt(Bs0, Bt, c0, nc, l, pb, vec4);
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        if (active) {
            const float* B = Bs0;
            float acc[4][8];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
            for (int i = 0; i < L.l4; i += 4) {
                float4 bv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) bv[a] = *reinterpret_cast<const float4*>(B + (tc + 16 * a) * pb + i);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float4 w0 = *reinterpret_cast<const float4*>(Ws + (i + r) * kp + 8 * tj);
                    const float4 w1 = *reinterpret_cast<const float4*>(Ws + (i + r) * kp + 8 * tj + 4);
                    const float ww[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const float bb = r == 0 ? bv[a].x : r == 1 ? bv[a].y : r == 2 ? bv[a].z : bv[a].w;
#pragma unroll
                        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(bb, ww[b], acc[a][b]);
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                float* dst = Rs + (tc + 16 * a) * kp + 8 * tj;
                *reinterpret_cast<float4*>(dst) = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
                *reinterpret_cast<float4*>(dst + 4) = make_float4(acc[a][4], acc[a][5], acc[a][6], acc[a][7]);
            }
        }
        __syncthreads();
        for (int e = tid; e < k * HH_NC; e += HH_NT) {
            const int j = e / HH_NC, c = e % HH_NC;
            if (c < nc) Rt[(int64_t)j * n + c0 + c] = Rs[c * kp + j];
        }
        __syncthreads();  // the B^T and R tiles are free for the next tile
    }
}

// Warp tile `t` of the partial sums (32 x 32 entries): T tiles (rows 32 r of T = rows of
// B H^T, columns 32 c; source 1 = the B^T tile) first, then V's upper tiles (r <= c;
// source 1 = the H^T tile).  Lane (tr, tc) = (lane % 8, lane / 8) owns rows 4 tr..,
// columns 8 tc..: per column of the tile it reads one 16-byte piece of source 1 and two
// of the H^T tile, all 32 lanes within one 128-byte row segment of each (no bank conflict).
struct HhTile {
    int src_b;  // 1: source 1 is the B^T tile, 0: H^T
    int o1, o2;
};

__device__ __forceinline__ HhTile hh_tile(const HhLayout& L, int t) {
    HhTile T;
    if (t < L.nt) {
        T.src_b = 1;
        T.o1 = 32 * (t % L.na);
        T.o2 = 32 * (t / L.na);
    } else {
        int v = t - L.nt, r = 0;
        while (v >= L.nb - r) {
            v -= L.nb - r;
            ++r;
        }
        T.src_b = 0;
        T.o1 = 32 * r;
        T.o2 = 32 * (r + v);
    }
    return T;
}

__device__ __forceinline__ void hh_accumulate(float (&acc)[4][8], const float* s1, int p1, const float* ht, int ph,
                                              int o1, int o2) {
#pragma unroll 4
    for (int c = 0; c < HH_NC; ++c) {
        const float4 a = *reinterpret_cast<const float4*>(s1 + c * p1 + o1);
        const float4 b0 = *reinterpret_cast<const float4*>(ht + c * ph + o2);
        const float4 b1 = *reinterpret_cast<const float4*>(ht + c * ph + o2 + 4);
        const float x[4] = {a.x, a.y, a.z, a.w};
        const float y[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(x[u], y[v], acc[u][v]);
    }
}

// T and V partial sums of the block's tiles: part[(t * gridDim.x + block) * 1024 + 32 r + c]
// for warp tile t, entry (r, c).  Warp w takes the warp tiles w, w + 8, ...
__global__ void __launch_bounds__(HH_NT, 1) tv_kernel(const float* __restrict__ Bt, int64_t n, int l,
                                                      const float* __restrict__ H, int k, int vec4,
                                                      float* __restrict__ part) {
    extern __shared__ __align__(16) float sm[];
    const HhLayout L = hh_layout(l, k);
    const int kp = L.kp, pb = L.pb, ph = L.ph;
    float* const Bs0 = sm;
    float* const Bs1 = sm + (size_t)HH_NC * pb;
    float* const Ht0 = sm + 2 * (size_t)HH_NC * pb;
    float* const Ht1 = Ht0 + (size_t)HH_NC * ph;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tr = lane & 7, tc = lane >> 3;
    for (int e = tid; e < 2 * HH_NC * (pb + ph); e += HH_NT) sm[e] = 0.f;  // padding stays zero
    __syncthreads();
    // columns c0.. of H transposed into an H^T tile (rows past nc and columns past k zero)
    auto load_ht = [&](float* T, int64_t c0, int nc) {
        for (int e = tid; e < kp * HH_NC; e += HH_NT) {
            const int j = e / HH_NC, c = e % HH_NC;
            const bool ok = j < k && c < nc;
            cp_async4(T + c * ph + j, ok ? H + (int64_t)j * n + c0 + c : H, ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const int64_t ntiles = (n + HH_NC - 1) / HH_NC;
    HhTile W[HH_WT];
    bool on[HH_WT];
#pragma unroll
    for (int q = 0; q < HH_WT; ++q) {
        const int t = warp + 8 * q;
        on[q] = t < L.jobs;
        W[q] = hh_tile(L, on[q] ? t : 0);
    }
    float acc[HH_WT][4][8];
#pragma unroll
    for (int q = 0; q < HH_WT; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 8; ++v) acc[q][u][v] = 0.f;
    int buf = 0;
    if ((int64_t)blockIdx.x < ntiles) {
        const int nc0 = hh_tile_cols(n, blockIdx.x);
        hh_load_bt(Bs0, Bt, (int64_t)blockIdx.x * HH_NC, nc0, l, pb, vec4);
        load_ht(Ht0, (int64_t)blockIdx.x * HH_NC, nc0);
    }
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, buf ^= 1) {
        const int64_t nxt = tile + gridDim.x;
        if (nxt < ntiles) {
            const int ncn = hh_tile_cols(n, nxt);
            hh_load_bt(buf ? Bs0 : Bs1, Bt, nxt * HH_NC, ncn, l, pb, vec4);
            load_ht(buf ? Ht0 : Ht1, nxt * HH_NC, ncn);
            asm volatile("cp.async.wait_group 2;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const float* Bc = buf ? Bs1 : Bs0;
        const float* Hc = buf ? Ht1 : Ht0;
#pragma unroll
        for (int q = 0; q < HH_WT; ++q)
            if (on[q])
                hh_accumulate(acc[q], W[q].src_b ? Bc : Hc, W[q].src_b ? pb : ph, Hc, ph, W[q].o1 + 4 * tr,
                              W[q].o2 + 8 * tc);
        __syncthreads();  // this buffer pair is refilled two tiles later
    }
#pragma unroll
    for (int q = 0; q < HH_WT; ++q) {
        if (!on[q]) continue;
        float* dst = part + ((size_t)(warp + 8 * q) * gridDim.x + blockIdx.x) * 1024;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 8; v += 4)
                *reinterpret_cast<float4*>(dst + 32 * (4 * tr + u) + 8 * tc + v) =
                    make_float4(acc[q][u][v], acc[q][u][v + 1], acc[q][u][v + 2], acc[q][u][v + 3]);
    }
}

// T^T (k x l) and V (k x k): entry (r, c) of warp tile t summed over the blocks in block
// order as a two-sum pair (pair_sum.cuh: about twice float32's precision, off the
// float64 pipe), rounded once.
__global__ void __launch_bounds__(128) tv_reduce_kernel(const float* __restrict__ part, int nblk, int l, int k,
                                                        float* __restrict__ Tt, float* __restrict__ V) {
    const HhLayout L = hh_layout(l, k);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= L.jobs * 1024) return;
    const int t = e / 1024, rc = e % 1024, r = rc / 32, c = rc % 32;
    const HhTile T = hh_tile(L, t);
    const int row = T.o1 + r, col = T.o2 + c;
    if (T.src_b ? (row >= l || col >= k) : (row >= k || col >= k || row > col)) return;
    const float* src = part + (size_t)t * nblk * 1024 + rc;
    float2 acc = make_float2(0.f, 0.f);
    int b = 0;
    for (; b + 8 <= nblk; b += 8) {
        float x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = src[(size_t)(b + u) * 1024];
#pragma unroll
        for (int u = 0; u < 8; ++u) two_sum_add(acc, x[u]);
    }
    for (; b < nblk; ++b) two_sum_add(acc, src[(size_t)b * 1024]);
    const float f = pair_value(acc);
    if (T.src_b) {
        Tt[(int64_t)col * l + row] = f;  // T(row, col)
    } else {
        V[row * k + col] = f;
        V[col * k + row] = f;
    }
}

}  // namespace

bool hhalf_fits(int l, int k) {
    if (l > RNMF_MAX_L || k > RNMF_MAX_L) return false;
    const HhLayout L = hh_layout(l, k);
    return L.jobs <= 8 * HH_WT && rt_floats(L) * 4 <= 227 * 1024 && tv_floats(L) * 4 <= 227 * 1024;
}

static unsigned hh_grid(rnmf_ctx* ctx, int64_t n) {
    const int64_t ntiles = (n + HH_NC - 1) / HH_NC;
    return (unsigned)(ntiles < ctx->num_sms ? ntiles : ctx->num_sms);
}

size_t hhalf_scratch_bytes(rnmf_ctx* ctx, int64_t n, int l, int k) {
    return (size_t)hh_layout(l, k).jobs * hh_grid(ctx, n) * 1024 * sizeof(float);
}

static int hh_vec4(const float* Bt, int l) { return (l % 4 == 0 && (reinterpret_cast<uintptr_t>(Bt) & 15) == 0) ? 1 : 0; }

bool launch_rtile(rnmf_ctx* ctx, const float* Bt, int64_t n, int l, const float* Wt, int k, float* Rt) {
    if (n <= 0) return true;
    const size_t smem = rt_floats(hh_layout(l, k)) * sizeof(float);
    cudaFuncSetAttribute(rtile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    prof_begin(ctx);
    const int64_t nt2 = (n + HH_NC - 1) / HH_NC;
    const unsigned g2 = (unsigned)(nt2 < 2 * ctx->num_sms ? nt2 : 2 * ctx->num_sms);
    rtile_kernel<<<g2, HH_NT, smem, ctx->stream>>>(Bt, n, l, Wt, k, Rt, hh_vec4(Bt, l));
    return launch_done(ctx, K_RTILE, 4.0 * n * l + 4.0 * n * k + 4.0 * l * k, 2.0 * n * l * k);
}

bool launch_tv(rnmf_ctx* ctx, const float* Bt, int64_t n, int l, const float* H, int k, float* Tt, float* V,
               float* scratch) {
    if (n <= 0) return true;
    const HhLayout L = hh_layout(l, k);
    const size_t smem = tv_floats(L) * sizeof(float);
    cudaFuncSetAttribute(tv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const unsigned grid = hh_grid(ctx, n);
    prof_begin(ctx);
    tv_kernel<<<grid, HH_NT, smem, ctx->stream>>>(Bt, n, l, H, k, hh_vec4(Bt, l), scratch);
    // compulsory traffic: B^T and H read once; flops: T (2 n l k) and V's upper blocks
    if (!launch_done(ctx, K_TVTILE, 4.0 * n * l + 4.0 * n * k, 2.0 * n * l * k + 1.0 * n * k * k)) return false;
    const int total = L.jobs * 1024;
    prof_begin(ctx);
    tv_reduce_kernel<<<(total + 127) / 128, 128, 0, ctx->stream>>>(scratch, (int)grid, l, k, Tt, V);
    return launch_done(ctx, K_TVTILE, 4.0 * total * grid + 4.0 * (l * k + k * k), (double)total * grid);
}
