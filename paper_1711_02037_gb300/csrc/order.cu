// order.cu - the shuffled update order of a sweep (Section 3.2: besides the two
// cyclic orders, the components may be visited in a random order that changes
// every sweep).
//
// Sweep t visits the k components in the order pi_t: j = 0..k-1 sorted by
// (u_j, j) ascending, u_j = word (j mod 4) of Philox4x32-10 block
// t ceil(k/4) + floor(j/4), key order_seed, counter stream 4.  Visiting
// components in the order pi is the same as running the cyclic sweep on
// factors whose components are stored in the order pi (W~ and W columns, H
// rows, and both indices of S): every update reads the current values of all
// components, whatever their slots.  So a shuffled sweep gathers the stored
// components into the order pi_t (slot r holds component pi_t(r)), runs the
// cyclic kernels, and the last sweep's order is undone at the end.  sigma[s]
// is the component held in slot s.
#include "philox.cuh"
#include "rnmf_internal.cuh"

namespace {

constexpr uint32_t STREAM_ORDER = 4;

// rho[r] = the slot that holds pi_t(r) now; sigma <- pi_t.  One block, k <= 128 threads.
__global__ void __launch_bounds__(128) order_draw_kernel(uint64_t seed, int t, int k, int* __restrict__ sigma,
                                                         int* __restrict__ rho) {
    __shared__ uint32_t key[128];
    __shared__ int pi[128], slot[128];
    const int j = threadIdx.x;
    const int nb = (k + 3) / 4;
    if (j < k) {
        uint32_t w[4];
        rnmf_rng::block(seed, STREAM_ORDER, 0, (uint64_t)t * nb + (uint64_t)(j >> 2), w);
        key[j] = w[j & 3];
        slot[sigma[j]] = j;
    }
    __syncthreads();
    if (j < k) {
        int r = 0;
        for (int i = 0; i < k; ++i) r += (key[i] < key[j] || (key[i] == key[j] && i < j)) ? 1 : 0;
        pi[r] = j;
    }
    __syncthreads();
    if (j < k) {
        rho[j] = slot[pi[j]];
        sigma[j] = pi[j];
    }
}

// Back to index order: rho[c] = the slot that holds component c; sigma <- identity.
__global__ void __launch_bounds__(128) order_restore_kernel(int k, int* __restrict__ sigma, int* __restrict__ rho) {
    __shared__ int slot[128];
    const int j = threadIdx.x;
    if (j < k) slot[sigma[j]] = j;
    __syncthreads();
    if (j < k) {
        rho[j] = slot[j];
        sigma[j] = j;
    }
}

__global__ void order_identity_kernel(int k, int* __restrict__ sigma) {
    if ((int)threadIdx.x < k) sigma[threadIdx.x] = threadIdx.x;
}

// dst row r = src row rho[r] (rows of `cols` floats)
__global__ void __launch_bounds__(256) gather_rows_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                          int k, int64_t cols, const int* __restrict__ rho) {
    const int64_t total = (int64_t)k * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / cols, c = e % cols;
        dst[e] = src[(int64_t)rho[r] * cols + c];
    }
}

// W~ (l x k): dst column r = src column rho[r]; S (k x k, float and double): both indices
__global__ void __launch_bounds__(256) gather_small_kernel(const float* __restrict__ Wt, float* __restrict__ Wt_d,
                                                           const float* __restrict__ S32, float* __restrict__ S32_d,
                                                           const double* __restrict__ S64, double* __restrict__ S64_d,
                                                           int l, int k, const int* __restrict__ rho) {
    for (int e = threadIdx.x; e < l * k; e += blockDim.x) Wt_d[e] = Wt[(e / k) * k + rho[e % k]];
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int src = rho[e / k] * k + rho[e % k];
        S32_d[e] = S32[src];
        S64_d[e] = S64[src];
    }
}

bool apply_order(rnmf_ctx* ctx, const OrderBufs& ob, float* Wc, int64_t m, float* H, int64_t n, float* Wt, int l,
                 float* S32, double* S64, int k) {
    const int64_t big = m > n ? m : n;
    const unsigned grid = (unsigned)((k * big + 255) / 256 < (int64_t)ctx->num_sms * 8 ? (k * big + 255) / 256
                                                                                       : (int64_t)ctx->num_sms * 8);
    gather_rows_kernel<<<grid, 256, 0, ctx->stream>>>(Wc, ob.tmp, k, m, ob.rho);
    if (cudaMemcpyAsync(Wc, ob.tmp, (size_t)k * m * 4, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
        return false;
    gather_rows_kernel<<<grid, 256, 0, ctx->stream>>>(H, ob.tmp, k, n, ob.rho);
    if (cudaMemcpyAsync(H, ob.tmp, (size_t)k * n * 4, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
        return false;
    float* t32 = ob.tmp;
    float* w32 = ob.tmp + k * k;
    double* t64 = reinterpret_cast<double*>(ob.tmp + ((k * k + l * k + 1) & ~1));
    gather_small_kernel<<<1, 256, 0, ctx->stream>>>(Wt, w32, S32, t32, S64, t64, l, k, ob.rho);
    ctx->launches += 3;
    return cudaGetLastError() == cudaSuccess &&
           cudaMemcpyAsync(Wt, w32, (size_t)l * k * 4, cudaMemcpyDeviceToDevice, ctx->stream) == cudaSuccess &&
           cudaMemcpyAsync(S32, t32, (size_t)k * k * 4, cudaMemcpyDeviceToDevice, ctx->stream) == cudaSuccess &&
           cudaMemcpyAsync(S64, t64, (size_t)k * k * 8, cudaMemcpyDeviceToDevice, ctx->stream) == cudaSuccess;
}

}  // namespace

size_t order_bytes(int64_t m, int64_t n, int l, int k) {
    const int64_t big = m > n ? m : n;
    const size_t small = ((size_t)k * k + (size_t)l * k + 2) * 4 + (size_t)k * k * 8;
    const size_t rows = (size_t)k * big * 4;
    return (rows > small ? rows : small) + 2 * 128 * sizeof(int) + 256;
}

OrderBufs order_take(rnmf_ctx* ctx, int64_t m, int64_t n, int l, int k) {
    OrderBufs ob;
    ob.sigma = (int*)arena_take(ctx, 128 * sizeof(int));
    ob.rho = (int*)arena_take(ctx, 128 * sizeof(int));
    ob.tmp = (float*)arena_take(ctx, order_bytes(m, n, l, k) - 2 * 128 * sizeof(int) - 256);
    return ob;
}

bool order_begin(rnmf_ctx* ctx, const OrderBufs& ob, int k) {
    order_identity_kernel<<<1, 128, 0, ctx->stream>>>(k, ob.sigma);
    ++ctx->launches;
    return cudaGetLastError() == cudaSuccess;
}

bool order_sweep(rnmf_ctx* ctx, const OrderBufs& ob, uint64_t seed, int t, float* Wc, int64_t m, float* H, int64_t n,
                 float* Wt, int l, float* S32, double* S64, int k) {
    order_draw_kernel<<<1, 128, 0, ctx->stream>>>(seed, t, k, ob.sigma, ob.rho);
    ++ctx->launches;
    return cudaGetLastError() == cudaSuccess && apply_order(ctx, ob, Wc, m, H, n, Wt, l, S32, S64, k);
}

bool order_end(rnmf_ctx* ctx, const OrderBufs& ob, float* Wc, int64_t m, float* H, int64_t n, float* Wt, int l,
               float* S32, double* S64, int k) {
    order_restore_kernel<<<1, 128, 0, ctx->stream>>>(k, ob.sigma, ob.rho);
    ++ctx->launches;
    return cudaGetLastError() == cudaSuccess && apply_order(ctx, ob, Wc, m, H, n, Wt, l, S32, S64, k);
}
