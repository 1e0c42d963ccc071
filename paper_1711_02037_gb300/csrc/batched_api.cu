// batched_api.cu - the batched ragged entry point: plan, autotuner, CUDA graph.
//
// A plan is built the first time a batch with a given list of sizes arrives:
// it lays every problem's buffers out in one device allocation, builds the tile
// lists of the shared QB launches (largest problems first, so the persistent
// grids finish together), times candidate sweep configurations on the batch
// itself (the autotuner), and captures the whole pipeline - QB, initial
// factors, sweeps - into one CUDA graph.  Later calls with the same sizes only
// upload the problems' pointers, seeds and options and replay the graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "batched.cuh"

namespace {

struct SweepClass {
    int csize, lq, km, nt;
    int* d_list;
    int count;
};

struct RbPlan {
    std::vector<int64_t> sig;
    int count = 0;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    RbInst* d_inst = nullptr;
    RbTile *t_m = nullptr, *t_n = nullptr, *g_m = nullptr, *g_n = nullptr;
    int n_tm = 0, n_tn = 0, n_gm = 0, n_gn = 0;
    int* d_counters = nullptr;
    int ncounters = 0;
    int* d_lists = nullptr;
    std::vector<RbInst> h_inst;
    std::vector<SweepClass> classes;
    int grid = 0;
    int maxq = 0;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;       // kernel launches per run
    int tuned_nt_small = 256;
    int tuned_tau = 0;
    float tune_ms[8] = {};
};

void plan_free(RbPlan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto e : p->ev) cudaEventDestroy(e);
    for (auto s : p->side) cudaStreamDestroy(s);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->ws) cudaFree(p->ws);
    delete p;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

rnmf_status set_err(rnmf_ctx* ctx, rnmf_status st, const std::string& msg) {
    ctx->last_error = msg;
    return st;
}

rnmf_status cuda_err(rnmf_ctx* ctx, const char* where) {
    cudaError_t e = cudaGetLastError();
    return set_err(ctx, RNMF_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Work of one sweep of problem i (multiply-adds): the W half streams Q once per
// column, the H half and T, V stream B^T and H.
double sweep_work(const RbInst& d) {
    const double lq = rb_lq(d.l), km = rb_km(d.k);
    return (double)d.k * d.m * lq * 2.0 + (double)d.n * (lq * km + km * km + (double)d.l * d.k + (double)d.k * d.k) +
           (double)d.m * d.k * d.k;
}

// Cluster size of problem i for threshold tau: the smallest power of two (<= 8)
// that brings its sweep work per CTA under tau (tau <= 0: always 1).
int cluster_size(const RbInst& d, double tau) {
    if (tau <= 0) return 1;
    const double w = sweep_work(d);
    int c = 1;
    while (c < RB_MAX_CLUSTER && w / c > tau) c *= 2;
    return c;
}

// Group problems into (cluster size, lq, threads) classes, largest work first.
void make_classes(RbPlan* p, double tau, int nt_small, std::vector<int>& flat,
                  std::vector<SweepClass>& out) {
    out.clear();
    flat.clear();
    const int sizes[4] = {1, 2, 4, 8};
    const int lqs[3] = {16, 32, 64};
    const int kms[2] = {16, 32};
    std::vector<int> order(p->count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return sweep_work(p->h_inst[a]) > sweep_work(p->h_inst[b]);
    });
    for (int cs : sizes)
        for (int lq : lqs)
            for (int km : kms) {
            SweepClass c{cs, lq, km, lq == 64 ? 256 : nt_small, nullptr, 0};
            const size_t start = flat.size();
            for (int i : order)
                if (cluster_size(p->h_inst[i], tau) == cs && rb_lq(p->h_inst[i].l) == lq &&
                    rb_km(p->h_inst[i].k) == km)
                    flat.push_back(i);
            c.count = (int)(flat.size() - start);
            c.d_list = reinterpret_cast<int*>(start);  // offset until the list is uploaded
            if (c.count) out.push_back(c);
        }
}

// Every launch of the QB steps and the initial factors, in order.  `counters`
// advances through the plan's atomic tile counters (zeroed at the start).
bool enqueue_qb(RbPlan* p, cudaStream_t s, int* kernels) {
    int ci = 0;
    int nk = 0;
    auto ctr = [&]() { return p->d_counters + (ci++); };
    auto qr = [&](int which, int gate) {
        for (int pass = 0; pass < 3; ++pass) {
            const int only = pass == 2;
            if (!rb_launch_gram(s, p->grid, p->d_inst, which ? p->g_n : p->g_m, which ? p->n_gn : p->n_gm, ctr(),
                                which, only, gate))
                return false;
            if (!rb_launch_chol(s, p->d_inst, p->count, which, pass, gate)) return false;
            if (!rb_launch_rows(s, p->grid, p->d_inst, which ? p->t_n : p->t_m, which ? p->n_tn : p->n_tm, ctr(),
                                which ? 2 : 1, only, gate))
                return false;
            nk += 3;
        }
        return true;
    };
    if (cudaMemsetAsync(p->d_counters, 0, sizeof(int) * p->ncounters, s) != cudaSuccess) return false;
    if (!rb_launch_omega(s, p->d_inst, p->count)) return false;
    if (!rb_launch_rows(s, p->grid, p->d_inst, p->t_m, p->n_tm, ctr(), 0, 0, 0)) return false;
    nk += 2;
    if (!qr(0, 0)) return false;
    for (int it = 1; it <= p->maxq; ++it) {
        if (!rb_launch_atx(s, p->grid, p->d_inst, p->t_n, p->n_tn, ctr(), it)) return false;
        if (!qr(1, it)) return false;
        if (!rb_launch_rows(s, p->grid, p->d_inst, p->t_m, p->n_tm, ctr(), 0, 0, it)) return false;
        if (!qr(0, it)) return false;
        nk += 2;
    }
    if (!rb_launch_atx(s, p->grid, p->d_inst, p->t_n, p->n_tn, ctr(), 0)) return false;
    if (!rb_launch_init(s, p->d_inst, p->count)) return false;
    nk += 2;
    if (ci > p->ncounters) return false;
    if (kernels) *kernels = nk;
    return true;
}

// The sweep classes, each on its own stream (forked from and joined to s).
bool enqueue_sweeps(RbPlan* p, cudaStream_t s, const std::vector<SweepClass>& classes, int iters_override) {
    if (classes.size() > p->side.size()) return false;
    if (cudaEventRecord(p->ev[0], s) != cudaSuccess) return false;
    for (size_t c = 0; c < classes.size(); ++c) {
        cudaStream_t ss = p->side[c];
        if (cudaStreamWaitEvent(ss, p->ev[0], 0) != cudaSuccess) return false;
        const SweepClass& k = classes[c];
        if (!rb_launch_sweeps(ss, p->d_inst, k.d_list, k.count, k.csize, k.lq, k.km, k.nt, iters_override))
            return false;
        if (cudaEventRecord(p->ev[1 + c], ss) != cudaSuccess) return false;
        if (cudaStreamWaitEvent(s, p->ev[1 + c], 0) != cudaSuccess) return false;
    }
    return true;
}

void tiles_over(const std::vector<RbInst>& inst, const std::vector<int>& order, bool over_n, int step_gram,
                std::vector<RbTile>& out) {
    for (int i : order) {
        const RbInst& d = inst[i];
        const int N = over_n ? d.n : d.m;
        const int step = step_gram ? RB_GR : d.bm;
        for (int r = 0; r < N; r += step) out.push_back(RbTile{i, r, std::min(N, r + step), 0});
    }
}

rnmf_status build_plan(rnmf_ctx* ctx, RbPlan* p, const rnmf_problem* probs, int count) {
    p->count = count;
    p->h_inst.resize(count);
    size_t bytes = round256(sizeof(RbInst) * count);
    std::vector<size_t> off(count);
    for (int i = 0; i < count; ++i) {
        RbInst& d = p->h_inst[i];
        memset(&d, 0, sizeof d);
        d.m = (int)probs[i].m;
        d.n = (int)probs[i].n;
        d.k = probs[i].k;
        d.l = probs[i].k + probs[i].p;
        d.ldq = (d.l + 3) / 4 * 4;
        d.q = probs[i].q;
        d.iters = probs[i].iters;
        d.bm = rb_tile_rows(d.l);
        p->maxq = std::max(p->maxq, d.q);
        off[i] = bytes;
        const int64_t nch = (std::max(d.m, d.n) + RB_GR - 1) / RB_GR;
        bytes += round256(sizeof(float) * (size_t)d.m * d.ldq) + round256(sizeof(float) * (size_t)d.n * d.ldq) +
                 round256(sizeof(float) * (size_t)d.k * d.m) + round256(sizeof(double) * nch * d.l * d.l) +
                 round256(sizeof(float) * d.l * d.l);
    }
    // tile lists: problems with more work per tile first
    std::vector<int> by_n(count), by_m(count);
    std::iota(by_n.begin(), by_n.end(), 0);
    std::iota(by_m.begin(), by_m.end(), 0);
    std::stable_sort(by_n.begin(), by_n.end(), [&](int a, int b) { return p->h_inst[a].n > p->h_inst[b].n; });
    std::stable_sort(by_m.begin(), by_m.end(), [&](int a, int b) { return p->h_inst[a].m > p->h_inst[b].m; });
    std::vector<RbTile> tm, tn, gm, gn;
    tiles_over(p->h_inst, by_n, false, 0, tm);  // rows of A: cost ~ n
    tiles_over(p->h_inst, by_m, true, 0, tn);   // columns of A: cost ~ m
    tiles_over(p->h_inst, by_m, false, 1, gm);
    tiles_over(p->h_inst, by_m, true, 1, gn);
    p->n_tm = (int)tm.size();
    p->n_tn = (int)tn.size();
    p->n_gm = (int)gm.size();
    p->n_gn = (int)gn.size();
    p->ncounters = 2 + 6 + p->maxq * 14 + 2;
    const size_t o_tm = bytes;
    bytes += round256(sizeof(RbTile) * tm.size());
    const size_t o_tn = bytes;
    bytes += round256(sizeof(RbTile) * tn.size());
    const size_t o_gm = bytes;
    bytes += round256(sizeof(RbTile) * gm.size());
    const size_t o_gn = bytes;
    bytes += round256(sizeof(RbTile) * gn.size());
    const size_t o_ctr = bytes;
    bytes += round256(sizeof(int) * p->ncounters);
    const size_t o_lists = bytes;
    bytes += round256(sizeof(int) * count);
    if (!scratch_fits(ctx, scratch_held(ctx) + bytes))
        return set_err(ctx, RNMF_ENOMEM, "rnmf_batched: workspace exceeds the context's scratch limit");
    if (cudaMalloc(&p->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        p->ws = nullptr;
        return set_err(ctx, RNMF_ENOMEM, "rnmf_batched: workspace allocation failed");
    }
    p->ws_bytes = bytes;
    p->d_inst = reinterpret_cast<RbInst*>(p->ws);
    for (int i = 0; i < count; ++i) {
        RbInst& d = p->h_inst[i];
        char* q = p->ws + off[i];
        const int64_t nch = (std::max(d.m, d.n) + RB_GR - 1) / RB_GR;
        d.Y = reinterpret_cast<float*>(q);
        q += round256(sizeof(float) * (size_t)d.m * d.ldq);
        d.Z = reinterpret_cast<float*>(q);
        q += round256(sizeof(float) * (size_t)d.n * d.ldq);
        d.Wc = reinterpret_cast<float*>(q);
        q += round256(sizeof(float) * (size_t)d.k * d.m);
        d.gpart = reinterpret_cast<double*>(q);
        q += round256(sizeof(double) * nch * d.l * d.l);
        d.Rinv = reinterpret_cast<float*>(q);
    }
    p->t_m = reinterpret_cast<RbTile*>(p->ws + o_tm);
    p->t_n = reinterpret_cast<RbTile*>(p->ws + o_tn);
    p->g_m = reinterpret_cast<RbTile*>(p->ws + o_gm);
    p->g_n = reinterpret_cast<RbTile*>(p->ws + o_gn);
    p->d_counters = reinterpret_cast<int*>(p->ws + o_ctr);
    p->d_lists = reinterpret_cast<int*>(p->ws + o_lists);
    cudaStream_t s = ctx->stream;
    if (cudaMemcpyAsync(p->t_m, tm.data(), sizeof(RbTile) * tm.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(p->t_n, tn.data(), sizeof(RbTile) * tn.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(p->g_m, gm.data(), sizeof(RbTile) * gm.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(p->g_n, gn.data(), sizeof(RbTile) * gn.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return cuda_err(ctx, "rnmf_batched: tile upload");
    if (cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess)
        return cuda_err(ctx, "rnmf_batched: stream");
    p->side.resize(24);
    p->ev.resize(25);
    for (auto& x : p->side)
        if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_err(ctx, "rnmf_batched: stream");
    for (auto& e : p->ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return cuda_err(ctx, "rnmf_batched: event");
    return RNMF_OK;
}

void fill_dynamic(RbPlan* p, const rnmf_problem* probs, const rnmf_opts& o) {
    for (int i = 0; i < p->count; ++i) {
        RbInst& d = p->h_inst[i];
        d.A = probs[i].A;
        d.W = probs[i].W;
        d.H = probs[i].H;
        d.lda = probs[i].lda;
        d.seed = probs[i].seed;
        d.inst = probs[i].instance;
        d.gram_mode = o.gram_mode;
        d.omega_dist = o.omega_dist;
        d.shifted = 0;
        d.status = 0;
    }
}

// Autotuner: candidate sweep configurations (cluster threshold x threads per CTA
// for l <= 32) timed on a few sweeps of this batch after one real QB run.
rnmf_status autotune(rnmf_ctx* ctx, RbPlan* p) {
    cudaStream_t s = ctx->stream;
    // tile-kernel grid: persistent, a multiple of the SM count
    p->grid = ctx->num_sms * 4;
    if (!enqueue_qb(p, s, nullptr)) return cuda_err(ctx, "rnmf_batched: QB (tuning run)");
    double wmax = 0;
    for (const auto& d : p->h_inst) wmax = std::max(wmax, sweep_work(d));
    const double taus[4] = {0.0, wmax / 2, wmax / 4, wmax / 8};
    const int nts[2] = {256, 512};
    const int tlo = ctx->batch_policy >= 0 ? ctx->batch_policy : 0;
    const int thi = ctx->batch_policy >= 0 ? ctx->batch_policy : 3;
    const int nlo = ctx->batch_threads == 512 ? 1 : 0;
    const int nhi = ctx->batch_threads == 256 ? 0 : 1;
    constexpr int TUNE_ITERS = 4;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    int cand = 0;
    std::vector<int> flat;
    std::vector<SweepClass> cls;
    for (int ti = tlo; ti <= thi; ++ti)
        for (int ni = nlo; ni <= nhi; ++ni, ++cand) {
            make_classes(p, taus[ti], nts[ni], flat, cls);
            if (cudaMemcpyAsync(p->d_lists, flat.data(), sizeof(int) * flat.size(), cudaMemcpyHostToDevice, s) !=
                cudaSuccess)
                return cuda_err(ctx, "rnmf_batched: list upload");
            for (auto& c : cls) c.d_list = p->d_lists + reinterpret_cast<size_t>(c.d_list);
            if (!rb_launch_init(s, p->d_inst, p->count)) return cuda_err(ctx, "rnmf_batched: init (tuning run)");
            cudaEventRecord(a, s);
            if (!enqueue_sweeps(p, s, cls, TUNE_ITERS)) return cuda_err(ctx, "rnmf_batched: sweeps (tuning run)");
            cudaEventRecord(b, s);
            if (cudaEventSynchronize(b) != cudaSuccess) return cuda_err(ctx, "rnmf_batched: tuning run");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            p->tune_ms[cand] = ms;
            if (ms < best) {
                best = ms;
                p->tuned_tau = ti;
                p->tuned_nt_small = nts[ni];
            }
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    make_classes(p, taus[p->tuned_tau], p->tuned_nt_small, flat, cls);
    if (cudaMemcpyAsync(p->d_lists, flat.data(), sizeof(int) * flat.size(), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return cuda_err(ctx, "rnmf_batched: list upload");
    for (auto& c : cls) c.d_list = p->d_lists + reinterpret_cast<size_t>(c.d_list);
    p->classes = cls;
    if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_err(ctx, "rnmf_batched: tuning");
    return RNMF_OK;
}

rnmf_status capture(rnmf_ctx* ctx, RbPlan* p) {
    if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return cuda_err(ctx, "rnmf_batched: begin capture");
    int nk = 0;
    const bool ok = enqueue_qb(p, p->cap, &nk) && enqueue_sweeps(p, p->cap, p->classes, -1);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(p->cap, &g);
    if (!ok || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        return cuda_err(ctx, "rnmf_batched: capture");
    }
    p->graph = g;
    if (cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) return cuda_err(ctx, "rnmf_batched: instantiate");
    p->kernels = nk + (int)p->classes.size();
    return RNMF_OK;
}

std::vector<int64_t> signature(const rnmf_problem* probs, int count) {
    std::vector<int64_t> sig;
    sig.reserve((size_t)count * 6 + 1);
    sig.push_back(count);
    for (int i = 0; i < count; ++i) {
        sig.push_back(probs[i].m);
        sig.push_back(probs[i].n);
        sig.push_back(probs[i].k);
        sig.push_back(probs[i].p);
        sig.push_back(probs[i].q);
        sig.push_back(probs[i].iters);
    }
    return sig;
}

}  // namespace

size_t rb_plan_bytes(rnmf_ctx* ctx) {
    const RbPlan* p = reinterpret_cast<const RbPlan*>(ctx->batch_plan);
    return p && p->ws ? p->ws_bytes : 0;
}

void rb_plan_release(rnmf_ctx* ctx) {
    plan_free(reinterpret_cast<RbPlan*>(ctx->batch_plan));
    ctx->batch_plan = nullptr;
}

extern "C" {

rnmf_status rnmf_batched(rnmf_ctx* ctx, const rnmf_problem* probs, int count, const rnmf_opts* opts,
                         int* status_out, rnmf_batch_stats* stats) {
    if (!ctx) return RNMF_EINVAL;
    if (count < 1 || !probs) return set_err(ctx, RNMF_EINVAL, "rnmf_batched: no problems");
    rnmf_opts o;
    rnmf_default_opts(&o);
    if (opts) o = *opts;
    if (o.gram_mode < 0 || o.gram_mode > 1 || o.omega_dist < 0 || o.omega_dist > 1 || o.precision != RNMF_PREC_FP32 ||
        o.alpha_W != 0.f || o.alpha_H != 0.f || o.beta_W != 0.f || o.beta_H != 0.f || o.order != RNMF_ORDER_CYCLIC ||
        o.init != RNMF_INIT_UNIFORM)
        return set_err(ctx, RNMF_EINVAL,
                       "rnmf_batched: unsupported options (FP32 form, gram_mode 0/1, no penalties, cyclic order)");
    for (int i = 0; i < count; ++i) {
        const rnmf_problem& q = probs[i];
        const int64_t l = (int64_t)q.k + q.p;
        char buf[160];
        if (!q.A || !q.W || !q.H || q.k < 1 || q.k > RB_MAX_K || q.p < 0 || l > RB_MAX_L || q.q < 0 ||
            q.iters < 0 || q.m < 1 || q.n < 1 || q.lda < q.n || l > q.m || l > q.n || q.m > (1 << 30) ||
            q.n > (1 << 30)) {
            snprintf(buf, sizeof buf,
                     "rnmf_batched: problem %d invalid (need 1 <= k <= %d, p >= 0, k + p <= min(m, n, %d), "
                     "q >= 0, iters >= 0, lda >= n, non-null pointers)",
                     i, RB_MAX_K, RB_MAX_L);
            return set_err(ctx, RNMF_EINVAL, buf);
        }
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_err(ctx, "cudaSetDevice");
    RbPlan* p = reinterpret_cast<RbPlan*>(ctx->batch_plan);
    const std::vector<int64_t> sig = signature(probs, count);
    int tuned = 0;
    if (!p || p->sig != sig) {
        rb_plan_release(ctx);
        p = new RbPlan();
        p->sig = sig;
        rnmf_status st = build_plan(ctx, p, probs, count);
        if (st == RNMF_OK) {
            fill_dynamic(p, probs, o);
            if (cudaMemcpyAsync(p->d_inst, p->h_inst.data(), sizeof(RbInst) * count, cudaMemcpyHostToDevice,
                                ctx->stream) != cudaSuccess)
                st = cuda_err(ctx, "rnmf_batched: upload");
        }
        if (st == RNMF_OK) st = autotune(ctx, p);
        if (st == RNMF_OK) st = capture(ctx, p);
        if (st != RNMF_OK) {
            plan_free(p);
            return st;
        }
        ctx->batch_plan = p;
        tuned = 1;
    }
    fill_dynamic(p, probs, o);
    if (cudaMemcpyAsync(p->d_inst, p->h_inst.data(), sizeof(RbInst) * count, cudaMemcpyHostToDevice, ctx->stream) !=
        cudaSuccess)
        return cuda_err(ctx, "rnmf_batched: upload");
    cudaEventRecord(ctx->ev1, ctx->stream);
    if (cudaGraphLaunch(p->exec, ctx->stream) != cudaSuccess) return cuda_err(ctx, "rnmf_batched: graph launch");
    cudaEventRecord(ctx->ev2, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_err(ctx, "rnmf_batched: run");
    ctx->launches += p->kernels;
    std::vector<RbInst> back(count);
    if (cudaMemcpy(back.data(), p->d_inst, sizeof(RbInst) * count, cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_err(ctx, "rnmf_batched: status");
    int failed = 0;
    for (int i = 0; i < count; ++i) {
        if (status_out) status_out[i] = back[i].status;
        if (back[i].status != 0) ++failed;
    }
    if (stats) {
        memset(stats, 0, sizeof *stats);
        cudaEventElapsedTime(&stats->ms, ctx->ev1, ctx->ev2);
        stats->tuned = tuned;
        stats->graph_kernels = p->kernels;
        for (const auto& c : p->classes) {
            const int idx = c.csize == 1 ? 0 : c.csize == 2 ? 1 : c.csize == 4 ? 2 : 3;
            stats->cluster_count[idx] += c.count;
        }
        stats->threads_small = p->tuned_nt_small;
        stats->failed = failed;
        for (int c = 0; c < 8; ++c) stats->tune_ms[c] = p->tune_ms[c];
    }
    if (failed) return set_err(ctx, RNMF_ENOTPD, "rnmf_batched: a CholeskyQR factorisation failed (see status_out)");
    return RNMF_OK;
}

rnmf_status rnmf_batched_config(rnmf_ctx* ctx, int max_cluster, int threads_small) {
    if (!ctx) return RNMF_EINVAL;
    int policy;
    switch (max_cluster) {
        case 0: policy = -1; break;
        case 1: policy = 0; break;
        case 2: policy = 1; break;
        case 4: policy = 2; break;
        case 8: policy = 3; break;
        default: return set_err(ctx, RNMF_EINVAL, "rnmf_batched_config: max_cluster must be 0, 1, 2, 4 or 8");
    }
    if (threads_small != 0 && threads_small != 256 && threads_small != 512)
        return set_err(ctx, RNMF_EINVAL, "rnmf_batched_config: threads_small must be 0, 256 or 512");
    ctx->batch_policy = policy;
    ctx->batch_threads = threads_small;
    rb_plan_release(ctx);
    return RNMF_OK;
}

rnmf_status rnmf_batched_rel_err(rnmf_ctx* ctx, const rnmf_problem* probs, int count, double* out) {
    if (!ctx) return RNMF_EINVAL;
    if (count < 1 || !probs || !out) return set_err(ctx, RNMF_EINVAL, "rnmf_batched_rel_err: bad argument");
    size_t need = 0;
    for (int i = 0; i < count; ++i) {
        if (!probs[i].A || !probs[i].W || !probs[i].H || probs[i].m < 1 || probs[i].n < 1 ||
            probs[i].lda < probs[i].n || probs[i].k < 1)
            return set_err(ctx, RNMF_EINVAL, "rnmf_batched_rel_err: bad problem");
        need = std::max(need, relerr_scratch_bytes(ctx, probs[i].m, probs[i].n));
    }
    const size_t sums = arena_round(need);
    if (arena_reserve(ctx, sums + arena_round(16 * (size_t)count)) != RNMF_OK)
        return set_err(ctx, RNMF_ENOMEM, "rnmf_batched_rel_err: scratch allocation failed");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_err(ctx, "cudaSetDevice");
    double* scratch = reinterpret_cast<double*>(arena_take(ctx, need));
    double* out2 = reinterpret_cast<double*>(arena_take(ctx, 16 * (size_t)count));
    for (int i = 0; i < count; ++i) {
        const rnmf_problem& q = probs[i];
        if (!launch_relerr(ctx, q.A, q.lda, q.W, q.k, 1, q.H, q.m, q.n, q.k, out2 + 2 * i, scratch))
            return cuda_err(ctx, "rnmf_batched_rel_err");
    }
    std::vector<double> h(2 * (size_t)count);
    if (cudaMemcpy(h.data(), out2, sizeof(double) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_err(ctx, "rnmf_batched_rel_err: copy");
    for (int i = 0; i < count; ++i) out[i] = h[2 * i + 1] > 0 ? std::sqrt(h[2 * i] / h[2 * i + 1]) : 0.0;
    return RNMF_OK;
}

}  // extern "C"
