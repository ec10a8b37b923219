// Host side of the EPTV library: geometry handles (FP64 ray tables stored in FP32),
// device workspace, the launch sequence of one outer iteration (Sec. 2.2 steps 1-3),
// CUDA-graph capture and the extern "C" entry points declared in eptv.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdarg>
#include <cstring>
#include <string>
#include <vector>

#include "eptv_internal.cuh"
#include "kernels.cuh"

namespace eptv {

static thread_local std::string g_last_error;

static int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int report_error(int code, const char *msg) { return fail(code, "%s", msg); }

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(EPTV_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                              \
    } while (0)

// Device allocation that is released together with its owner.
struct DevMem {
    std::vector<void *> ptrs;
    template <class T>
    int alloc(T **p, size_t count) {
        void *q = nullptr;
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc(&q, count * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(EPTV_ERR_NOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                        cudaGetErrorString(e));
        }
        ptrs.push_back(q);
        *p = static_cast<T *>(q);
        return 0;
    }
    void release() {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int key[12] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
    long long kernels = 0;     // kernel nodes in the captured outer iteration
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        kernels = 0;
        for (int &k : key) k = -1;
    }
};

// Batch over several handles (cached in the first handle).
struct BatchCache {
    std::vector<const void *> members;
    std::vector<int> modes;     // operator mode of each member when the batch was built
    Batch B;
    DevMem mem;
    GraphCache graph;
    void reset() {
        graph.reset();
        mem.release();
        members.clear();
        modes.clear();
        B = Batch{};
    }
};

}  // namespace eptv

using namespace eptv;

struct eptv_geometry {
    eptv_geometry_desc desc;
    std::vector<double> angles;
    int device = 0;
    DevMem mem;
    SliceDev sd{};          // host copy of this slice's descriptor (workspace pointers)
    Batch B;                // single-slice batch
    float *y_int = nullptr; // internal copy of the data
    int *d_map_custom = nullptr;   // [2] TileMap for generic selection
    cudaStream_t cap = nullptr;    // capture stream
    GraphCache graph;
    BatchCache batch;
    double *d_log = nullptr;       // per-iteration log of the last reconstruction
    size_t log_cap = 0;            // doubles allocated
    int log_outer = 0, log_gd = 0; // layout of the last reconstruction's log
    int op_mode = EPTV_OPERATOR_ON_THE_FLY;
    StoredMatrices stored;         // built on the first switch to EPTV_OPERATOR_STORED
    DevMem stored_mem;
};

namespace eptv {

void fill_params(const eptv_params *p, ParamsDev *d) {
    memset(d, 0, sizeof *d);
    d->lambda = p->lambda;
    d->mu = p->mu;
    d->sigma_q = p->sigma_q;
    d->sigma_floor = p->sigma_floor;
    d->eps = p->eps;
    d->t_fixed = p->t_fixed;
    d->armijo_c = p->armijo_c;
    d->armijo_shrink = p->armijo_shrink;
    d->armijo_grow = p->armijo_grow;
    d->t_max = p->t_max;
    d->t_init = p->t_init;
    d->n_outer = p->n_outer;
    d->cgls_iters = p->cgls_iters;
    d->n_gd = p->n_gd;
    d->step_rule = p->step_rule;
    d->max_trials = p->max_trials;
    d->weights_mode = p->weights_mode;
    d->prior_iters = p->prior_iters;
}

int check_params(const eptv_params *p) {
    if (!p) return fail(EPTV_ERR_ARG, "params is NULL");
    if (p->n_outer < 0 || p->cgls_iters < 0 || p->n_gd < 0)
        return fail(EPTV_ERR_ARG, "negative iteration count");
    if (!(p->lambda > 0.0) || !std::isfinite(p->lambda)) return fail(EPTV_ERR_ARG, "lambda must be > 0");
    if (!(p->eps > 0.0) || !std::isfinite(p->eps)) return fail(EPTV_ERR_ARG, "eps must be > 0");
    if (!(p->sigma_q >= 0.0 && p->sigma_q <= 1.0)) return fail(EPTV_ERR_ARG, "sigma_q must be in [0, 1]");
    if (p->step_rule != EPTV_STEP_ARMIJO && p->step_rule != EPTV_STEP_FIXED)
        return fail(EPTV_ERR_ARG, "bad step_rule %d", p->step_rule);
    if (p->step_rule == EPTV_STEP_ARMIJO) {
        if (p->max_trials < 1 || p->max_trials > kMaxTrials)
            return fail(EPTV_ERR_ARG, "max_trials must be in [1, %d]", kMaxTrials);
        if (!(p->armijo_shrink > 0.0 && p->armijo_shrink < 1.0))
            return fail(EPTV_ERR_ARG, "armijo_shrink must be in (0, 1)");
        if (!(p->armijo_grow > 0.0)) return fail(EPTV_ERR_ARG, "armijo_grow must be > 0");
        if (!(p->armijo_c >= 0.0 && p->armijo_c < 1.0)) return fail(EPTV_ERR_ARG, "armijo_c must be in [0, 1)");
    } else if (!std::isfinite(p->t_fixed)) {
        return fail(EPTV_ERR_ARG, "t_fixed must be finite");
    }
    if (p->weights_mode < 0 || p->weights_mode > 2) return fail(EPTV_ERR_ARG, "bad weights_mode");
    return 0;
}

static double t_init_of(const eptv_params *p) { return p->t_init > 0.0 ? p->t_init : 1.0 / p->lambda; }

// Blocks per slice of every kernel family.
static void family_blocks(const SliceDev &s, int out[FAM_COUNT]) {
    out[FAM_K1] = s.nv * ((s.nb + 31) / 32);
    out[FAM_K2] = ((s.nx + kTileW - 1) / kTileW) * ((s.ny + kTileH - 1) / kTileH);
    out[FAM_IMG] = ((s.nx + 31) / 32) * ((s.ny + 31) / 32);
    out[FAM_SINO] = (s.n_rays + 1023) / 1024;
    out[FAM_EDGE] = (s.n_edges + 2047) / 2048;
    out[FAM_TV] = ((s.nx + kTileW - 1) / kTileW) * ((s.ny + kGdTileRows - 1) / kGdTileRows);
    out[FAM_SPMV_P] = (s.n_rays + 31) / 32;
    out[FAM_SPMV_PT] = ((s.ny + 7) / 8) * ((s.nx + 31) / 32);
}

// Allocate the batch bookkeeping (maps, counters, partials, histograms, params) for the
// given slice descriptors and upload them.
static int build_batch(Batch &B, DevMem &mem, const std::vector<SliceDev> &sds) {
    B.n = (int)sds.size();
    B.h_sd = sds;
    B.h_start.assign((size_t)FAM_COUNT * (B.n + 1), 0);
    int maxblk = 0;
    for (int f = 0; f < FAM_COUNT; ++f) {
        int acc = 0;
        for (int i = 0; i < B.n; ++i) {
            int fb[FAM_COUNT];
            family_blocks(sds[i], fb);
            B.h_start[f * (B.n + 1) + i] = acc;
            acc += fb[f];
        }
        B.h_start[f * (B.n + 1) + B.n] = acc;
        maxblk = std::max(maxblk, acc);
    }
    // reduction bookkeeping per slice: one ticket counter and kPartialStride exact
    // accumulators (zero between launches)
    const int cstride = 1;
    const size_t astride = (size_t)kPartialStride * kAccCopies * kAccStride;
    int rc;
    if ((rc = mem.alloc(&B.d_sd, B.n))) return rc;
    if ((rc = mem.alloc(&B.d_start, B.h_start.size()))) return rc;
    if ((rc = mem.alloc(&B.d_counters, (size_t)B.n * cstride))) return rc;
    if ((rc = mem.alloc(&B.d_acc, (size_t)B.n * astride))) return rc;
    if ((rc = mem.alloc(&B.d_partials, (size_t)maxblk * kPartialStride))) return rc;
    for (int i = 0; i < B.n; ++i) {
        B.h_sd[i].ctr = B.d_counters + (size_t)i * cstride;
        B.h_sd[i].acc = B.d_acc + (size_t)i * astride;
    }
    if ((rc = mem.alloc(&B.d_hist, (size_t)B.n * kHistBins))) return rc;
    if ((rc = mem.alloc(&B.d_params, 1))) return rc;
    const size_t p2words = (size_t)kP2Sets * kP2SetWords;
    if ((rc = mem.alloc(&B.d_p2start, (size_t)B.n + 1))) return rc;
    if ((rc = mem.alloc(&B.d_p2bar, 2))) return rc;
    if ((rc = mem.alloc(&B.d_p2acc, (size_t)B.n * p2words))) return rc;
    if ((rc = mem.alloc(&B.d_p2hist, (size_t)B.n * kP2HistWords))) return rc;
    for (int i = 0; i < B.n; ++i) {
        B.h_sd[i].p2bar = B.d_p2bar;
        B.h_sd[i].p2acc = B.d_p2acc + (size_t)i * p2words;
        B.h_sd[i].p2hist = B.d_p2hist + (size_t)i * kP2HistWords;
    }
    CU(cudaMemcpy(B.d_sd, B.h_sd.data(), sizeof(SliceDev) * B.n, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(B.d_start, B.h_start.data(), sizeof(int) * B.h_start.size(), cudaMemcpyHostToDevice));
    CU(cudaMemset(B.d_counters, 0, sizeof(unsigned int) * (size_t)B.n * cstride));
    CU(cudaMemset(B.d_acc, 0, sizeof(unsigned long long) * (size_t)B.n * astride));
    CU(cudaMemset(B.d_hist, 0, sizeof(unsigned int) * (size_t)B.n * kHistBins));
    CU(cudaMemset(B.d_p2bar, 0, 2 * sizeof(unsigned int)));
    CU(cudaMemset(B.d_p2acc, 0, sizeof(unsigned long long) * (size_t)B.n * p2words));
    CU(cudaMemset(B.d_p2hist, 0, sizeof(unsigned int) * (size_t)B.n * kP2HistWords));
    return 0;
}

// The persistent (P2) kernel's barrier words and sigma histograms to zero, at the start of
// a call: after a bounded wait ran out in an earlier call they are not consistent.
static int reset_p2(const Batch &B, cudaStream_t st) {
    CU(cudaMemsetAsync(B.d_p2bar, 0, 2 * sizeof(unsigned int), st));
    CU(cudaMemsetAsync(B.d_p2hist, 0, sizeof(unsigned int) * (size_t)B.n * kP2HistWords, st));
    return 0;
}

static int upload_sd(Batch &B, cudaStream_t st) {
    CU(cudaMemcpyAsync(B.d_sd, B.h_sd.data(), sizeof(SliceDev) * B.n, cudaMemcpyHostToDevice, st));
    return 0;
}

static int upload_params(const Batch &B, const eptv_params *p, cudaStream_t st) {
    ParamsDev pd;
    fill_params(p, &pd);
    CU(cudaMemcpyAsync(B.d_params, &pd, sizeof pd, cudaMemcpyHostToDevice, st));
    return 0;
}

static int n_trials_of(const eptv_params *p) {
    return p->step_rule == EPTV_STEP_FIXED ? 1 : p->max_trials;
}

// ---------------------------------------------------------------- launch sequences

// P and P^T of a batch: the on-the-fly kernels (K1, K2) or the stored matrices.
static void op_project(const Batch &B, const ProjArgs &a, cudaStream_t st) {
    if (B.stored) launch_spmv_p(B, a, st);
    else launch_project(B, a, st);
}
static void op_backproject(const Batch &B, const BackArgs &a, cudaStream_t st) {
    if (B.stored || B.stored_pt) launch_spmv_pt(B, a, st);
    else launch_backproject(B, a, st);
}

// (P1): M CGLS iterations from u (App. I).  r = y - P u; s = P^T r; then M times
// q = P s, a; r -= a q; [t = P^T r, b; s = t + b s]; u += a s.  defer_last: the last
// u += a s is left to the caller (the persistent (P2) kernel applies it as it loads v).
static void enqueue_cgls(const Batch &B, int M, bool have_uT, cudaStream_t st, bool defer_last = false) {
    ProjArgs pr{};
    pr.img = IMG_U; pr.out = SINO_R; pr.resid = 1; pr.fin = FIN_NONE; pr.no_T = have_uT ? 0 : 1;
    op_project(B, pr, st);
    BackArgs bs{};
    bs.out = 0; bs.write_T = 1; bs.fin = FIN_GAMMA0;
    op_backproject(B, bs, st);
    for (int m = 0; m < M; ++m) {
        ProjArgs pq{};
        pq.img = IMG_S; pq.out = SINO_Q; pq.resid = 0; pq.fin = FIN_QQ_TO_A;
        op_project(B, pq, st);
        const bool more = (m + 1 < M);
        if (more) {
            launch_cgls_update_r(B, st);
            BackArgs bt{};
            bt.out = 1; bt.write_T = 0; bt.fin = FIN_B;
            op_backproject(B, bt, st);
        }
        if (more || !defer_last) launch_cgls_update_us(B, more ? 1 : 0, st);
    }
}

// Chooses the persistent (P2) kernel's launch plan for batch B and parameters p (outside
// any stream capture: it may upload the region map).  B.p2.ok == 0 selects the
// per-iteration K4 launches.
static int ensure_p2(Batch &B, const eptv_params *p, cudaStream_t st) {
    P2Plan plan;
    p2_plan(B, n_trials_of(p), p->n_gd, &plan);
    if (plan.ok && (plan.rtx != B.p2_rtx || plan.rty != B.p2_rty)) {
        p2_region_starts(B, plan.rtx, plan.rty, B.h_p2start);
        CU(cudaMemcpyAsync(B.d_p2start, B.h_p2start.data(), sizeof(int) * B.h_p2start.size(),
                           cudaMemcpyHostToDevice, st));
        CU(cudaStreamSynchronize(st));
        B.p2_rtx = plan.rtx;
        B.p2_rty = plan.rty;
    }
    B.p2 = plan;
    return 0;
}

// (P2) + clamp on v = u: either the persistent kernel K4p (sigma, all n_gd GD iterations,
// apply + clamp into u, u^T) or sigma (K5) and n_gd fused GD launches of K4 and K4u.
static bool p2_persistent(const Batch &B, const eptv_params *p) { return B.p2.ok && p->n_gd >= 1; }

// fold: the CGLS's last u += a s is still to be applied (only with the persistent kernel)
static void enqueue_p2(const Batch &B, const eptv_params *p, const float *v_override,
                       float *out_override, cudaStream_t st, bool fold = false) {
    if (p2_persistent(B, p)) {
        P2Args pa{};
        pa.v = v_override;
        pa.out = out_override;
        pa.n_gd = p->n_gd;
        pa.n_trials = n_trials_of(p);
        pa.bar_extra = B.p2_bar_extra;
        pa.wait_cycles = B.p2_wait_cycles;
        pa.fold = fold ? 1 : 0;
        launch_p2(B, B.p2, pa, st);   // a failure surfaces in the caller's launch check / capture
        return;
    }
    launch_sigma(B, v_override, st);
    for (int n = 0; n < p->n_gd; ++n) {
        GdArgs ga{};
        ga.first = (n == 0);
        ga.last = (n == p->n_gd - 1);
        ga.n_trials = n_trials_of(p);
        ga.v = v_override;
        ga.write_f = 1;
        launch_gd_iter(B, ga, n, st);
    }
    launch_gd_finish(B, p->n_gd, v_override, out_override, st);
}

static void enqueue_outer(const Batch &B, const eptv_params *p, cudaStream_t st) {
    const bool fold = p->cgls_iters > 0 && p2_persistent(B, p);
    enqueue_cgls(B, p->cgls_iters, true, st, fold);
    enqueue_p2(B, p, nullptr, nullptr, st, fold);
}

// Capture one outer iteration of batch B into a graph (cached per structural key).
static int outer_graph(const Batch &B, GraphCache &gc, cudaStream_t cap, const eptv_params *p) {
    const int key[12] = {p->cgls_iters, p->n_gd, n_trials_of(p), p->step_rule, B.n, B.k1_seg, B.k2_vg,
                         B.stored, B.bp_eq11, B.stored_pt, B.p2.ok, B.p2.rtx * 16 + B.p2.rty};
    if (gc.exec && memcmp(key, gc.key, sizeof key) == 0) return 0;
    gc.reset();
    cudaGraph_t graph = nullptr;
    CU(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    const long long c0 = g_launch_count;
    enqueue_outer(B, p, cap);
    const long long captured = g_launch_count - c0;
    g_launch_count = c0;      // captured launches run only when the graph is replayed
    cudaError_t le = cudaGetLastError();
    cudaError_t ee = cudaStreamEndCapture(cap, &graph);
    if (le != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(EPTV_ERR_CUDA, "graph capture failed: %s / %s", cudaGetErrorString(le),
                    cudaGetErrorString(ee));
    }
    cudaError_t ie = cudaGraphInstantiate(&gc.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        gc.exec = nullptr;
        return fail(EPTV_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(ie));
    }
    memcpy(gc.key, key, sizeof key);
    gc.kernels = captured;
    return 0;
}

static int launch_check() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(EPTV_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    return 0;
}

static int read_scalars(const SliceDev &sd, double *out, cudaStream_t st) {
    CU(cudaMemcpyAsync(out, sd.sc, sizeof(double) * kScalarStride, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return 0;
}

// ---------------------------------------------------------------- geometry handle

static int check_desc(const eptv_geometry_desc *d) {
    if (!d) return fail(EPTV_ERR_ARG, "desc is NULL");
    if (d->nx < 1 || d->ny < 1 || d->nx > 8192 || d->ny > 8192)
        return fail(EPTV_ERR_ARG, "image size %dx%d outside 1..8192", d->nx, d->ny);
    if (!(d->dx > 0) || !(d->dy > 0) || !std::isfinite(d->dx) || !std::isfinite(d->dy))
        return fail(EPTV_ERR_ARG, "pixel pitch must be > 0");
    if (d->n_views < 1 || d->n_bins < 1 || (long long)d->n_views * d->n_bins > (1LL << 28))
        return fail(EPTV_ERR_ARG, "bad view/bin count %d x %d", d->n_views, d->n_bins);
    if (!(d->dbeta > 0) || !std::isfinite(d->dbeta)) return fail(EPTV_ERR_ARG, "dbeta must be > 0");
    if (!std::isfinite(d->bin_offset)) return fail(EPTV_ERR_ARG, "bin_offset must be finite");
    if (d->detector != EPTV_DETECTOR_ARC && d->detector != EPTV_DETECTOR_FLAT)
        return fail(EPTV_ERR_ARG, "bad detector %d", d->detector);
    const double half_diag = 0.5 * std::hypot(d->nx * d->dx, d->ny * d->dy);
    if (!(d->sid > half_diag * 1.0001)) return fail(EPTV_ERR_ARG, "source inside the image circle (sid %g <= %g)", d->sid, half_diag);
    if (!(d->sdd > d->sid)) return fail(EPTV_ERR_ARG, "sdd must exceed sid");
    const double kmax = std::max(std::fabs(-(d->n_bins - 1) / 2.0 + d->bin_offset),
                                 std::fabs((d->n_bins - 1) / 2.0 + d->bin_offset));
    if (d->detector == EPTV_DETECTOR_ARC && kmax * d->dbeta >= 1.5)
        return fail(EPTV_ERR_ARG, "fan wider than +-1.5 rad");
    if (d->angles)
        for (int v = 0; v < d->n_views; ++v)
            if (!std::isfinite(d->angles[v])) return fail(EPTV_ERR_ARG, "angle %d not finite", v);
    return 0;
}

static float inv_or_big(double c) {
    if (std::fabs(c) < 1e-30) return c < 0 ? -1e30f : 1e30f;
    return (float)(1.0 / c);
}

}  // namespace eptv

// The batch over `geoms` cached in geoms[0] (built on first use or when the member list
// changes).  The caller has synchronised the stream that used the previous batch.
static int acquire_batch(int n, eptv_geometry *const *geoms, BatchCache &bc) {
    std::vector<const void *> members(geoms, geoms + n);
    std::vector<int> modes;
    for (int i = 0; i < n; ++i) modes.push_back(geoms[i]->op_mode);
    for (int i = 1; i < n; ++i)
        if (modes[i] != modes[0]) return fail(EPTV_ERR_ARG, "batch members use different operators");
    if (bc.members == members && bc.modes == modes) return 0;
    // the same members in another operator mode keep the launch shapes tuned for them
    const bool same = bc.members == members;
    const int k1 = bc.B.k1_seg, k2 = bc.B.k2_vg;
    bc.reset();
    std::vector<SliceDev> sds;
    for (int i = 0; i < n; ++i) sds.push_back(geoms[i]->sd);
    // a batch gives the projector many waves of blocks, which balance by themselves: keep
    // each slice's natural unit order (adjacent bins of a view run together)
    if (n > 1)
        for (SliceDev &sd : sds) sd.k1_order = nullptr;
    int rc = build_batch(bc.B, bc.mem, sds);
    if (rc) { bc.reset(); return rc; }
    bc.B.stored = modes[0] == EPTV_OPERATOR_STORED;
    bc.B.stored_pt = modes[0] == EPTV_OPERATOR_STORED_PT;
    bc.B.bp_eq11 = modes[0] == EPTV_OPERATOR_EQ11;
    if (same) {
        bc.B.k1_seg = k1;
        bc.B.k2_vg = k2;
    }
    bc.members = members;
    bc.modes = modes;
    return 0;
}

// Times every projector / back-projector launch shape on batch B (zero images, the
// batch's own buffers) and keeps the fastest: the ray-block shape of K1 (warps per 32
// rays: 4, 8, 16) and the view split of K2 (1, 2, 4, 8, 16 groups per pixel block).
static int autotune_batch(Batch &B, int *k1_out, int *k2_out) {
    cudaStream_t st = nullptr;
    for (const SliceDev &sd : B.h_sd) {
        CU(cudaMemsetAsync(sd.u, 0, sizeof(float) * sd.n_pix, st));
        CU(cudaMemsetAsync(sd.uT, 0, sizeof(float) * sd.n_pix, st));
        CU(cudaMemsetAsync(sd.r, 0, sizeof(float) * sd.n_rays, st));
    }
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    // One window of 20 back-to-back launches (CUDA events on the launching stream).
    auto window = [&](auto launch) -> float {
        cudaEventRecord(e0, st);
        for (int i = 0; i < 20; ++i) launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    // Each candidate is warmed up, then the candidates are timed in interleaved rounds
    // (so that a drift of clocks or of the other work on the GPU falls on all of them
    // alike) and ranked by their median window.
    auto pick = [&](const int *cand, int n, auto set, auto launch) -> int {
        constexpr int kRounds = 7;
        std::vector<float> t((size_t)n * kRounds);
        for (int c = 0; c < n; ++c) {
            set(cand[c]);
            for (int i = 0; i < 3; ++i) launch();
        }
        for (int r = 0; r < kRounds; ++r)
            for (int c = 0; c < n; ++c) {
                set(cand[c]);
                t[(size_t)c * kRounds + r] = window(launch);
            }
        int best = 0;
        float best_med = 3e38f;
        for (int c = 0; c < n; ++c) {
            float *w = t.data() + (size_t)c * kRounds;
            std::nth_element(w, w + kRounds / 2, w + kRounds);
            if (w[kRounds / 2] < best_med) { best_med = w[kRounds / 2]; best = c; }
        }
        return cand[best];
    };
    const long long saved = g_launch_count;
    ProjArgs pa{};
    pa.img = IMG_U; pa.out = SINO_Q; pa.fin = FIN_NONE;
    BackArgs ba{};
    ba.out = 1; ba.fin = FIN_NONE;
    const int k1c[] = {4, 8, 16}, k2c[] = {1, 2, 4, 8, 16};
    const int b1 = pick(k1c, 3, [&](int c) { B.k1_seg = c; }, [&] { launch_project(B, pa, st); });
    B.k1_seg = b1;
    const int b2 = pick(k2c, 5, [&](int c) { B.k2_vg = c; }, [&] { launch_backproject(B, ba, st); });
    B.k2_vg = b2;
    g_launch_count = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CU(cudaGetLastError());
    CU(cudaDeviceSynchronize());
    if (k1_out) *k1_out = b1;
    if (k2_out) *k2_out = b2;
    return 0;
}

extern "C" {

void eptv_default_params(eptv_params *p) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->n_outer = 50;
    p->cgls_iters = 3;
    p->n_gd = 10;
    p->lambda = 2000.0;
    p->mu = 1.0;
    p->sigma_q = 0.9;
    p->sigma_floor = 1e-12;
    p->eps = 1e-5;
    p->step_rule = EPTV_STEP_ARMIJO;
    p->t_fixed = 1e-4;
    p->armijo_c = 1e-4;
    p->armijo_shrink = 0.5;
    p->armijo_grow = 2.0;
    p->max_trials = 4;
    p->t_max = 0.0;
    p->t_init = 0.0;
    p->weights_mode = EPTV_WEIGHTS_EPTV;
    p->prior_iters = 0;
}

const char *eptv_last_error(void) { return g_last_error.c_str(); }

const char *eptv_version(void) { return "eptv-b300 0.1 (sm_103a)"; }

int eptv_create_geometry(const eptv_geometry_desc *desc, eptv_geometry **out) {
    if (!out) return fail(EPTV_ERR_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_desc(desc);
    if (rc) return rc;
    eptv_geometry *g = new eptv_geometry();
    g->desc = *desc;
    if (desc->angles) {
        g->angles.assign(desc->angles, desc->angles + desc->n_views);
        g->desc.angles = g->angles.data();
    }
    cudaGetDevice(&g->device);
    const int nx = desc->nx, ny = desc->ny, nv = desc->n_views, nb = desc->n_bins;
    const long long n_pix = (long long)nx * ny, n_rays = (long long)nv * nb;
    const long long n_edges = (long long)(nx + 1) * ny + (long long)nx * (ny + 1);

    // ray and view tables in FP64, stored FP32; per ray the rows (or columns) the
    // projector marches, for the order of its work units
    std::vector<RayRec> rays((size_t)n_rays);
    std::vector<ViewRec> views((size_t)nv);
    std::vector<double> march((size_t)n_rays, 0.0);
    const double hx = 0.5 * nx * desc->dx, hy = 0.5 * ny * desc->dy;
    for (int v = 0; v < nv; ++v) {
        const double th = desc->angles ? desc->angles[v] : 2.0 * M_PI * v / nv;
        const double c = std::cos(th), s = std::sin(th);
        const double Sx = desc->sid * c, Sy = desc->sid * s;
        const double cx = -c, cy = -s;
        views[v] = ViewRec{(float)Sx, (float)Sy, (float)cx, (float)cy};
        for (int k = 0; k < nb; ++k) {
            const double kk = k - (nb - 1) / 2.0 + desc->bin_offset;
            const double beta = desc->detector == EPTV_DETECTOR_ARC ? kk * desc->dbeta
                                                                   : std::atan(kk * desc->dbeta);
            const double cb = std::cos(beta), sb = std::sin(beta);
            const double dx = cx * cb - cy * sb, dy = cx * sb + cy * cb;
            const double proj = Sx * dx + Sy * dy;
            const double Px = Sx - proj * dx, Py = Sy - proj * dy;   // closest point to the isocentre
            rays[(size_t)v * nb + k] = RayRec{(float)Px, (float)Py, inv_or_big(dx), inv_or_big(dy)};
            double t0 = -1e300, t1 = 1e300;          // chord through the image square
            const double P[2] = {Px, Py}, D[2] = {dx, dy}, H[2] = {hx, hy};
            for (int a = 0; a < 2; ++a) {
                if (D[a] == 0.0) { if (std::fabs(P[a]) >= H[a]) t1 = -1e300; continue; }
                const double ta = (-H[a] - P[a]) / D[a], tb = (H[a] - P[a]) / D[a];
                t0 = std::max(t0, std::min(ta, tb));
                t1 = std::min(t1, std::max(ta, tb));
            }
            if (t1 > t0)
                march[(size_t)v * nb + k] = std::max(std::fabs(dx) * (t1 - t0) / desc->dx,
                                                     std::fabs(dy) * (t1 - t0) / desc->dy) + 1.0;
        }
    }
    // projector work units (view, 32 bins): cost = the longest march among its rays
    const int nbb = (nb + 31) / 32;
    std::vector<int> k1_order((size_t)nv * nbb);
    std::vector<double> k1_cost((size_t)nv * nbb, 0.0);
    for (int v = 0; v < nv; ++v)
        for (int k = 0; k < nb; ++k) {
            double &c = k1_cost[(size_t)v * nbb + k / 32];
            c = std::max(c, march[(size_t)v * nb + k]);
        }
    for (size_t i = 0; i < k1_order.size(); ++i) k1_order[i] = (int)i;
    std::stable_sort(k1_order.begin(), k1_order.end(),
                     [&](int a, int b) { return k1_cost[(size_t)a] > k1_cost[(size_t)b]; });

    SliceDev &sd = g->sd;
    memset(&sd, 0, sizeof sd);
    sd.nx = nx; sd.ny = ny; sd.nv = nv; sd.nb = nb;
    sd.dx = (float)desc->dx; sd.dy = (float)desc->dy;
    sd.x0 = (float)(-0.5 * nx * desc->dx); sd.y0 = (float)(-0.5 * ny * desc->dy);
    sd.kc = (float)((nb - 1) / 2.0 - desc->bin_offset);
    sd.inv_dbeta = (float)(1.0 / desc->dbeta);
    sd.detector = desc->detector;
    sd.n_pix = (int)n_pix;
    sd.n_rays = (int)n_rays;
    sd.n_edges = (int)n_edges;
    sd.sel_rank = 1;

    DevMem &m = g->mem;
    RayRec *d_ray = nullptr;
    ViewRec *d_view = nullptr;
    int *d_order = nullptr;
    float *img[9] = {};
    float *sino[2] = {};
    double *sc = nullptr;
    if ((rc = m.alloc(&d_ray, n_rays)) || (rc = m.alloc(&d_view, nv))) goto bad;
    if ((rc = m.alloc(&d_order, k1_order.size()))) goto bad;
    for (int i = 0; i < 9; ++i) if ((rc = m.alloc(&img[i], n_pix))) goto bad;
    for (int i = 0; i < 2; ++i) if ((rc = m.alloc(&sino[i], n_rays))) goto bad;
    if ((rc = m.alloc(&g->y_int, n_rays))) goto bad;
    if ((rc = m.alloc(&sd.tv_scr, n_edges))) goto bad;
    if ((rc = m.alloc(&sc, kScalarStride))) goto bad;
    if ((rc = m.alloc(&g->d_map_custom, 2))) goto bad;
    if (cudaMemcpy(d_ray, rays.data(), sizeof(RayRec) * n_rays, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_view, views.data(), sizeof(ViewRec) * nv, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_order, k1_order.data(), sizeof(int) * k1_order.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(sc, 0, sizeof(double) * kScalarStride) != cudaSuccess) {
        rc = fail(EPTV_ERR_CUDA, "upload of the geometry tables failed: %s", cudaGetErrorString(cudaGetLastError()));
        goto bad;
    }
    sd.ray = d_ray; sd.view = d_view; sd.k1_order = d_order;
    sd.u = img[0]; sd.uT = img[1]; sd.s = img[2]; sd.sT = img[3]; sd.t = img[4];
    sd.fa = img[5]; sd.fb = img[6]; sd.ga = img[7]; sd.gb = img[8];
    sd.r = sino[0]; sd.q = sino[1];
    sd.y = g->y_int;
    sd.sc = sc;
    rc = build_batch(g->B, m, std::vector<SliceDev>{sd});
    if (rc) goto bad;
    if (cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking) != cudaSuccess) {
        rc = fail(EPTV_ERR_CUDA, "cudaStreamCreate failed");
        goto bad;
    }
    *out = g;
    return 0;
bad:
    g->mem.release();
    delete g;
    return rc;
}

void eptv_destroy_geometry(eptv_geometry *g) {
    if (!g) return;
    cudaDeviceSynchronize();
    g->graph.reset();
    g->batch.reset();
    if (g->d_log) cudaFree(g->d_log);
    if (g->cap) cudaStreamDestroy(g->cap);
    g->stored_mem.release();
    g->mem.release();
    delete g;
}

int eptv_project_t(const eptv_geometry *gc, const float *d_f, const float *d_fT, float *d_y,
                   void *stream) {
    if (!gc || !d_f || !d_y) return fail(EPTV_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    ProjArgs a{};
    a.img_override = d_f;
    a.imgT_override = d_fT;
    a.out_override = d_y;
    a.fin = FIN_NONE;
    op_project(gc->B, a, st);
    return launch_check();
}

int eptv_transpose(const eptv_geometry *gc, const float *d_f, float *d_fT, void *stream) {
    if (!gc || !d_f || !d_fT) return fail(EPTV_ERR_ARG, "NULL argument");
    launch_transpose(gc->B, d_f, d_fT, (cudaStream_t)stream);
    return launch_check();
}

int eptv_project(const eptv_geometry *gc, const float *d_f, float *d_y, void *stream) {
    if (!gc || !d_f || !d_y) return fail(EPTV_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    // the transposed copy lives in the handle's scratch image t (not used across calls)
    launch_transpose(gc->B, d_f, gc->sd.t, st);
    int rc = launch_check();
    if (rc) return rc;
    return eptv_project_t(gc, d_f, gc->sd.t, d_y, stream);
}

int eptv_backproject(const eptv_geometry *gc, const float *d_y, float *d_f, void *stream) {
    if (!gc || !d_f || !d_y) return fail(EPTV_ERR_ARG, "NULL argument");
    BackArgs a{};
    a.in_override = d_y;
    a.out_override = d_f;
    a.fin = FIN_NONE;
    op_backproject(gc->B, a, (cudaStream_t)stream);
    return launch_check();
}

int eptv_backproject_eq11(const eptv_geometry *gc, const float *d_y, float *d_f, void *stream) {
    if (!gc || !d_f || !d_y) return fail(EPTV_ERR_ARG, "NULL argument");
    BackArgs a{};
    a.in_override = d_y;
    a.out_override = d_f;
    a.fin = FIN_NONE;
    a.eq11 = 1;
    launch_backproject(gc->B, a, (cudaStream_t)stream);
    return launch_check();
}

int eptv_cgls(const eptv_geometry *gc, int M, const float *d_y, float *d_u, void *stream) {
    if (!gc || !d_y || !d_u) return fail(EPTV_ERR_ARG, "NULL argument");
    if (M < 0) return fail(EPTV_ERR_ARG, "M < 0");
    eptv_geometry *g = const_cast<eptv_geometry *>(gc);
    cudaStream_t st = (cudaStream_t)stream;
    const SliceDev &sd = g->sd;
    CU(cudaMemcpyAsync(g->y_int, d_y, sizeof(float) * sd.n_rays, cudaMemcpyDeviceToDevice, st));
    CU(cudaMemcpyAsync(sd.u, d_u, sizeof(float) * sd.n_pix, cudaMemcpyDeviceToDevice, st));
    enqueue_cgls(g->B, M, false, st);
    int rc = launch_check();
    if (rc) return rc;
    CU(cudaMemcpyAsync(d_u, sd.u, sizeof(float) * sd.n_pix, cudaMemcpyDeviceToDevice, st));
    return 0;
}

int eptv_sigma(const eptv_geometry *gc, const eptv_params *p, const float *d_v, double *h_sigma,
               void *stream) {
    if (!gc || !d_v || !h_sigma) return fail(EPTV_ERR_ARG, "NULL argument");
    int rc = check_params(p);
    if (rc) return rc;
    eptv_geometry *g = const_cast<eptv_geometry *>(gc);
    cudaStream_t st = (cudaStream_t)stream;
    SliceDev &sd = g->B.h_sd[0];
    sd.sel_rank = std::min<long long>(std::max<long long>((long long)std::ceil(p->sigma_q * sd.n_edges), 1), sd.n_edges);
    if ((rc = upload_sd(g->B, st)) || (rc = upload_params(g->B, p, st))) return rc;
    launch_sigma(g->B, d_v, st);
    if ((rc = launch_check())) return rc;
    double sc[kScalarStride];
    if ((rc = read_scalars(sd, sc, st))) return rc;
    if (sc[SC_NONFINITE] != 0.0) return fail(EPTV_ERR_NONFINITE, "non-finite half-edge magnitude");
    *h_sigma = sc[SC_SIGMA];
    return 0;
}

int eptv_tv_gradient(const eptv_geometry *gc, const eptv_params *p, double sigma, const float *d_f,
                     const float *d_v, float *d_g, double *h_energy, void *stream) {
    if (!gc || !d_f || !d_v || !d_g) return fail(EPTV_ERR_ARG, "NULL argument");
    int rc = check_params(p);
    if (rc) return rc;
    if (p->weights_mode == EPTV_WEIGHTS_PRIOR) return fail(EPTV_ERR_ARG, "PRIOR weights not accepted here");
    if (!(sigma > 0.0)) return fail(EPTV_ERR_ARG, "sigma must be > 0");
    eptv_geometry *g = const_cast<eptv_geometry *>(gc);
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = upload_params(g->B, p, st))) return rc;
    launch_set_scalar(g->B, SC_SIGMA, sigma, st);
    GdArgs ga{};
    ga.first = 1;
    ga.fprev = d_f;
    ga.v = d_v;
    ga.gout = d_g;
    ga.fout = g->sd.fa;
    ga.write_f = 0;
    ga.n_trials = 0;
    ga.energy_only_fin = 1;
    launch_gd_iter(g->B, ga, 0, st);
    if ((rc = launch_check())) return rc;
    if (h_energy) {
        double sc[kScalarStride];
        if ((rc = read_scalars(g->sd, sc, st))) return rc;
        *h_energy = sc[SC_E_FIRST];
    }
    return 0;
}

int eptv_tv_step(const eptv_geometry *gc, const eptv_params *p, const float *d_v, float *d_f,
                 double *t_prev_io, float *d_weights_opt, eptv_stats *out_opt, void *stream) {
    if (!gc || !d_v || !d_f) return fail(EPTV_ERR_ARG, "NULL argument");
    int rc = check_params(p);
    if (rc) return rc;
    if (p->weights_mode == EPTV_WEIGHTS_PRIOR) return fail(EPTV_ERR_ARG, "PRIOR weights need eptv_reconstruct");
    eptv_geometry *g = const_cast<eptv_geometry *>(gc);
    cudaStream_t st = (cudaStream_t)stream;
    SliceDev &sd = g->B.h_sd[0];
    sd.sel_rank = std::min<long long>(std::max<long long>((long long)std::ceil(p->sigma_q * sd.n_edges), 1), sd.n_edges);
    sd.wout = d_weights_opt;
    rc = upload_sd(g->B, st);
    sd.wout = nullptr;
    if (rc || (rc = upload_params(g->B, p, st))) return rc;
    launch_set_scalar(g->B, SC_TPREV, t_prev_io ? *t_prev_io : t_init_of(p), st);
    launch_set_scalar(g->B, SC_NFAIL_P2, 0.0, st);
    launch_set_scalar(g->B, SC_NACC_P2, 0.0, st);
    launch_set_scalar(g->B, SC_NONFINITE, 0.0, st);
    launch_set_scalar(g->B, SC_TIMEOUT, 0.0, st);
    if ((rc = ensure_p2(g->B, p, st)) || (rc = reset_p2(g->B, st))) return rc;
    enqueue_p2(g->B, p, d_v, d_f, st);
    if ((rc = launch_check())) return rc;
    if ((rc = upload_sd(g->B, st))) return rc;     // clear the weights pointer for later calls
    if (t_prev_io || out_opt) {
        double sc[kScalarStride];
        if ((rc = read_scalars(sd, sc, st))) return rc;
        if (sc[SC_TIMEOUT] != 0.0) return fail(EPTV_ERR_TIMEOUT, "a bounded device wait of the (P2) kernel ran out");
        if (sc[SC_NONFINITE] != 0.0) return fail(EPTV_ERR_NONFINITE, "non-finite value in the TV step");
        if (t_prev_io) *t_prev_io = sc[SC_TPREV];
        if (out_opt) {
            out_opt->sigma = sc[SC_SIGMA];
            out_opt->energy_first = sc[SC_E_FIRST];
            out_opt->energy_last = sc[SC_E_LAST];
            out_opt->t_prev = sc[SC_TPREV];
            out_opt->n_accepted = (int)sc[SC_NACC_P2];
            out_opt->n_fail = (int)sc[SC_NFAIL_P2];
            out_opt->status = out_opt->n_fail ? EPTV_WARN_LINESEARCH : EPTV_OK;
        }
    }
    return 0;
}

// Shared by the single and batched reconstructions: runs n_outer graph replays over B.
static int run_outer(Batch &B, GraphCache &gc, cudaStream_t cap, const eptv_params *p,
                     cudaStream_t st) {
    int rc;
    if ((rc = upload_sd(B, st)) || (rc = upload_params(B, p, st))) return rc;
    if ((rc = ensure_p2(B, p, st)) || (rc = reset_p2(B, st))) return rc;
    launch_set_scalar(B, SC_TIMEOUT, 0.0, st);
    // f^(0): clamp the start image, build its transpose, reset the per-slice state
    launch_gd_finish(B, 0, nullptr, nullptr, st);
    launch_set_scalar(B, SC_OUTER, 0.0, st);
    launch_set_scalar(B, SC_TPREV, t_init_of(p), st);
    launch_set_scalar(B, SC_NFAIL, 0.0, st);
    launch_set_scalar(B, SC_NONFINITE, 0.0, st);
    if ((rc = launch_check())) return rc;
    if (p->n_outer == 0) return 0;
    if ((rc = outer_graph(B, gc, cap, p))) {
        if (!B.p2.ok) return rc;
        // a cooperative launch this driver does not capture: per-iteration K4 launches
        cudaGetLastError();
        B.p2_disabled = 1;
        B.p2 = P2Plan{};
        gc.reset();
        if ((rc = outer_graph(B, gc, cap, p))) return rc;
    }
    for (int k = 0; k < p->n_outer; ++k) CU(cudaGraphLaunch(gc.exec, st));
    g_launch_count += gc.kernels * p->n_outer;
    return 0;
}

int eptv_reconstruct(const eptv_geometry *gc, const eptv_params *p, const float *d_y, float *d_f,
                     const float *d_wprior_opt, eptv_report *rep_opt, void *stream) {
    if (!gc || !d_y || !d_f) return fail(EPTV_ERR_ARG, "NULL argument");
    int rc = check_params(p);
    if (rc) return rc;
    if (p->weights_mode == EPTV_WEIGHTS_PRIOR && !d_wprior_opt)
        return fail(EPTV_ERR_ARG, "PRIOR weights mode needs d_wprior_opt");
    eptv_geometry *g = const_cast<eptv_geometry *>(gc);
    cudaStream_t st = (cudaStream_t)stream;
    SliceDev &sd = g->B.h_sd[0];
    sd.sel_rank = std::min<long long>(std::max<long long>((long long)std::ceil(p->sigma_q * sd.n_edges), 1), sd.n_edges);
    sd.wprior = (p->weights_mode == EPTV_WEIGHTS_PRIOR) ? d_wprior_opt : nullptr;
    {
        const size_t need = (size_t)p->n_outer * (p->n_gd + 1);
        if (need > g->log_cap) {
            CU(cudaStreamSynchronize(st));
            if (g->d_log) cudaFree(g->d_log);
            g->d_log = nullptr;
            g->log_cap = 0;
            CU(cudaMalloc(&g->d_log, need * sizeof(double)));
            g->log_cap = need;
        }
        g->log_outer = p->n_outer;
        g->log_gd = p->n_gd;
        sd.log = g->d_log;
        sd.log_outer = p->n_outer;
        sd.log_gd = p->n_gd;
        if (need) CU(cudaMemsetAsync(g->d_log, 0, need * sizeof(double), st));
    }
    CU(cudaMemcpyAsync(g->y_int, d_y, sizeof(float) * sd.n_rays, cudaMemcpyDeviceToDevice, st));
    CU(cudaMemcpyAsync(sd.u, d_f, sizeof(float) * sd.n_pix, cudaMemcpyDeviceToDevice, st));
    const long long l0 = g_launch_count;
    if ((rc = run_outer(g->B, g->graph, g->cap, p, st))) return rc;
    const long long nl = g_launch_count - l0;
    CU(cudaMemcpyAsync(d_f, sd.u, sizeof(float) * sd.n_pix, cudaMemcpyDeviceToDevice, st));
    if (rep_opt) {
        rep_opt->n_launches = nl;
        double sc[kScalarStride];
        if ((rc = read_scalars(sd, sc, st))) return rc;
        if (sc[SC_TIMEOUT] != 0.0) return fail(EPTV_ERR_TIMEOUT, "a bounded device wait of the (P2) kernel ran out");
        if (sc[SC_NONFINITE] != 0.0) return fail(EPTV_ERR_NONFINITE, "non-finite value during the reconstruction");
        rep_opt->n_outer = p->n_outer;
        rep_opt->sigma_last = sc[SC_SIGMA];
        rep_opt->t_prev = sc[SC_TPREV];
        rep_opt->n_fail = (int)sc[SC_NFAIL];
        rep_opt->status = rep_opt->n_fail ? EPTV_WARN_LINESEARCH : EPTV_OK;
    }
    return 0;
}

int eptv_report_energy(const eptv_geometry *gc, const eptv_params *p, double sigma_ref,
                       const float *d_f, const float *d_y, double *h_energy, void *stream) {
    if (!gc || !d_f || !d_y || !h_energy) return fail(EPTV_ERR_ARG, "NULL argument");
    int rc = check_params(p);
    if (rc) return rc;
    if (!(sigma_ref > 0.0)) return fail(EPTV_ERR_ARG, "sigma_ref must be > 0");
    eptv_geometry *g = const_cast<eptv_geometry *>(gc);
    cudaStream_t st = (cudaStream_t)stream;
    eptv_params pe = *p;
    if (pe.weights_mode == EPTV_WEIGHTS_PRIOR) pe.weights_mode = EPTV_WEIGHTS_EPTV;
    if ((rc = upload_params(g->B, &pe, st))) return rc;
    launch_set_scalar(g->B, SC_NONFINITE, 0.0, st);
    ProjArgs a{};
    a.img_override = d_f;
    a.imgT_override = nullptr;
    a.out_override = g->sd.q;
    a.y_override = d_y;
    a.resid = 1;
    a.fin = FIN_NORM;
    op_project(g->B, a, st);
    launch_set_scalar(g->B, SC_SIGMA, sigma_ref, st);
    GdArgs ga{};
    ga.first = 1;
    ga.fprev = d_f;
    ga.v = d_f;
    ga.gout = g->sd.ga;
    ga.fout = g->sd.fa;
    ga.write_f = 0;
    ga.n_trials = 0;
    ga.energy_only_fin = 1;
    launch_gd_iter(g->B, ga, 0, st);
    if ((rc = launch_check())) return rc;
    double sc[kScalarStride];
    if ((rc = read_scalars(g->sd, sc, st))) return rc;
    if (sc[SC_NONFINITE] != 0.0) return fail(EPTV_ERR_NONFINITE, "non-finite energy");
    *h_energy = 0.5 * p->mu * sc[SC_NORM] + sc[SC_E_FIRST];
    return 0;
}

int eptv_get_log(const eptv_geometry *gc, double *h_steps, int steps_cap, double *h_sigmas,
                 int sigmas_cap, int *n_outer, int *n_gd) {
    if (!gc) return fail(EPTV_ERR_ARG, "NULL handle");
    if (n_outer) *n_outer = gc->log_outer;
    if (n_gd) *n_gd = gc->log_gd;
    if (!gc->d_log || gc->log_outer == 0) return 0;
    CU(cudaDeviceSynchronize());
    const size_t ns = (size_t)gc->log_outer * gc->log_gd;
    if (h_steps && steps_cap > 0)
        CU(cudaMemcpy(h_steps, gc->d_log, sizeof(double) * std::min<size_t>(ns, (size_t)steps_cap),
                      cudaMemcpyDeviceToHost));
    if (h_sigmas && sigmas_cap > 0)
        CU(cudaMemcpy(h_sigmas, gc->d_log + ns,
                      sizeof(double) * std::min<size_t>((size_t)gc->log_outer, (size_t)sigmas_cap),
                      cudaMemcpyDeviceToHost));
    return 0;
}

int eptv_select_kth(const eptv_geometry *gc, const float *d_vals, long n, long k, float *d_out,
                    void *stream) {
    if (!gc || !d_vals || !d_out) return fail(EPTV_ERR_ARG, "NULL argument");
    if (n < 1 || k < 1 || k > n) return fail(EPTV_ERR_ARG, "need 1 <= k <= n (k=%ld, n=%ld)", k, n);
    if (n > (1L << 40)) return fail(EPTV_ERR_ARG, "n too large");
    eptv_geometry *g = const_cast<eptv_geometry *>(gc);
    cudaStream_t st = (cudaStream_t)stream;
    const long long nblk = (n + 2047) / 2048;
    if (nblk > (1LL << 30)) return fail(EPTV_ERR_ARG, "n too large");
    // a one-slice map over nblk blocks (kept in the handle; stream-ordered upload)
    static thread_local int hmap[2];
    hmap[0] = 0;
    hmap[1] = (int)nblk;
    CU(cudaMemcpyAsync(g->d_map_custom, hmap, sizeof hmap, cudaMemcpyHostToDevice, st));
    TileMap m{g->d_map_custom, 1};
    launch_select_generic(g->B, m, (int)nblk, d_vals, (long long)n, (long long)k, d_out, st);
    return launch_check();
}

int eptv_reconstruct_batched(int n, eptv_geometry *const *geoms, const eptv_params *p,
                             const float *const *d_y, float *const *d_f, eptv_report *reps,
                             void *stream) {
    if (n < 1 || !geoms || !d_y || !d_f) return fail(EPTV_ERR_ARG, "bad batch arguments");
    int rc = check_params(p);
    if (rc) return rc;
    if (p->weights_mode == EPTV_WEIGHTS_PRIOR) return fail(EPTV_ERR_ARG, "PRIOR weights not supported in batches");
    for (int i = 0; i < n; ++i) {
        if (!geoms[i] || !d_y[i] || !d_f[i]) return fail(EPTV_ERR_ARG, "NULL entry %d", i);
        for (int j = 0; j < i; ++j)
            if (geoms[j] == geoms[i]) return fail(EPTV_ERR_ARG, "handle %d repeated in the batch", i);
    }
    cudaStream_t st = (cudaStream_t)stream;
    eptv_geometry *g0 = geoms[0];
    BatchCache &bc = g0->batch;
    cudaStreamSynchronize(st);
    if ((rc = acquire_batch(n, geoms, bc))) return rc;
    bc.B.p2_forbid = g0->B.p2_forbid;
    for (int i = 0; i < n; ++i) {
        SliceDev &sd = bc.B.h_sd[i];
        sd.sel_rank = std::min<long long>(std::max<long long>((long long)std::ceil(p->sigma_q * sd.n_edges), 1), sd.n_edges);
        sd.wprior = nullptr;
        CU(cudaMemcpyAsync(geoms[i]->y_int, d_y[i], sizeof(float) * sd.n_rays, cudaMemcpyDeviceToDevice, st));
        CU(cudaMemcpyAsync(sd.u, d_f[i], sizeof(float) * sd.n_pix, cudaMemcpyDeviceToDevice, st));
    }
    const long long l0 = g_launch_count;
    if ((rc = run_outer(bc.B, bc.graph, g0->cap, p, st))) return rc;
    const long long nl = g_launch_count - l0;
    for (int i = 0; i < n; ++i)
        CU(cudaMemcpyAsync(d_f[i], bc.B.h_sd[i].u, sizeof(float) * bc.B.h_sd[i].n_pix,
                           cudaMemcpyDeviceToDevice, st));
    if (reps) {
        CU(cudaStreamSynchronize(st));
        for (int i = 0; i < n; ++i) {
            double sc[kScalarStride];
            if ((rc = read_scalars(bc.B.h_sd[i], sc, st))) return rc;
            if (sc[SC_TIMEOUT] != 0.0) return fail(EPTV_ERR_TIMEOUT, "a bounded device wait ran out in slice %d", i);
            if (sc[SC_NONFINITE] != 0.0) return fail(EPTV_ERR_NONFINITE, "non-finite value in slice %d", i);
            reps[i].n_outer = p->n_outer;
            reps[i].n_launches = nl;
            reps[i].sigma_last = sc[SC_SIGMA];
            reps[i].t_prev = sc[SC_TPREV];
            reps[i].n_fail = (int)sc[SC_NFAIL];
            reps[i].status = reps[i].n_fail ? EPTV_WARN_LINESEARCH : EPTV_OK;
        }
    }
    return 0;
}

int eptv_set_tv_kernel(eptv_geometry *g, int mode) {
    if (!g) return fail(EPTV_ERR_ARG, "NULL handle");
    if (mode != EPTV_TV_AUTO && mode != EPTV_TV_PER_ITERATION) return fail(EPTV_ERR_ARG, "bad tv kernel mode %d", mode);
    g->B.p2_forbid = mode == EPTV_TV_PER_ITERATION;
    g->batch.B.p2_forbid = g->B.p2_forbid;
    return 0;
}

int eptv_debug_set_p2_wait(eptv_geometry *g, int extra_blocks, long long wait_cycles) {
    if (!g) return fail(EPTV_ERR_ARG, "NULL handle");
    if (extra_blocks < 0 || extra_blocks > 1024 || wait_cycles < 1000 || wait_cycles > 4000000000ll)
        return fail(EPTV_ERR_ARG, "extra_blocks in [0, 1024], wait_cycles in [1e3, 4e9]");
    g->B.p2_bar_extra = extra_blocks;
    g->B.p2_wait_cycles = wait_cycles;
    g->graph.reset();     // the captured launch carries the old values
    return 0;
}

int eptv_set_tuning(eptv_geometry *g, int k1_seg, int k2_vg) {
    if (!g) return fail(EPTV_ERR_ARG, "NULL handle");
    if (k1_seg != 4 && k1_seg != 8 && k1_seg != 16) return fail(EPTV_ERR_ARG, "k1_seg must be 4, 8 or 16");
    if (k2_vg != 1 && k2_vg != 2 && k2_vg != 4 && k2_vg != 8 && k2_vg != 16)
        return fail(EPTV_ERR_ARG, "k2_vg must be 1, 2, 4, 8 or 16");
    g->B.k1_seg = k1_seg;
    g->B.k2_vg = k2_vg;
    return 0;
}

int eptv_autotune(eptv_geometry *g, int *k1_seg, int *k2_vg) {
    if (!g) return fail(EPTV_ERR_ARG, "NULL handle");
    CU(cudaDeviceSynchronize());
    return autotune_batch(g->B, k1_seg, k2_vg);
}

int eptv_autotune_batched(int n, eptv_geometry *const *geoms, int *k1_seg, int *k2_vg) {
    if (n < 1 || !geoms) return fail(EPTV_ERR_ARG, "bad batch arguments");
    for (int i = 0; i < n; ++i)
        if (!geoms[i]) return fail(EPTV_ERR_ARG, "NULL entry %d", i);
    CU(cudaDeviceSynchronize());
    int rc = acquire_batch(n, geoms, geoms[0]->batch);
    if (rc) return rc;
    return autotune_batch(geoms[0]->batch.B, k1_seg, k2_vg);
}


static cudaError_t stored_alloc(void *ctx, void **p, size_t bytes) {
    DevMem *m = static_cast<DevMem *>(ctx);
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return e;
    m->ptrs.push_back(q);
    *p = q;
    return cudaSuccess;
}

int eptv_set_operator(eptv_geometry *g, int mode, long long *h_nnz_opt) {
    if (!g) return fail(EPTV_ERR_ARG, "NULL handle");
    if (mode != EPTV_OPERATOR_ON_THE_FLY && mode != EPTV_OPERATOR_STORED && mode != EPTV_OPERATOR_EQ11 &&
        mode != EPTV_OPERATOR_STORED_PT)
        return fail(EPTV_ERR_ARG, "unknown operator mode %d", mode);
    CU(cudaDeviceSynchronize());
    const bool need = mode == EPTV_OPERATOR_STORED || mode == EPTV_OPERATOR_STORED_PT;
    if (need && !g->stored.p_ptr) {
        StoredMatrices m;
        cudaError_t e = build_stored(g->sd, g->B.d_sd, stored_alloc, &g->stored_mem, &m, nullptr);
        if (e != cudaSuccess) {
            cudaGetLastError();
            g->stored_mem.release();
            if (e == cudaErrorInvalidValue)
                return fail(EPTV_ERR_ARG, "stored matrix too large (a row of P longer than 4096 "
                                          "entries, or 2^31 entries or more)");
            if (e == cudaErrorMemoryAllocation) return fail(EPTV_ERR_NOMEM, "no device memory for the stored matrices");
            return fail(EPTV_ERR_CUDA, "building the stored matrices failed: %s", cudaGetErrorString(e));
        }
        // the leading P^T slices whose entries fit in half of L2 (read evict_last)
        int dev = 0, l2 = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
            l2 = 0;
        cudaGetLastError();
        const int n_sl = ((g->sd.nx + 31) / 32) * g->sd.ny;
        std::vector<int> sptr((size_t)n_sl + 1);
        CU(cudaMemcpy(sptr.data(), m.pt_sptr, sizeof(int) * sptr.size(), cudaMemcpyDeviceToHost));
        const long long keep_entries = (long long)l2 / 2 / 8;            // 8 B per entry
        int keep = 0;
        while (keep < n_sl && sptr[(size_t)keep + 1] <= keep_entries) ++keep;
        m.pt_keep = keep;
        g->stored = m;
    }
    const bool on = mode == EPTV_OPERATOR_STORED;
    for (SliceDev *sd : {&g->sd, &g->B.h_sd[0]}) {
        sd->p_sptr = on ? g->stored.p_sptr : nullptr;
        sd->p_slen = on ? g->stored.p_slen : nullptr;
        sd->p_scol = on ? g->stored.p_scol : nullptr;
        sd->p_sval = on ? g->stored.p_sval : nullptr;
        sd->pt_sptr = need ? g->stored.pt_sptr : nullptr;
        sd->pt_slen = need ? g->stored.pt_slen : nullptr;
        sd->pt_scol = need ? g->stored.pt_scol : nullptr;
        sd->pt_sval = need ? g->stored.pt_sval : nullptr;
        sd->pt_keep = need ? g->stored.pt_keep : 0;
    }
    CU(cudaMemcpy(g->B.d_sd, g->B.h_sd.data(), sizeof(SliceDev), cudaMemcpyHostToDevice));
    g->B.stored = on ? 1 : 0;
    g->B.stored_pt = mode == EPTV_OPERATOR_STORED_PT ? 1 : 0;
    g->B.bp_eq11 = mode == EPTV_OPERATOR_EQ11 ? 1 : 0;
    g->op_mode = mode;
    g->graph.reset();
    if (h_nnz_opt) *h_nnz_opt = g->stored.nnz_p;
    return 0;
}

int eptv_autotune_operator(eptv_geometry *g, long long max_matrix_bytes, int *mode_out) {
    if (!g) return fail(EPTV_ERR_ARG, "NULL handle");
    if (g->op_mode != EPTV_OPERATOR_ON_THE_FLY && g->op_mode != EPTV_OPERATOR_STORED_PT)
        return fail(EPTV_ERR_ARG, "operator autotuning starts from EPTV_OPERATOR_ON_THE_FLY or _STORED_PT");
    int rc = 0;
    const SliceDev &sd = g->sd;
    // about 32 bytes per entry of P (CSR and SELL-32 of P and P^T); a ray has at most
    // nx + ny entries, so this bound is known before anything is built
    const long long bound = 32ll * (long long)sd.n_rays * (long long)(sd.nx + sd.ny);
    int best = EPTV_OPERATOR_ON_THE_FLY;
    if (bound <= max_matrix_bytes) {
        if ((rc = eptv_set_operator(g, EPTV_OPERATOR_STORED_PT, nullptr))) {
            if (rc != EPTV_ERR_NOMEM && rc != EPTV_ERR_ARG) return rc;
            rc = 0;                                  // too large to build: stays on the fly
        } else {
            Batch &B = g->B;
            cudaStream_t st = nullptr;
            CU(cudaMemsetAsync(sd.r, 0, sizeof(float) * sd.n_rays, st));
            cudaEvent_t e0, e1;
            CU(cudaEventCreate(&e0));
            CU(cudaEventCreate(&e1));
            BackArgs ba{};
            ba.out = 1; ba.fin = FIN_NONE;
            const long long saved = g_launch_count;
            // P^T from the kernel (its tuned shape) and from the stored matrix, timed in
            // interleaved rounds of 20 launches and ranked by the median round
            constexpr int kRounds = 7;
            float t[2][kRounds];
            for (int c = 0; c < 2; ++c) {
                B.stored_pt = c;
                for (int i = 0; i < 3; ++i) op_backproject(B, ba, st);
            }
            for (int r = 0; r < kRounds; ++r)
                for (int c = 0; c < 2; ++c) {
                    B.stored_pt = c;
                    cudaEventRecord(e0, st);
                    for (int i = 0; i < 20; ++i) op_backproject(B, ba, st);
                    cudaEventRecord(e1, st);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    t[c][r] = ms;
                }
            g_launch_count = saved;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            CU(cudaGetLastError());
            std::nth_element(t[0], t[0] + kRounds / 2, t[0] + kRounds);
            std::nth_element(t[1], t[1] + kRounds / 2, t[1] + kRounds);
            if (t[1][kRounds / 2] < t[0][kRounds / 2]) best = EPTV_OPERATOR_STORED_PT;
        }
    }
    if ((rc = eptv_set_operator(g, best, nullptr))) return rc;
    if (best == EPTV_OPERATOR_ON_THE_FLY && g->stored.p_ptr) {   // not used: give the memory back
        g->stored_mem.release();
        g->stored = StoredMatrices{};
    }
    if (mode_out) *mode_out = best;
    return 0;
}

int eptv_matrix_info(const eptv_geometry *g, int which, long long *h_rows, long long *h_nnz,
                     long long *h_sell_opt) {
    if (!g || !h_rows || !h_nnz) return fail(EPTV_ERR_ARG, "NULL argument");
    if (which != 0 && which != 1) return fail(EPTV_ERR_ARG, "which must be 0 (P) or 1 (P^T)");
    if (!g->stored.p_ptr) return fail(EPTV_ERR_ARG, "the stored matrices have not been built");
    *h_rows = which == 0 ? g->sd.n_rays : g->sd.n_pix;
    *h_nnz = which == 0 ? g->stored.nnz_p : g->stored.nnz_pt;
    if (h_sell_opt) *h_sell_opt = which == 0 ? g->stored.sell_p : g->stored.sell_pt;
    return 0;
}

int eptv_copy_matrix(const eptv_geometry *g, int which, int *d_ptr, int *d_col, float *d_val, void *stream) {
    long long rows, nnz;
    int rc = eptv_matrix_info(g, which, &rows, &nnz, nullptr);
    if (rc) return rc;
    if (!d_ptr || !d_col || !d_val) return fail(EPTV_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    const StoredMatrices &m = g->stored;
    CU(cudaMemcpyAsync(d_ptr, which == 0 ? m.p_ptr : m.pt_ptr, sizeof(int) * (size_t)(rows + 1),
                       cudaMemcpyDeviceToDevice, st));
    CU(cudaMemcpyAsync(d_col, which == 0 ? m.p_col : m.pt_col, sizeof(int) * (size_t)nnz,
                       cudaMemcpyDeviceToDevice, st));
    CU(cudaMemcpyAsync(d_val, which == 0 ? m.p_val : m.pt_val, sizeof(float) * (size_t)nnz,
                       cudaMemcpyDeviceToDevice, st));
    return 0;
}

int eptv_quality_metrics(const eptv_geometry *g, const float *d_f, const float *d_ref_opt,
                         const int *h_roi_opt, double edge_scale, unsigned char *d_edges_opt,
                         unsigned char *d_edges_ref_opt, eptv_quality *out, void *stream) {
    if (!g || !d_f || !out) return fail(EPTV_ERR_ARG, "NULL argument");
    if (!(edge_scale > 0.0)) return fail(EPTV_ERR_ARG, "edge_scale must be > 0");
    const int nx = g->sd.nx, ny = g->sd.ny;
    int rx0 = 0, ry0 = 0, rw = 0, rh = 0;
    if (h_roi_opt) {
        rx0 = h_roi_opt[0]; ry0 = h_roi_opt[1]; rw = h_roi_opt[2]; rh = h_roi_opt[3];
        if (rw < 1 || rh < 1 || rx0 < 0 || ry0 < 0 || rx0 + rw > nx || ry0 + rh > ny)
            return fail(EPTV_ERR_ARG, "ROI outside the image");
    }
    cudaStream_t st = (cudaStream_t)stream;
    launch_quality(g->B, d_f, d_ref_opt, rx0, ry0, rw, rh, edge_scale * edge_scale, d_edges_opt,
                   d_ref_opt ? d_edges_ref_opt : nullptr, st);
    int rc = launch_check();
    if (rc) return rc;
    double sc[kScalarStride];
    if ((rc = read_scalars(g->sd, sc, st))) return rc;
    const double nan = std::nan("");
    const double N = (double)nx * ny;
    const double nb = sc[SC_Q0 + 6], nr = sc[SC_Q0 + 7], both = sc[SC_Q0 + 8];
    out->edges = (long long)nb;
    out->edges_ref = d_ref_opt ? (long long)nr : 0;
    out->edges_both = d_ref_opt ? (long long)both : 0;
    out->rel_error = d_ref_opt ? sc[SC_Q0] / sc[SC_Q0 + 1] : nan;
    const double vb = nb - nb * nb / N, vr = nr - nr * nr / N;
    out->ecc = (d_ref_opt && vb > 0.0 && vr > 0.0) ? (both - nb * nr / N) / std::sqrt(vb * vr) : nan;
    if (h_roi_opt) {
        const double n = (double)rw * rh;
        const double m = sc[SC_Q0 + 4] / n;
        const double var = sc[SC_Q0 + 5] / n - m * m;
        out->snr_db = 10.0 * std::log10(m * m / var);
    } else {
        out->snr_db = nan;
    }
    return 0;
}

}  // extern "C"
