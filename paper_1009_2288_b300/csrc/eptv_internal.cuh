// Internal definitions of the sm_103a EPTV library: per-slice descriptors, launch plans,
// the canonical plane-crossing arithmetic shared by the projector (K1) and its exact
// adjoint (K2), and block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "eptv.h"

namespace eptv {

// ---------------------------------------------------------------------------------
// Canonical crossing parameter of a grid line.
//
// The system-matrix element p_ij (Eq. 1) is the length of ray i inside pixel j.  With
// a ray r(t) = P + t d (|d| = 1, P the point of the line closest to the isocentre) and
// the grid line coordinate X_k = origin + k * pitch, the line is crossed at
//     t_k = (X_k - P) * (1 / d).
// Pixel (i, j) is the intersection of column slab [X_i, X_{i+1}] and row slab
// [Y_j, Y_{j+1}], so  p_ij = max(0, min(tx_hi, ty_hi) - max(tx_lo, ty_lo)).
// The projector and the back projector evaluate every t_k with exactly this sequence
// of correctly rounded single-precision operations (no contraction), so both see
// bit-identical p_ij and P^T is the exact transpose of P up to summation order.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float grid_line(float k, float pitch, float origin) {
    return __fmaf_rn(k, pitch, origin);
}
__device__ __forceinline__ float cross_t(float X, float p, float inv) {
    return __fmul_rn(__fsub_rn(X, p), inv);
}
__device__ __forceinline__ float seg_len(float lo_a, float hi_a, float lo_b, float hi_b) {
    return fmaxf(0.0f, __fsub_rn(fminf(hi_a, hi_b), fmaxf(lo_a, lo_b)));
}

// Ray record, FP32, built on the host in FP64: {P_x, P_y, 1/d_x, 1/d_y}.  The direction
// is oriented so that its major component is positive (the major axis is y when the
// ray crosses rows faster than columns: |d_y|/dy >= |d_x|/dx).  A zero component is
// stored with 1/d = +-1e30 so that no NaN can arise.
struct RayRec { float px, py, ix, iy; };

// Per-view record for the pixel-driven adjoint: source S and central direction c (FP32).
struct ViewRec { float sx, sy, cx, cy; };

// Scalars kept per slice in device memory (FP64).
enum Scalar {
    SC_GAMMA = 0,    // |P^T r|^2 of the current CGLS iterate
    SC_QQ,           // |P s|^2
    SC_A,            // CGLS step a
    SC_B,            // CGLS step b
    SC_SIGMA,        // sigma of the current (P2) solve
    SC_TPREV,        // previous accepted Armijo step
    SC_TSTEP,        // step taken by the last GD iteration (applied by the next kernel)
    SC_E_FIRST,      // (P2) energy at the first GD iterate
    SC_E_LAST,       // (P2) energy after the last step (frozen weights)
    SC_NORM,         // generic reduction result (energy / norm queries)
    SC_NORM2,        // second generic reduction result
    SC_NFAIL,        // number of failed line searches (as double)
    SC_NFAIL_P2,     // failures within the current (P2) solve
    SC_NACC_P2,      // accepted steps within the current (P2) solve
    SC_OUTER,        // outer iteration counter
    SC_NONFINITE,    // set to 1 when a reduction met NaN / Inf
    SC_SEL_PREFIX,   // radix select: fixed bit prefix (as double, exact below 2^53)
    SC_SEL_RANK,     // radix select: remaining 1-based rank within the prefix
    SC_Q0,           // image-quality sums (quality.cu): SC_Q0 .. SC_Q0 + 8
    SC_COUNT = SC_Q0 + 9
};
constexpr int kScalarStride = 32;   // doubles per slice (>= SC_COUNT)

// Parameters as seen by the kernels (copied once per call).
struct ParamsDev {
    double lambda, mu, sigma_q, sigma_floor, eps;
    double t_fixed, armijo_c, armijo_shrink, armijo_grow, t_max, t_init;
    int n_outer, cgls_iters, n_gd, step_rule, max_trials, weights_mode, prior_iters;
    int pad;
};

// Device descriptor of one slice: geometry and the buffers the kernels work on.
struct SliceDev {
    int nx, ny, nv, nb;
    float dx, dy, x0, y0;
    float kc;            // fractional-bin offset: u = beta / dbeta + kc
    float inv_dbeta;
    int detector;
    int n_pix, n_rays;
    long long sel_rank;  // 1-based rank of sigma among the half-edges
    int n_edges;         // (nx+1) ny + nx (ny+1)
    const RayRec *ray;   // [nv * nb]
    const ViewRec *view; // [nv]
    // solver state (device workspace of the handle, or caller buffers)
    const float *y;      // data sinogram
    float *u, *uT;       // current image / CGLS iterate and its transpose
    float *s, *sT, *t;   // CGLS image vectors
    float *r, *q;        // CGLS sinogram vectors
    float *fa, *fb;      // (P2) iterate ping-pong
    float *ga, *gb;      // (P2) gradient ping-pong
    float *tv_scr;       // [n_edges] FP32 scratch (half-edge magnitudes for sigma)
    const float *wprior; // per-pixel prior weight map, or null
    float *wout;         // optional output of the final edge weights
    double *sc;          // [kScalarStride] scalars
    double *log;         // optional per-iteration log: [n_outer * n_gd] steps, then [n_outer] sigmas
    int log_outer;       // capacity in outer iterations (0: no log)
    int log_gd;          // GD iterations per outer iteration in the log layout
    // reduction bookkeeping of this slice in its batch: ticket counters ([0] final level,
    // [1 + g] group g) and the group partial sums ([group][kPartialStride] doubles)
    unsigned int *ctr;
    double *gpart;
    // stored operator (null unless selected): SELL-32 P (rows = rays), P^T (rows = pixels)
    const int *p_sptr, *p_slen, *p_scol;
    const float *p_sval;
    const int *pt_sptr, *pt_slen, *pt_scol;
    const float *pt_sval;
};

// Launch plan of one kernel family over a set of slices: slice s owns the blocks
// [start[s], start[s+1]).
struct TileMap {
    const int *start;    // device, n + 1 entries
    int n;
};

__device__ __forceinline__ int find_slice(const TileMap &m, int block, int *local) {
    int lo = 0, hi = m.n - 1;
    while (lo < hi) {           // largest s with start[s] <= block
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(m.start + mid) <= block) lo = mid; else hi = mid - 1;
    }
    *local = block - __ldg(m.start + lo);
    return lo;
}

// ---------------------------------------------------------------------------------
// Reductions.  Each block reduces its per-thread values (FP32 within a warp, FP64
// across warps), writes them to partials[block][*], and the last block of a slice to
// finish (atomic ticket) sums that slice's partials in block order -- a fixed order,
// so results are deterministic -- and runs a finaliser.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int NV, int NT>
__device__ __forceinline__ void block_sum_to(const float (&v)[NV], double *out /* NV, smem or global */,
                                             double *smem /* NV * (NT/32) */) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        float s = warp_sum(v[k]);
        if (lane == 0) smem[k * (NT / 32) + w] = (double)s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double acc = 0.0;
        for (int i = 0; i < NT / 32; ++i) acc += smem[threadIdx.x * (NT / 32) + i];
        out[threadIdx.x] = acc;
    }
}

// Returns true in all threads of the block that finished last for its slice.
__device__ __forceinline__ bool last_block_of_slice(unsigned int *counter, int n_blocks, int *flag_smem) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int ticket = atomicAdd(counter, 1u);
        int last = (ticket == (unsigned int)(n_blocks - 1));
        if (last) *counter = 0u;     // re-arm for the next launch (stream-ordered)
        *flag_smem = last;
    }
    __syncthreads();
    if (*flag_smem) __threadfence();
    return *flag_smem != 0;
}

// Blocks per first-level group of the two-level reduction below; doubles per block (and
// per group) in the partial-sum arrays.
constexpr int kRedGroup = 32;
constexpr int kMaxTrials = 16;
constexpr int kPartialStride = kMaxTrials + 8;

// All NT threads of a finishing block: res[k] = sum over blocks first .. first + count - 1
// of src[block * stride + k], k < NV (NV <= 32), as a fixed-shape tree, so the result is
// deterministic.  FP64 adds have a long latency on this GPU, so the tree is wide rather than
// deep: thread t takes value k = t % NVP (NVP = NV rounded up to a power of two) and blocks
// j, j + J, ... (j = t / NVP, J = NT / NVP); the threads of a warp that hold the same k
// combine by shuffles, and thread k adds the NT/32 warp results.
template <int NV, int NT>
__device__ __forceinline__ void group_sum(const double *src, int stride, int first, int count,
                                          double *wpart /* NV * NT/32, smem */, double *res /* NV */) {
    constexpr int NVP = NV <= 1 ? 1 : NV <= 2 ? 2 : NV <= 4 ? 4 : NV <= 8 ? 8 : NV <= 16 ? 16 : 32;
    constexpr int J = NT / NVP, NW = NT / 32;
    const int t = threadIdx.x, k = t % NVP, j = t / NVP;
    double a = 0.0;
    if (k < NV) {
        int b = j;
        if (b < count) a = __ldcg(src + (size_t)(first + b) * stride + k);
        for (b += J; b < count; b += J) a += __ldcg(src + (size_t)(first + b) * stride + k);
    }
#pragma unroll
    for (int o = NVP; o < 32; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    const int lane = t & 31, w = t >> 5;
    if (lane < NV) wpart[w * NV + lane] = a;
    __syncthreads();
    if (t < NV) {
        double r = 0.0;
        for (int i = 0; i < NW; ++i) r += wpart[i * NV + t];
        res[t] = r;
    }
    __syncthreads();
}

// Two-level deterministic reduction of the NV per-block partial sums that the nblk blocks
// of a slice wrote to partials[b0 + lb][0 .. NV) (row stride `stride`), lb = the calling
// block's index within the slice.  Every kRedGroup consecutive blocks form a group: the
// block of a group that finishes last (atomic ticket) sums the group in block order and
// stores the result in S.gpart; the group finisher that comes last sums the group results
// in group order.  Returns true only in that block, with the totals in res (smem).
// Spreads the FP64 work over nblk / kRedGroup SMs instead of one.
template <int NV, int NT>
__device__ __forceinline__ bool reduce_slice(const SliceDev &S, const double *partials, int stride, int b0,
                                             int nblk, int lb, double *wpart, double *res, int *flag) {
    const int ng = (nblk + kRedGroup - 1) / kRedGroup;
    const int g = lb / kRedGroup;
    const int gsize = min(kRedGroup, nblk - g * kRedGroup);
    if (!last_block_of_slice(S.ctr + 1 + g, gsize, flag)) return false;
    group_sum<NV, NT>(partials, stride, b0 + g * kRedGroup, gsize, wpart, res);
    if (ng == 1) return true;
    if (threadIdx.x < NV) S.gpart[(size_t)g * kPartialStride + threadIdx.x] = res[threadIdx.x];
    if (!last_block_of_slice(S.ctr, ng, flag)) return false;
    group_sum<NV, NT>(S.gpart, kPartialStride, 0, ng, wpart, res);
    return true;
}

// ---------------------------------------------------------------------------------
// Launch helpers (host).
// ---------------------------------------------------------------------------------
struct Workspace;   // defined in geometry.cu

}  // namespace eptv
