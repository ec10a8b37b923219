// Internal definitions of the sm_103a EPTV library: per-slice descriptors, launch plans,
// the canonical plane-crossing arithmetic shared by the projector (K1) and its exact
// adjoint (K2), and block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "eptv.h"

namespace eptv {

// ---------------------------------------------------------------------------------
// Programmatic dependent launch.  A kernel started by launch_pdl may be scheduled while
// the previous kernel of its stream (or CUDA graph) still finishes; it calls pdl_wait()
// before its first access to global memory, which returns once that kernel has completed
// and its writes are visible (at once when there is no such dependency).  Only kernels
// that begin with pdl_wait() are launched this way.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

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
    SC_TIMEOUT = SC_Q0 + 9,   // set to 1 when a bounded device wait ran out
    SC_COUNT
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
    const int *k1_order; // [nv * ceil(nb / 32)] projector work units, heaviest first (or null)
    // solver state (device workspace of the handle, or caller buffers)
    const float *y;      // data sinogram
    float *u, *uT;       // current image / CGLS iterate and its transpose
    float *s, *sT, *t;   // CGLS image vectors
    float *r, *q;        // CGLS sinogram vectors
    float *fa, *fb;      // (P2) iterate ping-pong
    float *ga, *gb;      // (P2) gradient ping-pong
    float *tv_scr;       // [n_edges] FP32 scratch (half-edge T^2 for the sigma selection)
    const float *wprior; // per-pixel prior weight map, or null
    float *wout;         // optional output of the final edge weights
    double *sc;          // [kScalarStride] scalars
    double *log;         // optional per-iteration log: [n_outer * n_gd] steps, then [n_outer] sigmas
    int log_outer;       // capacity in outer iterations (0: no log)
    int log_gd;          // GD iterations per outer iteration in the log layout
    // reduction bookkeeping of this slice in its batch: the ticket counter ctr[0] and the
    // exact accumulators ([kPartialStride][kAccCopies][kAccStride] words, zero between
    // launches)
    unsigned int *ctr;
    unsigned long long *acc;
    // persistent (P2) kernel K4p: the batch's grid-barrier words (p2bar[0] the arrival
    // count, p2bar[1] its value when the next launch starts), this slice's three rotating
    // exact-accumulator sets and its three sigma-selection histograms (kP2HistWords words,
    // zero between launches)
    unsigned int *p2bar;
    unsigned long long *p2acc;
    unsigned int *p2hist;
    // stored operator (null unless selected): SELL-32 P (rows = rays), P^T (rows = pixels)
    const int *p_sptr, *p_slen, *p_scol;
    const float *p_sval;
    const int *pt_sptr, *pt_slen, *pt_scol;
    const float *pt_sval;
    int pt_keep;         // P^T slices [0, pt_keep) are read with an L2 evict_last policy
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

// Doubles per block in the partial-sum arrays (the most values one reduction carries).
constexpr int kMaxTrials = 16;
constexpr int kPartialStride = kMaxTrials + 8;

// Exact, order-independent sums of FP64 block partials.  A value x is a binary fixed-point
// number with its least significant bit at 2^kAccLsbExp; that number is split into 32-bit
// chunks, and chunk c is added with a 64-bit integer atomic into word c of the value's
// accumulator.  Integer addition is associative, so the total does not depend on the order
// in which blocks finish, and the block that finishes last rounds the exact total once to
// FP64.  Every block partial of the kernels is a sum of FP32 numbers, hence a multiple of
// 2^-149, so for them the total is the correctly rounded exact sum; finite bits below
// 2^kAccLsbExp (smaller doubles) are truncated toward zero.  Non-finite values, and
// magnitudes of 2^191 and above, set flags (result NaN, or +-Inf); the two top words stay
// free for carries, so a total of up to 2^31 values cannot overflow.  Each value has
// kAccCopies accumulators (block b adds into copy b mod kAccCopies), so that blocks
// finishing together do not queue on the same addresses; the copies are summed (exactly)
// when the total is read.
constexpr int kAccChunks = 12;                 // bits 2^-149 .. 2^234
constexpr int kAccStride = kAccChunks + 1;     // + one word of flags
constexpr int kAccCopies = 8;                  // divides 32
constexpr int kAccLsbExp = -149;
constexpr unsigned long long kAccNaN = 1ull, kAccPosInf = 2ull, kAccNegInf = 4ull;

// Adds x into one accumulator copy (kAccStride words).
__device__ __forceinline__ void acc_add(unsigned long long *acc, double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const bool neg = (b >> 63) != 0;
    const int ex = (int)((b >> 52) & 0x7FFull);
    unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (ex == 0x7FF) {
        atomicOr(acc + kAccChunks, m ? kAccNaN : (neg ? kAccNegInf : kAccPosInf));
        return;
    }
    if (ex) m |= 1ull << 52;
    if (m == 0ull) return;
    int sh = (ex ? ex : 1) - 1075 - kAccLsbExp;            // |x| = m 2^(sh + kAccLsbExp)
    if (sh < 0) {
        if (sh <= -53) return;
        m >>= -sh;
        sh = 0;
        if (m == 0ull) return;
    }
    if (sh > 32 * (kAccChunks - 4) + 31) {                 // |x| >= 2^191
        atomicOr(acc + kAccChunks, neg ? kAccNegInf : kAccPosInf);
        return;
    }
    const int c = sh >> 5, r = sh & 31;
    const unsigned long long lo = m << r;                  // m < 2^53: m 2^r < 2^84
    const unsigned long long hi = r ? (m >> (64 - r)) : 0ull;
    const unsigned long long d[3] = {lo & 0xFFFFFFFFull, lo >> 32, hi};
#pragma unroll
    for (int q = 0; q < 3; ++q)
        if (d[q]) atomicAdd(acc + c + q, neg ? (0ull - d[q]) : d[q]);
}

// The exact total held in the words w (two's complement chunks, carries not yet
// propagated) and flags, rounded to nearest FP64.
__device__ __forceinline__ double acc_round(const long long (&w)[kAccChunks], unsigned long long flags) {
    if ((flags & kAccNaN) || (flags & (kAccPosInf | kAccNegInf)) == (kAccPosInf | kAccNegInf))
        return __longlong_as_double(0x7FF8000000000000ll);
    if (flags & kAccPosInf) return __longlong_as_double(0x7FF0000000000000ll);
    if (flags & kAccNegInf) return __longlong_as_double((long long)0xFFF0000000000000ull);
    // carries: 32-bit digits, the sign in the final carry (0 or -1: |total| < 2^222)
    unsigned int dg[kAccChunks];
    long long carry = 0;
#pragma unroll
    for (int i = 0; i < kAccChunks; ++i) {
        const long long t = w[i] + carry;
        dg[i] = (unsigned int)(t & 0xFFFFFFFFll);
        carry = t >> 32;                                   // floor division by 2^32
    }
    const bool neg = carry < 0;
    if (neg) {                                             // magnitude: two's complement
        unsigned long long c1 = 1ull;
#pragma unroll
        for (int i = 0; i < kAccChunks; ++i) {
            const unsigned long long t = (unsigned long long)(~dg[i]) + c1;
            dg[i] = (unsigned int)t;
            c1 = t >> 32;
        }
    }
    // leading digit h and the two below it (selects, not indexing: stays in registers)
    int h = -1;
#pragma unroll
    for (int i = 0; i < kAccChunks; ++i)
        if (dg[i]) h = i;
    if (h < 0) return 0.0;
    unsigned long long d0 = 0u, d1 = 0u, d2 = 0u;
    bool sticky = false;
#pragma unroll
    for (int i = 0; i < kAccChunks; ++i) {
        if (i == h) d0 = dg[i];
        if (i == h - 1) d1 = dg[i];
        if (i == h - 2) d2 = dg[i];
        if (i < h - 2) sticky |= dg[i] != 0u;
    }
    // the top 64 bits of the magnitude (leading one at bit 63) and a sticky bit for the
    // rest; the value is t64 2^e.  Rounded to 53 bits, nearest even, in integer arithmetic
    // (|total| < 2^235: no overflow; >= 2^-149: no subnormal)
    const int lz = __clz((unsigned int)d0);
    const unsigned long long top = (d0 << 32) | d1;
    const unsigned long long t64 = lz ? ((top << lz) | (d2 >> (32 - lz))) : top;
    sticky |= (lz ? ((d2 << lz) & 0xFFFFFFFFull) : d2) != 0ull;
    int e = 32 * (h - 1) - lz + kAccLsbExp;
    unsigned long long m = t64 >> 11;                      // 53 bits
    const unsigned long long rest = t64 & 0x7FFull;
    const bool half = (rest & 0x400ull) != 0;
    const bool below = (rest & 0x3FFull) != 0 || sticky;
    if (half && (below || (m & 1ull))) {
        ++m;
        if (m >> 53) { m >>= 1; ++e; }
    }
    const unsigned long long biased = (unsigned long long)(e + 11 + 52 + 1023);
    const unsigned long long bits = (biased << 52) | (m & 0xFFFFFFFFFFFFFull) | (neg ? (1ull << 63) : 0ull);
    return __longlong_as_double((long long)bits);
}

// Adds the FP32 value x exactly into one accumulator copy (kAccStride words, global or
// shared memory): its 24-bit significand lands in at most two 32-bit chunks, with integer
// atomics only (no FP64 arithmetic).  Same total as acc_add((double)x).
__device__ __forceinline__ void acc_add_f32(unsigned long long *acc, float x) {
    const unsigned int b = __float_as_uint(x);
    const bool neg = (b >> 31) != 0;
    const int ex = (int)((b >> 23) & 0xFFu);
    unsigned int m = b & 0x7FFFFFu;
    if (ex == 0xFF) {
        atomicOr(acc + kAccChunks, m ? kAccNaN : (neg ? kAccNegInf : kAccPosInf));
        return;
    }
    if (ex) m |= 0x800000u;
    if (m == 0u) return;
    const int sh = (ex ? ex : 1) - 1;                       // |x| = m 2^(sh + kAccLsbExp)
    const int c = sh >> 5, r = sh & 31;
    const unsigned long long v = (unsigned long long)m << r;  // < 2^55
    const unsigned long long lo = v & 0xFFFFFFFFull, hi = v >> 32;
    atomicAdd(acc + c, neg ? (0ull - lo) : lo);
    if (hi) atomicAdd(acc + c + 1, neg ? (0ull - hi) : hi);
}

// All NT threads of a block (NT a multiple of 32), after every contribution is visible:
// res[k] = the total of value k (k < NV) over its kAccCopies copies (acc[k][copy][word]);
// re-zeroes the accumulators unless ZERO is false.  Lane groups of kAccCopies read one copy
// each and add the words with shuffles (integer sums: exact).
template <int NV, int NT, bool ZERO = true, int C = kAccCopies>
__device__ __forceinline__ void acc_read(unsigned long long *acc, double *res) {
    static_assert(C >= 1 && C <= kAccCopies && (C & (C - 1)) == 0, "copies: a power of two");
    for (int base = 0; base < NV * C; base += NT) {
        const int t = base + (int)threadIdx.x;
        const bool mine = t < NV * C;
        long long w[kAccChunks];
        unsigned long long fl = 0ull;
        unsigned long long *a = acc + ((size_t)(mine ? (t / C) * kAccCopies + t % C : 0)) * kAccStride;
#pragma unroll
        for (int i = 0; i < kAccChunks; ++i) w[i] = mine ? (long long)__ldcg(a + i) : 0ll;
        if (mine) {
            fl = __ldcg(a + kAccChunks);
            if (ZERO) {
#pragma unroll
                for (int i = 0; i < kAccStride; ++i) a[i] = 0ull;
            }
        }
#pragma unroll
        for (int o = 1; o < C; o <<= 1) {
#pragma unroll
            for (int i = 0; i < kAccChunks; ++i) w[i] += __shfl_xor_sync(0xffffffffu, w[i], o);
            fl |= __shfl_xor_sync(0xffffffffu, fl, o);
        }
        if (mine && (t % C) == 0) res[t / C] = acc_round(w, fl);
    }
}

// One warp: the FP32 warp sums of its NV per-thread values, each added exactly (integer
// atomics) into the block's shared accumulator sacc[k] (kAccStride words) by lane k.
template <int NV>
__device__ __forceinline__ void warp_acc(const float (&v)[NV], unsigned long long *sacc) {
    static_assert(NV <= 32, "one lane per value");
    const int lane = threadIdx.x & 31;
    float mine = 0.0f;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const float sv = warp_sum(v[k]);
        if (lane == k) mine = sv;
    }
    if (lane < NV) acc_add_f32(sacc + lane * kAccStride, mine);
}

// All NT threads, after the block's contributions to sacc are complete (__syncthreads):
// adds the nonzero words of the block's shared accumulators (NV values) into copy `copy`
// of the global accumulators gacc ([value][kAccCopies][kAccStride] words).
template <int NV, int NT>
__device__ __forceinline__ void acc_push(const unsigned long long *sacc, unsigned long long *gacc, int copy) {
    for (int w = threadIdx.x; w < NV * kAccStride; w += NT) {
        const int k = w / kAccStride, i = w - k * kAccStride;
        const unsigned long long x = sacc[w];
        if (x) {
            unsigned long long *dst = gacc + ((size_t)k * kAccCopies + copy) * kAccStride + i;
            if (i == kAccChunks) atomicOr(dst, x);
            else atomicAdd(dst, x);
        }
    }
}

// Deterministic reduction of the NV per-block partial sums that the nblk blocks of a slice
// wrote to partials[b0 + lb][0 .. NV) (row stride `stride`), lb = the calling block's index
// within the slice: every block adds its row into the slice's exact accumulators, and the
// block that finishes last (atomic ticket) reads the totals.  Returns true only in that
// block, with the totals in res (smem).  (wpart: unused, kept for the call sites' shape.)
template <int NV, int NT>
__device__ __forceinline__ bool reduce_slice(const SliceDev &S, const double *partials, int stride, int b0,
                                             int nblk, int lb, double *wpart, double *res, int *flag) {
    (void)wpart;
    __syncthreads();                                       // the row may come from any thread
    if (threadIdx.x < NV)
        acc_add(S.acc + ((size_t)threadIdx.x * kAccCopies + (lb % kAccCopies)) * kAccStride,
                partials[(size_t)(b0 + lb) * stride + threadIdx.x]);
    if (!last_block_of_slice(S.ctr, nblk, flag)) return false;
    acc_read<NV, NT>(S.acc, res);
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------------
// Launch helpers (host).
// ---------------------------------------------------------------------------------
struct Workspace;   // defined in geometry.cu

}  // namespace eptv
