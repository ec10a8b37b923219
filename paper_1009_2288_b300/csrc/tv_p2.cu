// K4p: the whole (P2) descent of one outer iteration -- n_gd gradient-descent iterations
// with Armijo steps (Sec. 2.2; Eqs. 5, 9, A2, A3) and the clamp of step 3 -- in ONE
// cooperative launch.
//
// Each block owns a rectangle ("region") of RTX x RTY of the 32 x 8 tiles that K4 launches
// one block per, and keeps in shared memory, for all GD iterations: the iterate f on the
// region + 2-pixel halo, v on the region + 1, and g on the region + 2.  First, sigma
// (Sec. 2.1): the sel_rank-th smallest half-edge magnitude T of v over the slice, by K5's
// exact radix selection (12 + 12 + 8 bits of the FP32 keys) over the half-edges each block
// owns (its pixels' left and upper sides, and the right / bottom image border in the last
// region column / row), one grid barrier after each pass, every block scanning the slice's
// histogram itself.  Then per GD iteration:
//   phase 2  T, w, q = w D / T of every half-edge around the region + 1 (Eqs. A3, 5);
//   phase 3  g = lambda (f - v) + dJ/df on the region + 1 (Eqs. 9, A2); the owned values go
//            to an exchange image;
//   phase 4  per tile (tile_sums, the per-thread assignment K4 uses): the fidelity sums
//            <g, f-v>, |g|^2, |f-v|^2 and, for the first three trial steps, the energy
//            change of the owned half-edges with the weights frozen; each warp adds its FP32
//            sums exactly (integer fixed point) into the block's accumulators, and the
//            block's words go into the slice's accumulators (one set per barrier, three in
//            rotation);
//   barrier  one grid-wide arrival / wait (bounded), polled by one warp; meanwhile
//            warp 1 prepares the next iteration's trial steps for every possible outcome;
//   decide   every block reads the exact totals and takes the same FP64 Armijo decision
//            (the first passing trial); when none of the three passes, the remaining
//            trials are summed the same way behind one more barrier and the decision is
//            taken over all of them; the slice's first block keeps the record and writes
//            it to the slice's scalars and log once, at the end;
//   apply    f <- f - t g on the region + 2, the ring 2 of g read from the neighbours'
//            exchange values of this iteration.
// After the last iteration the owned pixels get f = max(f, 0) (step 3) and go to u and u^T.
//
// Because the per-pixel / per-edge arithmetic is K4's (tv_stencil.cuh), every warp's sums
// are the same fixed functions of its tile in both kernels, and everything above a warp is
// summed exactly, K4p produces bit for bit the same iterates, steps and scalars as n_gd
// launches of K4 followed by K4u.
//
// Co-residency: the launch is cooperative (all blocks resident or the launch fails), and
// every wait has a bound: a block that waits longer than about a second sets SC_TIMEOUT in
// its slice's scalars and returns, so that the host reports EPTV_ERR_TIMEOUT instead of a
// hung context.  The launch re-arms itself: the barrier counter only grows (p2bar[1] holds
// its value at the start of the next launch, compares are modulo 2^32), each accumulator
// set is zeroed by the slice's first block before its first use, and the selection
// histograms are zeroed once every block has passed the first GD barrier.  The host zeroes
// the barrier words and histograms at the start of every call (after a wait that ran out
// they are not consistent).
#include <algorithm>
#include <atomic>

#include "eptv_internal.cuh"
#include "kernels.cuh"
#include "tv_stencil.cuh"

namespace eptv {

// ------------------------------------------------------------------ grid barrier

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_gpu(unsigned int *p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits until *bar reaches target (modulo 2^32: the counter only grows), at most
// max_cycles SM cycles and at most kP2WaitSpins polls (~2.7 s with the back-off).  Returns
// false if a bound ran out.
constexpr long long kP2WaitSpins = 1ll << 26;

__device__ __forceinline__ bool p2_wait(const unsigned int *bar, unsigned int target,
                                        long long max_cycles, volatile int *seen) {
    const long long t0 = clock64();
    for (long long spins = 0; spins < kP2WaitSpins; ++spins) {
        if (*seen) return true;                            // another warp of the block saw it
        if ((int)(ld_acquire_gpu(bar) - target) >= 0) {
            *seen = 1;
            return true;
        }
        if (spins > 256) __nanosleep(32);
        if ((spins & 63) == 63 && clock64() - t0 > max_cycles) return false;
    }
    return false;
}

// Accumulator copies K4p's blocks spread their words over (block b: copy b mod kP2Copies).
// Every block reads all copies after each barrier, and with one block per SM the push
// atomics of 128 blocks on one copy cost less than the longer read-out of more copies
// (per GD iteration at 512^2: 4 copies 13.0 us, 2 copies 12.6, 1 copy 12.1).
constexpr int kP2Copies = 1;

// Armijo trials evaluated before a GD iteration's grid barrier (at most the run's
// max_trials).  The others are evaluated behind one more barrier, and only when none of
// these passes.  A trial's exact total does not depend on which evaluation produced it,
// so the decision is bit for bit that of one evaluation of every trial.  With
// t0 = min(2 t_prev, t_max) the accepted trial is nearly always one of the first three
// (the first 12 outer iterations at 512^2, 40 views x 888 bins: 22 % the first, 52 % the
// second, 25 % the third, none later).
constexpr int kP2FirstTrials = 3;

// One pass of the selection scan, run by every block on the slice's histogram gh (NB
// bins): the bin holding the remaining rank (1-based) and the rank within it, to *s_bin and
// *s_rank.  Bins are summed per thread (PER consecutive bins), the thread sums are
// prefix-summed across the block, and the thread whose bins hold the rank searches them.
template <int NT, int NB>
__device__ __forceinline__ void p2_sel_scan(const unsigned int *gh, long long rank,
                                            unsigned long long *s_w, int *s_bin, long long *s_rank) {
    constexpr int PER = NB >= NT ? NB / NT : 1;
    static_assert(NB >= NT ? NB % NT == 0 : true, "bins split evenly over the threads");
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    unsigned int v[PER];
    unsigned long long local = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int b = t * PER + q;
        v[q] = (b < NB) ? __ldcg(gh + b) : 0u;
        local += v[q];
    }
    unsigned long long inc = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    unsigned long long before = 0;
    for (int i = 0; i < w; ++i) before += s_w[i];
    inc += before;
    const unsigned long long exc = inc - local;
    if ((long long)exc < rank && rank <= (long long)inc) {
        unsigned long long cum = exc;
        int b = t * PER;
        for (int q = 0; q < PER; ++q, ++b) {
            if ((long long)(cum + v[q]) >= rank) break;
            cum += v[q];
        }
        *s_bin = b;
        *s_rank = rank - (long long)cum;
    }
    __syncthreads();
}

// ------------------------------------------------------------------ layout

template <int RTX, int RTY, int KT>
struct P2Shape {
    static constexpr int RW = RTX * kTileW, RH = RTY * kGdTileRows;
    static constexpr int TILES = RTX * RTY;
    static constexpr int NG = TILES < 4 ? TILES : 4;       // tile groups of 128 threads
    static constexpr int NT = 128 * NG;
    static constexpr int NV = KT + 4;
    static constexpr int FW = RW + 4, FH = RH + 4;         // f, g, prior map: region + 2
    static constexpr int VW = RW + 2, VH = RH + 2;         // v and the g region: region + 1
    static constexpr int QXW = RW + 3, QXH = RH + 2;       // x-edges around the g region
    static constexpr int QYW = RW + 2, QYH = RH + 3;       // y-edges around the g region
    static constexpr int KTP = (KT + 3) & ~3;
    static constexpr int N_DBL = NV + KT + 4;  // tot, s_td, t_prev / decision
    static constexpr int N_FLT = KTP + 3 * FH * FW + VH * VW + 3 * QXH * QXW + 3 * QYH * QYW;
    static constexpr size_t SMEM = sizeof(double) * N_DBL + sizeof(float) * N_FLT;
};

template <int RTX, int RTY, int KT>
__global__ void __launch_bounds__(P2Shape<RTX, RTY, KT>::NT, 1)
k4p_descent(const SliceDev *__restrict__ sls, TileMap map, const ParamsDev *__restrict__ P,
            P2Args pa)
{
    using Sh = P2Shape<RTX, RTY, KT>;
    constexpr int RW = Sh::RW, RH = Sh::RH, NV = Sh::NV, NG = Sh::NG;
    constexpr int FW = Sh::FW, FH = Sh::FH, VW = Sh::VW, VH = Sh::VH;
    constexpr int QXW = Sh::QXW, QXH = Sh::QXH, QYW = Sh::QYW, QYH = Sh::QYH;
    constexpr int NT = Sh::NT;

    extern __shared__ __align__(16) double p2_smem[];
    double *tot = p2_smem;                       // [NV] exact totals
    double *s_td = tot + NV;                     // [KT] trial steps (FP64 copies)
    double *s_misc = s_td + KT;                  // t_prev, t_step, flags
    float *s_t = reinterpret_cast<float *>(s_misc + 4);
    float *F = s_t + Sh::KTP;
    float *G = F + FH * FW;
    float *Wp = G + FH * FW;
    float *V = Wp + FH * FW;
    float *QX = V + VH * VW;
    float *TX = QX + QXH * QXW;
    float *WX = TX + QXH * QXW;
    float *QY = WX + QXH * QXW;
    float *TY = QY + QYH * QYW;
    float *WY = TY + QYH * QYW;
    __shared__ int s_abort;
    __shared__ int s_seen[2];                              // barrier seen (per iteration parity)
    // warps polling the barrier (lane 0 each; the first to see it tells the others through
    // s_seen).  One: more polls in flight were measured slower (4 warps +0.2 us, 8 warps
    // +1.8 us per GD iteration at 512^2), their loads queue on the counter's line.
    constexpr int kPollers = 1;
    __shared__ unsigned long long sacc[NV * kAccStride];   // the block's exact sums
    __shared__ double s_tot2[NV];                          // totals of a second trial evaluation
    __shared__ int s_more;                                 // the iteration evaluates more trials
    // candidate trial steps of the next iteration ((K + 1) K <= 32: K <= 4)
    constexpr bool kCand = (KT + 1) * KT <= 32;
    __shared__ float cand_f[kCand ? (KT + 1) * KT : 1];
    __shared__ double cand_d[kCand ? (KT + 1) * KT : 1];
    __shared__ unsigned int s_hist[kHistBins];             // sigma: the block's histogram
    __shared__ unsigned long long s_w[NT / 32];
    __shared__ int s_bin;
    __shared__ long long s_rank;
    struct Record { double e_first, t_step, e_last, t_prev; int nacc, nfail, bad; };
    Record rec{0.0, 0.0, 0.0, 0.0, 0, 0, 0};

    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const int nx = S.nx, ny = S.ny;
    const int tiles_x = (nx + kTileW - 1) / kTileW, tiles_y = (ny + kGdTileRows - 1) / kGdTileRows;
    const int regions_x = (tiles_x + RTX - 1) / RTX;
    const int ry = local / regions_x, rx = local - ry * regions_x;
    const int RX0 = rx * RW, RY0 = ry * RH;
    const int tid = threadIdx.x;
    const int K = pa.n_trials;
    const float eps2 = (float)(P->eps * P->eps);
    const float lam = (float)P->lambda;
    const float *vv = pa.v ? pa.v : S.u;
    unsigned long long *acc_slice = S.p2acc;
    (void)tiles_y;

    int mode = P->weights_mode;
    if (mode == EPTV_WEIGHTS_PRIOR) {
        mode = (S.wprior && S.sc[SC_OUTER] < (double)P->prior_iters) ? EPTV_WEIGHTS_PRIOR
                                                                      : EPTV_WEIGHTS_EPTV;
    }
    const int k_outer = (int)S.sc[SC_OUTER];
    // barrier b of this launch (0, 1, 2: the sigma passes; then one or two per GD
    // iteration) completes when the counter reaches base + (b + 1) per_bar
    const unsigned int base = ld_acquire_gpu(S.p2bar + 1);
    const unsigned int per_bar = gridDim.x + (unsigned int)pa.bar_extra;
    const int nblk = __ldg(map.start + si + 1) - __ldg(map.start + si);
    if (tid == 0) {
        s_misc[0] = S.sc[SC_TPREV];
        s_abort = 0;
        s_seen[0] = 0;
        s_seen[1] = 0;
    }

    // v at pixel p; pa.fold: the CGLS left its last update u += a s to this kernel (the
    // arithmetic of k3_update_us, so v is bit for bit the u that update would store)
    const float fold_a = pa.fold ? (float)S.sc[SC_A] : 0.0f;
    auto v_at = [&](int p) -> float {
        const float x = __ldcg(vv + p);
        return pa.fold ? fmaf(fold_a, __ldcg(S.s + p), x) : x;
    };
    // f = v on the region + 2 (0 outside the image), g = 0, the prior map (edge-replicated)
    for (int idx = tid; idx < FH * FW; idx += NT) {
        const int r = idx / FW, c = idx - r * FW;
        const int i = RX0 - 2 + c, j = RY0 - 2 + r;
        float fv = 0.0f;
        if (i >= 0 && i < nx && j >= 0 && j < ny) fv = v_at(j * nx + i);
        F[idx] = fv;
        G[idx] = 0.0f;
        if (mode == EPTV_WEIGHTS_PRIOR) {
            const int ci = min(max(i, 0), nx - 1), cj = min(max(j, 0), ny - 1);
            Wp[idx] = __ldg(S.wprior + (size_t)cj * nx + ci);
        } else {
            Wp[idx] = 0.0f;
        }
    }
    for (int idx = tid; idx < VH * VW; idx += NT) {
        const int r = idx / VW, c = idx - r * VW;
        const int i = RX0 - 1 + c, j = RY0 - 1 + r;
        float vx = 0.0f;
        if (i >= 0 && i < nx && j >= 0 && j < ny) vx = v_at(j * nx + i);
        V[idx] = vx;
    }
    // the slice's first accumulator set is used first after the sigma barriers
    if (local == 0)
        for (int w = tid; w < NV * kAccCopies * kAccStride; w += NT) acc_slice[w] = 0ull;
    if (tid == 0 && K > 0) trial_steps(P, s_misc[0], K, s_t, s_td);     // first GD iteration's
    __syncthreads();

    // one grid barrier (number b), arrival after the block's writes; false if a wait ran out
    auto grid_sync = [&](int b) -> bool {
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            red_release_add_gpu(S.p2bar, 1u);
        }
        if ((tid & 31) == 0 && (tid >> 5) < kPollers) {
            if (!p2_wait(S.p2bar, base + (unsigned int)(b + 1) * per_bar, pa.wait_cycles, &s_seen[b & 1]))
                s_abort = 1;
            __threadfence();
        }
        if (tid == 0) s_seen[(b + 1) & 1] = 0;             // re-armed for the next barrier
        __syncthreads();
        return !s_abort;
    };

    // sigma: the keys of T^2 (K5's half_edge_T2) of the owned half-edges of v, x-edges
    // (i, j) between (i - 1, j) and (i, j) first, then y-edges between (i, j - 1) and (i, j);
    // sqrtf is monotone, so sigma = sqrtf(the k-th smallest T^2), bit for bit the k-th
    // smallest T
    constexpr int KEYS = (2 * (RW + 1) * (RH + 1) + NT - 1) / NT;
    unsigned int keys[KEYS];
    const int cx1 = min(RX0 + RW, nx), cy1 = min(RY0 + RH, ny);
    const int ncol = cx1 - RX0, nrow = cy1 - RY0;
    const int nxe = ncol + (RX0 + RW >= nx ? 1 : 0);       // x-edge columns owned
    const int nye = nrow + (RY0 + RH >= ny ? 1 : 0);       // y-edge rows owned
    const int n_ox = nxe * nrow, n_own = n_ox + ncol * nye;
    bool nonfinite = false;
#pragma unroll
    for (int k = 0; k < KEYS; ++k) {
        const int e = tid + k * NT;
        unsigned int key = 0u;
        if (e < n_own) {
            float D, T2;
            if (e < n_ox) {
                const int r = e / nxe, c = e - r * nxe;
                const float *q = F + (r + 2) * FW + (c + 1);            // pixel (i - 1, j)
                T2 = edge_T2(eps2, q[0], q[1], q[FW], q[FW + 1], q[-FW], q[-FW + 1], &D);
            } else {
                const int e2 = e - n_ox, r = e2 / ncol, c = e2 - r * ncol;
                const float *q = F + (r + 1) * FW + (c + 2);            // pixel (i, j - 1)
                T2 = edge_T2(eps2, q[0], q[FW], q[1], q[FW + 1], q[-1], q[FW - 1], &D);
            }
            nonfinite |= !isfinite(T2);
            key = sel_key(T2);
        }
        keys[k] = key;
    }
    if (nonfinite) S.sc[SC_NONFINITE] = 1.0;
    long long rank = S.sel_rank;
    unsigned int prefix = 0u;
    for (int pass = 0; pass < 3; ++pass) {
        const int nbins = (pass == 2) ? 256 : kHistBins;
        for (int b = tid; b < nbins; b += NT) s_hist[b] = 0u;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KEYS; ++k)
            if (tid + k * NT < n_own) sel_hist_add(s_hist, keys[k], pass, prefix);
        __syncthreads();
        unsigned int *gh = S.p2hist + pass * kHistBins;
        for (int b = tid; b < nbins; b += NT) {
            const unsigned int c = s_hist[b];
            if (c) atomicAdd(gh + b, c);
        }
        if (!grid_sync(pass)) {
            if (tid == 0) S.sc[SC_TIMEOUT] = 1.0;
            return;
        }
        if (pass == 2) p2_sel_scan<NT, 256>(gh, rank, s_w, &s_bin, &s_rank);
        else p2_sel_scan<NT, kHistBins>(gh, rank, s_w, &s_bin, &s_rank);
        rank = s_rank;
        prefix = (pass == 0) ? (unsigned int)s_bin : (prefix << (pass == 1 ? 12 : 8)) | (unsigned int)s_bin;
    }
    const double sigma = fmax((double)sqrtf(__uint_as_float(prefix)), P->sigma_floor);
    if (local == 0 && tid == 0) {
        S.sc[SC_SIGMA] = sigma;
        if (S.log && k_outer >= 0 && k_outer < S.log_outer)
            S.log[(size_t)S.log_outer * S.log_gd + k_outer] = sigma;
    }
    const float sig = (float)sigma;
    const float inv_s2 = 1.0f / (sig * sig);

    const int grp = tid >> 7, vt = tid & 127;
    constexpr int kRing = 2 * FW + 2 * (FH - 2);
    static_assert(kRing <= NT, "one ring position per thread");
    // GD-phase barriers passed so far: barrier number 3 + ab, accumulator set ab mod kP2Sets
    // (a second evaluation of trials adds a barrier; every block takes the same decisions,
    // so every block counts the same barriers)
    int ab = 0;
    const int K1 = min(K, kP2FirstTrials);
    // the slice's next accumulator set, zeroed in the phase before the barrier that
    // precedes its use (its last use was read by every block before that barrier's
    // predecessor)
    auto zero_next_set = [&]() {
        if (local == 0) {
            unsigned long long *nxt = acc_slice + (size_t)((ab + 1) % kP2Sets) * kP2SetWords;
            for (int w = tid; w < NV * kAccCopies * kAccStride; w += NT) nxt[w] = 0ull;
        }
    };
    // phase 4 for the trials m0 .. m0 + nk - 1: the tiles' sums (tile_sums, the per-thread
    // assignment K4 uses), group grp (128 threads) takes TILES / NG tiles; every warp adds
    // its FP32 sums exactly into the block's accumulators (no barrier between the warps),
    // and the block's words go to the accumulator set ab.  2 x 4 regions: group grp takes
    // tile (row grp, column grp & 1) and (row grp + 2 mod 4, the other column), so that in
    // a region on the image's right or lower border (whose border tiles give one warp of
    // the tile an extra round) every group has at most one border tile.  fid: the fidelity
    // and energy sums are wanted (the first evaluation of the iteration).
    auto tile_phase = [&](int m0, int nk, bool fid, float *wout) {
        for (int k = 0; k < Sh::TILES / NG; ++k) {
            const int q = (RTX == 2 && RTY == 4) ? ((k == 0 ? grp : ((grp + 2) & 3)) * RTX + ((grp & 1) ^ k))
                                                 : grp + k * NG;
            const int ox = (q % RTX) * kTileW, oy = (q / RTX) * kGdTileRows;
            const int X0 = RX0 + ox, Y0 = RY0 + oy;
            float vals[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) vals[k] = 0.0f;
            if (X0 < nx && Y0 < ny) {
                float dJ[KT];
#pragma unroll
                for (int m = 0; m < KT; ++m) dJ[m] = 0.0f;
                tile_sums<KT>(vt, X0, Y0, nx, ny, F + oy * FW + ox, FW, G + (oy + 1) * FW + ox + 1, FW,
                              V + oy * VW + ox, VW, TX + oy * QXW + ox, WX + oy * QXW + ox, QXW,
                              TY + oy * QYW + ox, WY + oy * QYW + ox, QYW, nk, s_t + m0, eps2, wout,
                              &vals[0], &vals[1], &vals[2], &vals[3], dJ);
                if (!fid) vals[0] = vals[1] = vals[2] = vals[3] = 0.0f;
#pragma unroll
                for (int m = 0; m < KT; ++m) vals[4 + m] = dJ[m];
            }
            warp_acc<NV>(vals, sacc);
        }
        __syncthreads();
        acc_push<NV, NT>(sacc, acc_slice + (size_t)(ab % kP2Sets) * kP2SetWords, blockIdx.x % kP2Copies);
    };
    // the final decision r of GD iteration it (warp 0, lane 0 stores)
    auto take_decision = [&](const GdDecision &r, int it) {
        if (tid == 0) {
            s_misc[1] = r.t_step;
            s_misc[0] = r.t_prev;
            if (local == 0) {          // the slice's record, written to its scalars at the end
                if (it == 0) rec.e_first = r.e0;
                rec.t_step = r.t_step;
                rec.e_last = r.e_last;
                rec.t_prev = r.t_prev;
                rec.nacc += r.accepted;
                rec.nfail += 1 - r.accepted;
                rec.bad |= r.bad;
                if (S.log && k_outer >= 0 && k_outer < S.log_outer && it < S.log_gd)
                    S.log[(size_t)k_outer * S.log_gd + it] = r.t_step;
            }
            if (!(kCand && K > 1) && K > 0 && P->step_rule != EPTV_STEP_FIXED)
                trial_steps(P, r.t_prev, K, s_t, s_td);      // for the next iteration
            s_misc[2] = (double)r.index;
        }
    };
    for (int it = 0; it < pa.n_gd; ++it) {
        for (int w = tid; w < NV * kAccStride; w += NT) sacc[w] = 0ull;
        zero_next_set();

        // phase 2: half-edges around the g region (x-edge (a, b) and y-edge (a, b) of one
        // position share four of their six f values)
        for (int idx = tid; idx < QYH * QXW; idx += NT) {
            const int a = idx / QXW, b = idx - a * QXW;
            const float f00 = F[a * FW + b], f01 = F[a * FW + b + 1];
            const float f10 = F[(a + 1) * FW + b], f11 = F[(a + 1) * FW + b + 1];
            if (a < QXH) {
                const int e = RX0 - 1 + b, j = RY0 - 1 + a;
                float q = 0.f, T = 0.f, w = 0.f;
                if (e >= 0 && e <= nx && j >= 0 && j < ny)
                    edge_eval(mode, eps2, inv_s2, f10, f11, F[(a + 2) * FW + b], F[(a + 2) * FW + b + 1],
                              f00, f01, Wp + (a + 1) * FW + b, 1, &q, &T, &w);
                QX[a * QXW + b] = q; TX[a * QXW + b] = T; WX[a * QXW + b] = w;
            }
            if (b < QYW) {
                const int e = RY0 - 1 + a, i = RX0 - 1 + b;
                float q = 0.f, T = 0.f, w = 0.f;
                if (e >= 0 && e <= ny && i >= 0 && i < nx)
                    edge_eval(mode, eps2, inv_s2, f01, f11, F[a * FW + b + 2], F[(a + 1) * FW + b + 2],
                              f00, f10, Wp + a * FW + b + 1, FW, &q, &T, &w);
                QY[a * QYW + b] = q; TY[a * QYW + b] = T; WY[a * QYW + b] = w;
            }
        }
        __syncthreads();

        // phase 3: g on the g region; owned values to the exchange image of this iteration
        float *gx = (it & 1) ? S.gb : S.ga;
        for (int idx = tid; idx < VH * VW; idx += NT) {
            const int yy = idx / VW, xx = idx - yy * VW;
            const int i = RX0 - 1 + xx, j = RY0 - 1 + yy;
            float g = 0.0f;
            if (i >= 0 && i < nx && j >= 0 && j < ny) {
                float d;
                g = grad_value(lam, F[(yy + 1) * FW + xx + 1], V[idx], QX[yy * QXW + xx],
                               QX[yy * QXW + xx + 1], QY[yy * QYW + xx], QY[(yy + 1) * QYW + xx], &d);
                if (xx >= 1 && xx <= RW && yy >= 1 && yy <= RH) gx[j * nx + i] = g;
            }
            G[(yy + 1) * FW + xx + 1] = g;
        }
        __syncthreads();

        // phase 4: the fidelity and energy sums and the first K1 trials
        tile_phase(0, K1, true, (it == pa.n_gd - 1) ? S.wout : nullptr);
        unsigned long long *set = acc_slice + (size_t)(ab % kP2Sets) * kP2SetWords;

        // grid barrier: every block's accumulations and exchange values are visible after it
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            red_release_add_gpu(S.p2bar, 1u);
        }
        // while the barrier is pending: the next iteration's trial steps for every outcome
        // (accepted trial c, or c = K: a failed search), lane c K + m of warp 1
        if (kCand && (tid >> 5) == 1 && K > 1) {
            const int lane = tid & 31;
            if (lane < (K + 1) * K) {
                const int c = lane / K, m = lane - c * K;
                const double tp = (c < K) ? s_td[c] : s_td[K - 1] * P->armijo_shrink / P->armijo_grow;
                const double tmax = P->t_max > 0.0 ? P->t_max : 1.0 / P->lambda;
                double t = fmin(P->armijo_grow * tp, tmax);
                for (int q = 0; q < m; ++q) t *= P->armijo_shrink;
                cand_f[lane] = (float)t;
                cand_d[lane] = (double)(float)t;
            }
        }
        // lane 0 of the kPollers polling warps; the first to see every arrival tells the
        // others through s_seen
        const int bnum = 3 + ab;
        if ((tid & 31) == 0 && (tid >> 5) < kPollers) {
            const unsigned int need = base + (unsigned int)(bnum + 1) * per_bar;
            if (!p2_wait(S.p2bar, need, pa.wait_cycles, &s_seen[bnum & 1])) s_abort = 1;
            __threadfence();
        }
        if (tid == 0) s_seen[(bnum + 1) & 1] = 0;        // re-armed for the next barrier
        __syncthreads();
        if (s_abort) {
            if (tid == 0) S.sc[SC_TIMEOUT] = 1.0;
            return;
        }
        ++ab;
        if (it == 0)      // every block has read the sigma histograms: zero them for the next launch
            for (int w = local * NT + tid; w < kP2HistWords; w += nblk * NT) S.p2hist[w] = 0u;

        // ring 2 of g: the neighbours' exchange values of this iteration (loads issued before
        // the exact read, stored after it)
        float ring_g = 0.0f;
        int ring_at = -1;
        if (tid < kRing) {
            int r, c;
            if (tid < FW) { r = 0; c = tid; }
            else if (tid < 2 * FW) { r = FH - 1; c = tid - FW; }
            else { const int k = tid - 2 * FW; r = 1 + (k >> 1); c = (k & 1) ? FW - 1 : 0; }
            const int i = RX0 - 2 + c, j = RY0 - 2 + r;
            ring_at = r * FW + c;
            if (i >= 0 && i < nx && j >= 0 && j < ny) ring_g = __ldcg(gx + (j * nx + i));
        }
        // the exact totals of this iteration (read, not cleared: every block reads them)
        acc_read<NV, NT, false, kP2Copies>(set, tot);
        __syncthreads();
        // the decision over the first K1 trials; it is final unless none of them passes
        // and trials are left
        if (tid < 32) {
            const GdDecision r = gd_decide(tot, s_td, K1, P, s_misc[0]);
            const bool more = P->step_rule != EPTV_STEP_FIXED && !r.accepted && K1 < K;
            if (tid == 0) s_more = more;
            if (!more) take_decision(r, it);
        }
        __syncthreads();
        // ring 2 is not read by the tile sums (they use g on the region + 1 only)
        if (ring_at >= 0) G[ring_at] = ring_g;
        if (s_more) {
            // the trials K1 .. K - 1 (f, g and the edge terms are unchanged), behind one
            // more barrier
            for (int w = tid; w < NV * kAccStride; w += NT) sacc[w] = 0ull;
            zero_next_set();
            __syncthreads();
            tile_phase(K1, K - K1, false, nullptr);
            unsigned long long *set2 = acc_slice + (size_t)(ab % kP2Sets) * kP2SetWords;
            if (!grid_sync(3 + ab)) {
                if (tid == 0) S.sc[SC_TIMEOUT] = 1.0;
                return;
            }
            ++ab;
            acc_read<NV, NT, false, kP2Copies>(set2, s_tot2);
            __syncthreads();
            if (tid < 32) {
                // the totals of all K trials, then the decision one evaluation of every
                // trial takes
                if (tid < K - K1) tot[4 + K1 + tid] = s_tot2[4 + tid];
                __syncwarp();
                take_decision(gd_decide(tot, s_td, K, P, s_misc[0]), it);
            }
            __syncthreads();
        }
        if (kCand && K > 1 && tid < K && P->step_rule != EPTV_STEP_FIXED) {
            const int c = (int)s_misc[2];
            s_t[tid] = cand_f[c * K + tid];
            s_td[tid] = cand_d[c * K + tid];
        }
        __syncthreads();
        const float tap = (float)s_misc[1];
        if (tap != 0.0f) {
            for (int idx = tid; idx < FH * FW; idx += NT) {
                const int r = idx / FW, c = idx - r * FW;
                const int i = RX0 - 2 + c, j = RY0 - 2 + r;
                if (i >= 0 && i < nx && j >= 0 && j < ny) F[idx] = fmaf(-tap, G[idx], F[idx]);
            }
        }
        __syncthreads();
    }

    // step 3: f = max(f, 0) on the owned pixels -> u (or the caller's output) and u^T
    float *out = pa.out ? pa.out : S.u;
    for (int idx = tid; idx < RH * RW; idx += NT) {
        const int r = idx / RW, c = idx - r * RW;
        const int i = RX0 + c, j = RY0 + r;
        if (i < nx && j < ny) out[j * nx + i] = fmaxf(F[(r + 2) * FW + c + 2], 0.0f);
    }
    if (S.uT && !pa.out) {
        for (int idx = tid; idx < RH * RW; idx += NT) {
            const int c = idx / RH, r = idx - c * RH;    // consecutive threads: consecutive rows
            const int i = RX0 + c, j = RY0 + r;
            if (i < nx && j < ny) S.uT[(size_t)i * ny + j] = fmaxf(F[(r + 2) * FW + c + 2], 0.0f);
        }
    }
    if (blockIdx.x == 0 && tid == 0)       // every block has passed the last barrier
        S.p2bar[1] = base + (unsigned int)(3 + ab) * per_bar;
    if (local == 0 && tid == 0) {
        double *sc = S.sc;
        sc[SC_E_FIRST] = rec.e_first;
        sc[SC_TSTEP] = rec.t_step;
        sc[SC_E_LAST] = rec.e_last;
        if (P->step_rule == EPTV_STEP_FIXED) {
            sc[SC_NACC_P2] += (double)pa.n_gd;
        } else {
            sc[SC_TPREV] = rec.t_prev;
            sc[SC_NACC_P2] += (double)rec.nacc;
            sc[SC_NFAIL] += (double)rec.nfail;
            sc[SC_NFAIL_P2] += (double)rec.nfail;
        }
        if (rec.bad) sc[SC_NONFINITE] = 1.0;
        sc[SC_OUTER] += 1.0;
    }
}

// ------------------------------------------------------------------ host side

namespace {

struct P2Kernel {
    const void *fn;
    int rtx, rty, kt, nt;
    size_t smem;
};

template <int RTX, int RTY, int KT>
P2Kernel p2_kernel() {
    using Sh = P2Shape<RTX, RTY, KT>;
    return P2Kernel{(const void *)&k4p_descent<RTX, RTY, KT>, RTX, RTY, KT, Sh::NT, Sh::SMEM};
}

P2Kernel p2_lookup(int rtx, int rty, int kt) {
#define EPTV_P2_CASE(X, Y)                                                 \
    if (rtx == X && rty == Y) {                                            \
        if (kt == 1) return p2_kernel<X, Y, 1>();                          \
        if (kt == 4) return p2_kernel<X, Y, 4>();                          \
        return p2_kernel<X, Y, 8>();                                       \
    }
    EPTV_P2_CASE(2, 4)
    EPTV_P2_CASE(1, 4)
    EPTV_P2_CASE(1, 2)
    EPTV_P2_CASE(1, 1)
#undef EPTV_P2_CASE
    return P2Kernel{nullptr, 0, 0, 0, 0, 0};
}

int kt_of(int n_trials) {
    if (n_trials <= 1) return 1;
    if (n_trials <= 4) return 4;
    if (n_trials <= 8) return 8;
    return 0;
}

}  // namespace

int p2_plan(Batch &B, int n_trials, int n_gd, P2Plan *plan) {
    plan->ok = 0;
    const int kt = kt_of(n_trials);
    if (!kt || n_gd < 1 || n_gd > (1 << 20) || B.p2_disabled || B.p2_forbid) return 0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        return 0;
    }
    static const int shapes[4][2] = {{2, 4}, {1, 4}, {1, 2}, {1, 1}};
    long long best_cost = -1;
    for (const auto &sh : shapes) {
        const P2Kernel k = p2_lookup(sh[0], sh[1], kt);
        if (!k.fn) continue;
        if (cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k.fn, k.nt, k.smem) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            continue;
        }
        long long regions = 0;
        for (const SliceDev &s : B.h_sd) {
            const int tx = (s.nx + kTileW - 1) / kTileW, ty = (s.ny + kGdTileRows - 1) / kGdTileRows;
            regions += (long long)((tx + sh[0] - 1) / sh[0]) * ((ty + sh[1] - 1) / sh[1]);
        }
        if (regions > (long long)occ * sms) continue;
        // the most tiles one SM works through per GD iteration
        const long long cost = (long long)sh[0] * sh[1] * ((regions + sms - 1) / sms);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            plan->ok = 1;
            plan->rtx = sh[0];
            plan->rty = sh[1];
            plan->kt = kt;
            plan->nt = k.nt;
            plan->smem = k.smem;
            plan->blocks = (int)regions;
        }
    }
    return 0;
}

// Start offsets of the regions of each slice for a region shape (host array, n + 1 entries).
void p2_region_starts(const Batch &B, int rtx, int rty, std::vector<int> &starts) {
    starts.assign(B.n + 1, 0);
    int acc = 0;
    for (int i = 0; i < B.n; ++i) {
        const SliceDev &s = B.h_sd[i];
        const int tx = (s.nx + kTileW - 1) / kTileW, ty = (s.ny + kGdTileRows - 1) / kGdTileRows;
        starts[i] = acc;
        acc += ((tx + rtx - 1) / rtx) * ((ty + rty - 1) / rty);
    }
    starts[B.n] = acc;
}

cudaError_t launch_p2(const Batch &B, const P2Plan &plan, const P2Args &pa, cudaStream_t st) {
    const P2Kernel k = p2_lookup(plan.rtx, plan.rty, plan.kt);
    if (!k.fn) return cudaErrorInvalidValue;
    ++g_launch_count;
    TileMap map{B.d_p2start, B.n};
    const SliceDev *sd = B.d_sd;
    const ParamsDev *pp = B.d_params;
    P2Args a = pa;
    void *args[] = {(void *)&sd, (void *)&map, (void *)&pp, (void *)&a};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.blocks);
    cfg.blockDim = dim3(k.nt);
    cfg.dynamicSmemBytes = k.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, k.fn, args);
}

}  // namespace eptv
