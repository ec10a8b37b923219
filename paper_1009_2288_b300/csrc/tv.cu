// K4/K5: the (P2) step -- edge-preserving TV descent (Sec. 2.2, Eqs. 5, 9, A2, A3).
//
// K5 sigma: the ceil(q n)-th smallest half-edge magnitude T of v (Sec. 2.1), found
//    exactly by a 3-pass radix selection over the FP32 bit patterns (12 + 12 + 8 bits) of
//    T^2: sqrtf is monotone, so sqrtf of the k-th smallest T^2 is the k-th smallest
//    sqrtf(T^2) = T, bit for bit, and one square root replaces one per half-edge.  Pass 0
//    computes every T^2 (fused stencil) and histograms the top 12 bits; each pass's last
//    block scans the histogram and narrows the prefix.
// K4 one gradient-descent iteration, fused: apply the previous step f = f' - t' g'
//    on the fly, stage f (tile + 2-pixel halo) and v in shared memory, compute T, the
//    weights w = exp(-T^2/sigma^2) and w D / T at every half-edge, the gradient
//    g = lambda (f - v) + dJ/df (Eq. A2) on the tile + 1 halo, and for all Armijo trial
//    steps t_m at once the energy change of f - t_m g with the weights frozen:
//      fidelity: lambda (-t <g, f-v> + t^2/2 |g|^2)  (two global sums),
//      TV:       sum_e w_e (T_e(f - t g) - T_e(f)), each term in the cancellation-free
//                form t (t b_e - 2 a_e) / (T'_e + T_e).
//    The last block takes the Armijo decision in FP64 and stores the step; the next
//    kernel applies it.  One launch per GD iteration, no host round trip.
// K4u apply the last step, clamp f >= 0 (step 3 of the algorithm), write f and f^T.
#include <atomic>

#include "eptv_internal.cuh"
#include "kernels.cuh"
#include "tv_stencil.cuh"

namespace eptv {

// ------------------------------------------------------------------ half-edge stencil

__device__ __forceinline__ float img_at(const float *f, int nx, int ny, int i, int j) {
    return (i >= 0 && i < nx && j >= 0 && j < ny) ? __ldg(f + (size_t)j * nx + i) : 0.0f;
}

// T^2 of half-edge e of the slice (x-edges first: e = j (nx+1) + i, between (i-1, j) and
// (i, j); then y-edges: X + j nx + i, between (i, j-1) and (i, j)).
__device__ __forceinline__ float half_edge_T2(const float *f, int nx, int ny, float eps2, int e) {
    const int X = (nx + 1) * ny;
    float D;
    if (e < X) {
        const int j = e / (nx + 1), i = e - j * (nx + 1);
        return edge_T2(eps2, img_at(f, nx, ny, i - 1, j), img_at(f, nx, ny, i, j),
                       img_at(f, nx, ny, i - 1, j + 1), img_at(f, nx, ny, i, j + 1),
                       img_at(f, nx, ny, i - 1, j - 1), img_at(f, nx, ny, i, j - 1), &D);
    }
    e -= X;
    const int j = e / nx, i = e - j * nx;
    return edge_T2(eps2, img_at(f, nx, ny, i, j - 1), img_at(f, nx, ny, i, j),
                   img_at(f, nx, ny, i + 1, j - 1), img_at(f, nx, ny, i + 1, j),
                   img_at(f, nx, ny, i - 1, j - 1), img_at(f, nx, ny, i - 1, j), &D);
}

// ------------------------------------------------------------------ radix selection


struct SelCtx {
    const float *vals;
    long long n;
    double *sc;
    unsigned int *hist;
    unsigned int *counter;
    int n_blocks, b0;
};


// Last block (256 threads): find the bucket holding the remaining rank and narrow the
// prefix.  The histogram is read with independent loads (16 per thread), the per-thread
// bucket groups are prefix-summed across the block, and the thread whose group holds
// the rank searches its own buckets.  Returns the selected key after pass 2 (in all
// threads), else 0.  Re-arms the histogram (zero) for the next pass.
__device__ unsigned int sel_scan(unsigned int *hist, double *sc, int pass, long long rank0,
                                 unsigned int *s_cnt /* 256 */, long long *s_res) {
    const int nbins = (pass == 2) ? 256 : kHistBins;
    const int per = nbins / 256;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    unsigned int v[16];
    unsigned long long local = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = (q < per) ? __ldcg(hist + t * per + q) : 0u;
#pragma unroll
    for (int q = 0; q < 16; ++q) local += v[q];
    // inclusive scan of the 256 group counts: warp shuffles, then warp totals
    unsigned long long inc = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    __shared__ unsigned long long s_warp[8];
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    unsigned long long before = 0;
    for (int i = 0; i < w; ++i) before += s_warp[i];
    inc += before;
    const unsigned long long exc = inc - local;
    const long long rank = (pass == 0) ? rank0 : (long long)sc[SC_SEL_RANK];
    const unsigned int prefix = (pass == 0) ? 0u : (unsigned int)sc[SC_SEL_PREFIX];
    __syncthreads();
    if ((long long)exc < rank && rank <= (long long)inc) {
        unsigned long long cum = exc;
        int b = t * per;
        for (int q = 0; q < per; ++q, ++b) {
            if ((long long)(cum + v[q]) >= rank) break;
            cum += v[q];
        }
        unsigned int pre;
        if (pass == 0) pre = (unsigned int)b;
        else if (pass == 1) pre = (prefix << 12) | (unsigned int)b;
        else pre = (prefix << 8) | (unsigned int)b;
        sc[SC_SEL_RANK] = (double)(rank - (long long)cum);
        sc[SC_SEL_PREFIX] = (double)pre;
        *s_res = (long long)pre;
    }
    (void)s_cnt;
    __syncthreads();
    for (int q = 0; q < per; ++q) hist[t * per + q] = 0u;     // re-arm for the next pass
    return (pass == 2) ? (unsigned int)(*s_res) : 0u;
}

// Pass 0 of sigma: T^2 of every half-edge of v -> scratch, histogram of the top 12 bits.
__global__ void __launch_bounds__(256)
k5_sigma_edges(const SliceDev *__restrict__ sls, TileMap map, const ParamsDev *__restrict__ P,
               const float *v_override, unsigned int *__restrict__ hist_all)
{
    pdl_wait();
    __shared__ unsigned int sh[kHistBins];
    __shared__ unsigned int s_cnt[256];
    __shared__ long long s_res;
    __shared__ int last_flag;
    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    for (int b = threadIdx.x; b < kHistBins; b += 256) sh[b] = 0u;
    __syncthreads();
    const float *v = v_override ? v_override : S.u;
    const float eps2 = (float)(P->eps * P->eps);
    const int e0 = local * 2048;
    float Tv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {               // all stencil loads before any atomic
        const int e = e0 + q * 256 + threadIdx.x;
        Tv[q] = (e < S.n_edges) ? half_edge_T2(v, S.nx, S.ny, eps2, e) : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int e = e0 + q * 256 + threadIdx.x;
        if (e < S.n_edges) {
            const float T = Tv[q];
            S.tv_scr[e] = T;
            if (!isfinite(T)) S.sc[SC_NONFINITE] = 1.0;
            sel_hist_add(sh, sel_key(T), 0, 0u);
        }
    }
    __syncthreads();
    unsigned int *hist = hist_all + (size_t)si * kHistBins;
    for (int b = threadIdx.x; b < kHistBins; b += 256) {
        const unsigned int c = sh[b];
        if (c) atomicAdd(hist + b, c);
    }
    const int b0 = __ldg(map.start + si);
    const int nblk = __ldg(map.start + si + 1) - b0;
    if (!last_block_of_slice(S.ctr, nblk, &last_flag)) return;
    sel_scan(hist, S.sc, 0, S.sel_rank, s_cnt, &s_res);
}

// Passes 1, 2 of sigma (on the scratch T array), or passes 0-2 of a generic selection.
__global__ void __launch_bounds__(256)
k5_radix_pass(const SliceDev *__restrict__ sls, TileMap map, const ParamsDev *__restrict__ P,
              int pass, unsigned int *__restrict__ hist_all, const float *vals_override, long long n_override, long long rank_override,
              float *out_override)
{
    pdl_wait();
    __shared__ unsigned int sh[kHistBins];
    __shared__ unsigned int s_cnt[256];
    __shared__ long long s_res;
    __shared__ int last_flag;
    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const float *vals = vals_override ? vals_override : S.tv_scr;
    const long long n = vals_override ? n_override : (long long)S.n_edges;
    const int nbins = (pass == 2) ? 256 : kHistBins;
    for (int b = threadIdx.x; b < nbins; b += 256) sh[b] = 0u;
    __syncthreads();
    const unsigned int prefix = (pass == 0) ? 0u : (unsigned int)S.sc[SC_SEL_PREFIX];
    const long long e0 = (long long)local * 2048;
    float xv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {               // issue the 8 loads before any atomic
        const long long e = e0 + q * 256 + threadIdx.x;
        xv[q] = 0.0f;
        if (e < n) xv[q] = __ldg(vals + e);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const long long e = e0 + q * 256 + threadIdx.x;
        if (e < n) sel_hist_add(sh, sel_key(xv[q]), pass, prefix);
    }
    __syncthreads();
    unsigned int *hist = hist_all + (size_t)si * kHistBins;
    for (int b = threadIdx.x; b < nbins; b += 256) {
        const unsigned int c = sh[b];
        if (c) atomicAdd(hist + b, c);
    }
    const int b0 = __ldg(map.start + si);
    const int nblk = __ldg(map.start + si + 1) - b0;
    if (!last_block_of_slice(S.ctr, nblk, &last_flag)) return;
    const long long rank0 = vals_override ? rank_override : S.sel_rank;
    const unsigned int key = sel_scan(hist, S.sc, pass, rank0, s_cnt, &s_res);
    if (pass == 2 && threadIdx.x == 0) {
        const float val = __uint_as_float(key);
        if (out_override) {
            *out_override = val;
            S.sc[SC_NORM] = (double)val;
        } else {
            S.sc[SC_SIGMA] = fmax((double)sqrtf(val), P->sigma_floor);    // val: the k-th smallest T^2
            if (S.log) {
                const int k = (int)S.sc[SC_OUTER];
                if (k >= 0 && k < S.log_outer)
                    S.log[(size_t)S.log_outer * S.log_gd + k] = S.sc[SC_SIGMA];
            }
        }
    }
}

// ------------------------------------------------------------------ fused GD iteration

constexpr int kGdThreads = 128;                     // threads per 32 x 8 tile
constexpr int kGdTileH = kGdTileRows;                // tile rows of the GD kernel
constexpr int FW = kTileW + 4, FH = kGdTileH + 4;    // f region (2-pixel halo)
constexpr int GW = kTileW + 2, GH = kGdTileH + 2;    // g region (1-pixel halo)
constexpr int QXW = kTileW + 3, QXH = GH;            // x-edges around the g region
constexpr int QYW = GW, QYH = kGdTileH + 3;          // y-edges around the g region



// WIDE: the launch has more tiles than 8 blocks per SM hold at once (a batch), and 12
// resident blocks of 40 registers hide more of each tile's load -> stencil -> reduction
// latency chain than 8 blocks of 64 registers; a single slice fits in one wave of 8, where
// the extra spills only cost.
template <int KT, bool WIDE>
__global__ void __launch_bounds__(kGdThreads, WIDE ? 12 : 1)
k4_gd(const SliceDev *__restrict__ sls, TileMap map, const ParamsDev *__restrict__ P, GdArgs ga,
      int iter, double *__restrict__ partials)
{
    pdl_wait();
    __shared__ float F[FH][FW];
    __shared__ float W[FH][FW];          // prior map (PRIOR mode only)
    __shared__ float V[GH][GW];
    __shared__ float G[GH][GW];
    __shared__ float QX[QXH][QXW], TXs[QXH][QXW], WX[QXH][QXW];
    __shared__ float QY[QYH][QYW], TYs[QYH][QYW], WY[QYH][QYW];
    __shared__ float s_t[KT];
    __shared__ double s_td[KT];
    __shared__ unsigned long long sacc[(KT + 4) * kAccStride];
    __shared__ float s_tapply;
    __shared__ int last_flag;

    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const int nx = S.nx, ny = S.ny;
    const int tiles_x = (nx + kTileW - 1) / kTileW;
    const int tyb = local / tiles_x, txb = local - tyb * tiles_x;
    const int X0 = txb * kTileW, Y0 = tyb * kGdTileH;
    const int tid = threadIdx.x;
    const int K = ga.n_trials;
    const float eps2 = (float)(P->eps * P->eps);
    const float lam = (float)P->lambda;

    // buffers of this iteration
    const int par = iter & 1;
    const float *fprev = ga.fprev ? ga.fprev : (ga.first ? (ga.v ? ga.v : S.u) : (par ? S.fa : S.fb));
    const float *gprev = ga.gprev ? ga.gprev : (par ? S.ga : S.gb);
    const float *vv = ga.v ? ga.v : S.u;
    float *fout = ga.fout ? ga.fout : (par ? S.fb : S.fa);
    float *gout = ga.gout ? ga.gout : (par ? S.gb : S.ga);

    int mode = P->weights_mode;
    if (mode == EPTV_WEIGHTS_PRIOR) {
        mode = (S.wprior && S.sc[SC_OUTER] < (double)P->prior_iters) ? EPTV_WEIGHTS_PRIOR
                                                                      : EPTV_WEIGHTS_EPTV;
    }
    const float sig = (float)S.sc[SC_SIGMA];
    const float inv_s2 = 1.0f / (sig * sig);

    for (int w = tid; w < (KT + 4) * kAccStride; w += kGdThreads) sacc[w] = 0ull;
    (void)partials;
    if (tid == 0) s_tapply = ga.first ? 0.0f : (float)S.sc[SC_TSTEP];
    if (tid == 0 && K > 0) trial_steps(P, S.sc[SC_TPREV], K, s_t, s_td);
    __syncthreads();
    const float tap = s_tapply;

    // phase 1: f on the tile + 2 halo (previous step applied), v on tile + 1 halo
    for (int idx = tid; idx < FH * FW; idx += kGdThreads) {
        const int yy = idx / FW, xx = idx - yy * FW;
        const int i = X0 - 2 + xx, j = Y0 - 2 + yy;
        float fv = 0.0f;
        if (i >= 0 && i < nx && j >= 0 && j < ny) {
            const int p = j * nx + i;                   // images hold < 2^31 pixels
            fv = __ldg(fprev + p);
            if (tap != 0.0f) fv = fmaf(-tap, __ldg(gprev + p), fv);
        }
        F[yy][xx] = fv;
        if (mode == EPTV_WEIGHTS_PRIOR) {
            const int ci = min(max(i, 0), nx - 1), cj = min(max(j, 0), ny - 1);
            W[yy][xx] = __ldg(S.wprior + (size_t)cj * nx + ci);
        }
    }
    for (int idx = tid; idx < GH * GW; idx += kGdThreads) {
        const int yy = idx / GW, xx = idx - yy * GW;
        const int i = X0 - 1 + xx, j = Y0 - 1 + yy;
        float vx = 0.0f;
        if (i >= 0 && i < nx && j >= 0 && j < ny) vx = __ldg(vv + (j * nx + i));
        V[yy][xx] = vx;
    }
    __syncthreads();

    // phase 2: half-edges around the g region.  One pass over the union of the x-edge
    // region (QXH x QXW) and the y-edge region (QYH x QYW): position (a, b) holds x-edge
    // (a, b) and y-edge (a, b), which share four of their six F values.
    for (int idx = tid; idx < QYH * QXW; idx += kGdThreads) {
        const int a = idx / QXW, b = idx - a * QXW;
        const float f00 = F[a][b], f01 = F[a][b + 1], f10 = F[a + 1][b], f11 = F[a + 1][b + 1];
        if (a < QXH) {
            // x-edge: between (e-1, j) and (e, j); F rows a .. a+2, columns b, b+1
            const int e = X0 - 1 + b, j = Y0 - 1 + a;
            float q = 0.f, T = 0.f, w = 0.f;
            if (e >= 0 && e <= nx && j >= 0 && j < ny)
                edge_eval(mode, eps2, inv_s2, f10, f11, F[a + 2][b], F[a + 2][b + 1], f00, f01,
                          &W[a + 1][b], 1, &q, &T, &w);
            QX[a][b] = q; TXs[a][b] = T; WX[a][b] = w;
        }
        if (b < QYW) {
            // y-edge: between (i, e-1) and (i, e); F rows a, a+1, columns b .. b+2
            const int e = Y0 - 1 + a, i = X0 - 1 + b;
            float q = 0.f, T = 0.f, w = 0.f;
            if (e >= 0 && e <= ny && i >= 0 && i < nx)
                edge_eval(mode, eps2, inv_s2, f01, f11, F[a][b + 2], F[a + 1][b + 2], f00, f10,
                          &W[a][b + 1], FW, &q, &T, &w);
            QY[a][b] = q; TYs[a][b] = T; WY[a][b] = w;
        }
    }
    __syncthreads();

    // phase 3: g = lambda (f - v) + dJ/df on the g region (Eq. 9, A2)
    for (int idx = tid; idx < GH * GW; idx += kGdThreads) {
        const int yy = idx / GW, xx = idx - yy * GW;
        const int i = X0 - 1 + xx, j = Y0 - 1 + yy;
        float g = 0.0f;
        if (i >= 0 && i < nx && j >= 0 && j < ny) {
            const float f = F[yy + 1][xx + 1];
            float d;
            g = grad_value(lam, f, V[yy][xx], QX[yy][xx], QX[yy][xx + 1], QY[yy][xx], QY[yy + 1][xx], &d);
            if (xx >= 1 && xx <= kTileW && yy >= 1 && yy <= kGdTileH) {
                const int p = j * nx + i;
                gout[p] = g;
                if (ga.write_f) fout[p] = f;
            }
        }
        G[yy][xx] = g;
    }
    __syncthreads();

    // phase 4: the tile's sums -- fidelity, energy and trial energy changes of its owned
    // half-edges (the same per-thread assignment as the persistent kernel)
    constexpr int NV = KT + 4;
    float vals[NV];
    float sA = 0.f, sB = 0.f, sF = 0.f, sJ = 0.f;
    float dJ[KT];
#pragma unroll
    for (int m = 0; m < KT; ++m) dJ[m] = 0.0f;
    tile_sums<KT>(tid, X0, Y0, nx, ny, &F[0][0], FW, &G[0][0], GW, &V[0][0], GW, &TXs[0][0], &WX[0][0],
                  QXW, &TYs[0][0], &WY[0][0], QYW, K, s_t, eps2, (ga.last && S.wout) ? S.wout : nullptr,
                  &sA, &sB, &sF, &sJ, dJ);

    // phase 5: each warp's sums added exactly into the block's accumulators, the block's
    // words into the slice's (copy local % kAccCopies); the last block decides the step
    vals[0] = sA; vals[1] = sB; vals[2] = sF; vals[3] = sJ;
#pragma unroll
    for (int m = 0; m < KT; ++m) vals[4 + m] = dJ[m];
    warp_acc<NV>(vals, sacc);
    __syncthreads();
    acc_push<NV, kGdThreads>(sacc, S.acc, local % kAccCopies);
    const int b0 = __ldg(map.start + si);
    const int nblk = __ldg(map.start + si + 1) - b0;
    __shared__ double tot[NV];
    if (!last_block_of_slice(S.ctr, nblk, &last_flag)) return;
    acc_read<NV, kGdThreads>(S.acc, tot);
    __syncthreads();
    if (tid < 32) {
        if (ga.energy_only_fin) {
            if (tid == 0) {
                const double E0 = 0.5 * P->lambda * tot[2] + tot[3];
                S.sc[SC_E_FIRST] = E0;
                S.sc[SC_NORM2] = tot[1];
                if (!isfinite(E0) || !isfinite(tot[0]) || !isfinite(tot[1])) S.sc[SC_NONFINITE] = 1.0;
            }
        } else {
            const GdDecision r = gd_decide(tot, s_td, K, P, 0.0);
            if (tid == 0) gd_record(S, P, r, ga.first != 0, iter);
        }
    }
}

// K4u: f = max(f' - t g', 0) -> u and u^T; advances the outer-iteration counter.
__global__ void __launch_bounds__(256)
k4_finish(const SliceDev *__restrict__ sls, TileMap map, int n_gd, const float *f0_override,
          float *out_override)
{
    pdl_wait();
    __shared__ float tile[32][33];
    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const int nx = S.nx, ny = S.ny;
    const int tiles_x = (nx + 31) >> 5;
    const int tyb = local / tiles_x, txb = local - tyb * tiles_x;
    const int par = (n_gd - 1) & 1;
    const float *fp = (n_gd == 0) ? (f0_override ? f0_override : S.u) : (par ? S.fb : S.fa);
    const float *gp = par ? S.gb : S.ga;
    const float t = (n_gd == 0) ? 0.0f : (float)S.sc[SC_TSTEP];
    float *out = out_override ? out_override : S.u;
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    const int i = txb * 32 + lx;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int jj = ly + 8 * q, j = tyb * 32 + jj;
        if (i < nx && j < ny) {
            const size_t p = (size_t)j * nx + i;
            float f = fp[p];
            if (t != 0.0f) f = fmaf(-t, gp[p], f);
            f = fmaxf(f, 0.0f);
            out[p] = f;
            tile[jj][lx] = f;
        }
    }
    if (local == 0 && threadIdx.x == 0) S.sc[SC_OUTER] += 1.0;
    if (S.uT == nullptr || out_override) return;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int ii = ly + 8 * q;
        const int gi = txb * 32 + ii, gj = tyb * 32 + lx;
        if (gi < nx && gj < ny) S.uT[(size_t)gi * ny + gj] = tile[lx][ii];
    }
}

// --------------------------------------------------------------------- launchers

void launch_sigma(const Batch &B, const float *v_override, cudaStream_t st) {
    ++g_launch_count;
    launch_pdl(k5_sigma_edges, B.blocks(FAM_EDGE), 256, 0, st, B.d_sd, B.map(FAM_EDGE), B.d_params,
               v_override, B.d_hist);
    for (int pass = 1; pass <= 2; ++pass, ++g_launch_count)
        launch_pdl(k5_radix_pass, B.blocks(FAM_EDGE), 256, 0, st, B.d_sd, B.map(FAM_EDGE), B.d_params, pass,
                   B.d_hist, (const float *)nullptr, 0ll, 0ll, (float *)nullptr);
}

void launch_select_generic(const Batch &B, const TileMap &m, int nblk, const float *vals,
                           long long n, long long k, float *out, cudaStream_t st) {
    for (int pass = 0; pass <= 2; ++pass, ++g_launch_count)
        launch_pdl(k5_radix_pass, nblk, 256, 0, st, B.d_sd, m, B.d_params, pass, B.d_hist, vals, n, k, out);
}

// SMs of the current device (queried once per device; host threads may race to fill the
// cache, all with the same value)
static int sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return 148; }
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 148;
        }
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

template <int KT>
static void launch_k4(int nb, bool wide, const Batch &B, const TileMap &m, const GdArgs &ga, int iter,
                      cudaStream_t st) {
    if (wide) launch_pdl(k4_gd<KT, true>, nb, kGdThreads, 0, st, B.d_sd, m, B.d_params, ga, iter, B.d_partials);
    else launch_pdl(k4_gd<KT, false>, nb, kGdThreads, 0, st, B.d_sd, m, B.d_params, ga, iter, B.d_partials);
}

void launch_gd_iter(const Batch &B, const GdArgs &ga, int iter, cudaStream_t st) {
    ++g_launch_count;
    const int nb = B.blocks(FAM_TV);
    const TileMap m = B.map(FAM_TV);
    const bool wide = nb > 8 * sm_count();
    if (ga.n_trials <= 1) launch_k4<1>(nb, wide, B, m, ga, iter, st);
    else if (ga.n_trials <= 4) launch_k4<4>(nb, wide, B, m, ga, iter, st);
    else if (ga.n_trials <= 8) launch_k4<8>(nb, wide, B, m, ga, iter, st);
    else launch_k4<16>(nb, wide, B, m, ga, iter, st);
}

void launch_gd_finish(const Batch &B, int n_gd, const float *f0_override, float *out_override,
                      cudaStream_t st) {
    ++g_launch_count;
    launch_pdl(k4_finish, B.blocks(FAM_IMG), 256, 0, st, B.d_sd, B.map(FAM_IMG), n_gd, f0_override,
               out_override);
}

}  // namespace eptv
