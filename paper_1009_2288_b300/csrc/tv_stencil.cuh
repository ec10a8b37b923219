// Per-edge and per-pixel arithmetic of the (P2) descent step (Eqs. 5, 9, A2, A3), shared
// by the one-launch-per-GD-iteration kernel K4 (tv.cu) and the persistent kernel K4p
// (tv_p2.cu), so that both evaluate every half-edge magnitude, weight, gradient value,
// trial energy change and step decision with the same instruction sequence.
#pragma once

#include "eptv_internal.cuh"

namespace eptv {

// T^2 of the x half-edge between pixels a=(i-1,j) and b=(i,j) given the six values
// around it: a_d, b_d (row j-1), a, b (row j), a_u, b_u (row j+1).  Eq. (A3).
__device__ __forceinline__ float edge_T2(float eps2, float a, float b, float a_u, float b_u,
                                         float a_d, float b_d, float *D) {
    const float d = b - a;
    const float mc = 0.5f * (a + b), mu = 0.5f * (a_u + b_u), md = 0.5f * (a_d + b_d);
    const float cu = mu - mc, cd = mc - md;
    *D = d;
    return eps2 + d * d + 0.5f * cu * cu + 0.5f * cd * cd;
}

// One half-edge (either orientation; the argument order of edge_T2): magnitude T, weight
// w (Eq. 5, 1 for plain TV, or the mean of the prior values wp[0], wp[wstep] of its two
// pixels) and the flux q = w D / T of Eq. (A2).
__device__ __forceinline__ void edge_eval(int mode, float eps2, float inv_s2, float a, float b,
                                          float a_u, float b_u, float a_d, float b_d, const float *wp,
                                          int wstep, float *q, float *T, float *w) {
    float D;
    const float T2 = edge_T2(eps2, a, b, a_u, b_u, a_d, b_d, &D);
    const float rs = rsqrtf(T2);           // T2 >= eps^2 > 0
    *T = T2 * rs;
    float ww;
    if (mode == EPTV_WEIGHTS_EPTV) ww = __expf(-T2 * inv_s2);
    else if (mode == EPTV_WEIGHTS_ONE) ww = 1.0f;
    else ww = 0.5f * (wp[0] + wp[wstep]);   // prior map values of the edge's two pixels
    *w = ww;
    *q = ww * D * rs;
}

// g = lambda (f - v) + dJ/df at one pixel (Eq. 9 with Eq. A2): the fluxes of its left,
// right, lower and upper half-edges.  Returns g and stores d = f - v.
__device__ __forceinline__ float grad_value(float lam, float f, float v, float qxl, float qxr,
                                            float qyl, float qyr, float *d) {
    const float dd = f - v;
    const float div = (qxr - qxl) + (qyr - qyl);
    *d = dd;
    return lam * dd - div;
}

// Energy change of one half-edge along the step -t g, with the weights frozen:
//   T'^2 = T^2 - 2 t a + t^2 b,  a = D dD + 1/2 (c1 dc1 + c2 dc2),  b = dD^2 + 1/2 (dc1^2 + dc2^2)
// (D, c1, c2 of Eq. A3 at f; dD, dc1, dc2 the same differences of g).  Pixel values in the
// orientation of edge_T2: lo / hi the two pixels, lo_u / hi_u the next row (column), lo_d /
// hi_d the previous one; same for g.
__device__ __forceinline__ void edge_ab(float lo, float hi, float lo_u, float hi_u, float lo_d,
                                        float hi_d, float glo, float ghi, float glo_u, float ghi_u,
                                        float glo_d, float ghi_d, float *ae, float *be) {
    const float D = hi - lo;
    const float mc = 0.5f * (lo + hi);
    const float c1 = 0.5f * (lo_u + hi_u) - mc;
    const float c2 = mc - 0.5f * (lo_d + hi_d);
    const float dD = ghi - glo;
    const float gc = 0.5f * (glo + ghi);
    const float dc1 = 0.5f * (glo_u + ghi_u) - gc;
    const float dc2 = gc - 0.5f * (glo_d + ghi_d);
    *ae = D * dD + 0.5f * (c1 * dc1 + c2 * dc2);
    *be = dD * dD + 0.5f * (dc1 * dc1 + dc2 * dc2);
}

// dJ[m] += w (T'(t_m) - T) for the x- and y-edge of one position and every trial step,
// in the cancellation-free form t (t b - 2 a) / (T' + T).  EDGES = 1 / 2 evaluates only the
// x / y term: for a position that owns only that edge the other one has weight 0 and a
// finite change (T' + T >= eps), so it would add an exact zero.
template <int KT, int EDGES = 3>
__device__ __forceinline__ void trial_accum(int K, const float *s_t, float eps2, float Tx, float wx,
                                            float aex, float bex, float Ty, float wy, float aey,
                                            float bey, float (&dJ)[KT]) {
    const float T2x = Tx * Tx, T2y = Ty * Ty;
#pragma unroll
    for (int m = 0; m < KT; ++m) {
        if (m < K) {
            const float t = s_t[m];
            if (EDGES & 1) {
                const float numx = t * fmaf(t, bex, -2.0f * aex);
                const float T2nx = fmaxf(T2x + numx, eps2);   // T'^2 >= eps^2
                const float Tnx = T2nx * rsqrtf(T2nx);
                dJ[m] = fmaf(wx, __fdividef(numx, Tnx + Tx), dJ[m]);
            }
            if (EDGES & 2) {
                const float numy = t * fmaf(t, bey, -2.0f * aey);
                const float T2ny = fmaxf(T2y + numy, eps2);
                const float Tny = T2ny * rsqrtf(T2ny);
                dJ[m] = fmaf(wy, __fdividef(numy, Tny + Ty), dJ[m]);
            }
        }
    }
}

// Trial steps of one GD iteration: t0, t0 s, t0 s^2, ... (repeated products: exact for
// s = 1/2), t0 = min(grow t_prev, t_max) for Armijo, t_fixed for fixed steps.
__device__ __forceinline__ void trial_steps(const ParamsDev *P, double t_prev, int K, float *s_t,
                                            double *s_td) {
    double t;
    if (P->step_rule == EPTV_STEP_FIXED) t = P->t_fixed;
    else {
        const double tmax = P->t_max > 0.0 ? P->t_max : 1.0 / P->lambda;
        t = fmin(P->armijo_grow * t_prev, tmax);
    }
    for (int m = 0; m < K; ++m) {
        s_t[m] = (float)t;
        s_td[m] = (double)(float)t;
        t *= P->armijo_shrink;
    }
}

// Outcome of one GD iteration's step decision.
struct GdDecision {
    double t_step;     // step taken (0 after a failed search)
    double t_prev;     // t_prev for the next search
    double e_last;     // (P2) energy after the step (frozen weights)
    double e0;         // energy at the current iterate
    int accepted;      // 1: a trial passed (or fixed step), 0: failed search
    int index;         // the accepted trial (0 for fixed steps), K after a failed search
    int bad;           // a total or an evaluated trial was not finite
};

// The step decision of one GD iteration from the exact totals tot = {<g, f-v>, |g|^2,
// |f-v|^2, J, dJ_0 .. dJ_{K-1}} (Eq. 9's energy lambda/2 |f-v|^2 + J; Armijo on
// E(f - t g) <= E(f) - c t |g|^2).  Called by all 32 lanes of one warp: trial m is
// evaluated in lane m, and the accepted step is the first trial that passes, as in a
// sequential search.
__device__ __forceinline__ GdDecision gd_decide(const double *tot, const double *s_td, int K,
                                                const ParamsDev *P, double t_prev_in) {
    const int lane = threadIdx.x & 31;
    const double A = tot[0], Bg = tot[1];
    const double lamd = P->lambda;
    GdDecision r;
    r.e0 = 0.5 * lamd * tot[2] + tot[3];
    r.bad = !isfinite(r.e0) || !isfinite(A) || !isfinite(Bg);
    const bool armijo = P->step_rule != EPTV_STEP_FIXED;
    double d = 0.0;
    bool pass = false, nonfinite = false;
    if (armijo && lane < K) {
        const double t = s_td[lane];
        d = lamd * (-t * A + 0.5 * t * t * Bg) + tot[4 + lane];
        nonfinite = !isfinite(d);
        pass = d <= -P->armijo_c * t * Bg;
    }
    const unsigned pass_mask = __ballot_sync(0xffffffffu, pass);
    const unsigned bad_mask = __ballot_sync(0xffffffffu, nonfinite);
    const int acc_m = pass_mask ? __ffs(pass_mask) - 1 : -1;
    const double dE = __shfl_sync(0xffffffffu, d, acc_m >= 0 ? acc_m : 0);
    if (!armijo) {
        const double t = s_td[0];
        r.t_step = t;
        r.t_prev = t_prev_in;
        r.e_last = r.e0 + lamd * (-t * A + 0.5 * t * t * Bg) + tot[4];
        r.accepted = 1;
        r.index = 0;
        return r;
    }
    // trials a sequential search would have evaluated: up to the accepted one
    const unsigned seen = acc_m >= 0 ? ((2u << acc_m) - 1u) : ((1u << K) - 1u);
    if (bad_mask & seen) r.bad = 1;
    if (acc_m >= 0) {
        r.t_step = s_td[acc_m];
        r.t_prev = s_td[acc_m];
        r.e_last = r.e0 + dE;
        r.accepted = 1;
        r.index = acc_m;
    } else {
        r.t_step = 0.0;
        r.t_prev = s_td[K - 1] * P->armijo_shrink / P->armijo_grow;
        r.e_last = r.e0;
        r.accepted = 0;
        r.index = K;
    }
    return r;
}

// Records a decision in the slice's scalars and log (one thread).
__device__ __forceinline__ void gd_record(const SliceDev &S, const ParamsDev *P, const GdDecision &r,
                                          bool first, int iter) {
    double *sc = S.sc;
    if (first) sc[SC_E_FIRST] = r.e0;
    sc[SC_TSTEP] = r.t_step;
    sc[SC_E_LAST] = r.e_last;
    if (P->step_rule == EPTV_STEP_FIXED) {
        sc[SC_NACC_P2] += 1.0;
    } else {
        sc[SC_TPREV] = r.t_prev;
        if (r.accepted) sc[SC_NACC_P2] += 1.0;
        else {
            sc[SC_NFAIL] += 1.0;
            sc[SC_NFAIL_P2] += 1.0;
        }
    }
    if (r.bad) sc[SC_NONFINITE] = 1.0;
    if (S.log) {
        const int k = (int)sc[SC_OUTER];
        if (k >= 0 && k < S.log_outer && iter < S.log_gd) S.log[(size_t)k * S.log_gd + iter] = sc[SC_TSTEP];
    }
}

}  // namespace eptv

namespace eptv {

// One position (a, b) of a 32 x 8 tile (tile_sums below): the fidelity terms of pixel
// (X0 + b, Y0 + a) when it is the tile's, and the energy / trial terms of its left x-edge
// and upper y-edge when the tile owns them (EDGES = 1 / 2: a border position that can own
// only its x- / y-edge).
template <int KT, int EDGES = 3>
__device__ __forceinline__ void tile_position(int a, int b, int X0, int Y0, int nx, int ny,
                                              const float *F, int fs, const float *G, int gs,
                                              const float *V, int vs, const float *TX,
                                              const float *WX, int xs, const float *TY,
                                              const float *WY, int ys, int K, const float *s_t,
                                              float eps2, float *wout, float *sA, float *sB,
                                              float *sF, float *sJ, float (&dJ)[KT]) {
    constexpr int TW = 32, TH = 8;
    const int i = X0 + b, j = Y0 + a;
    if (a < TH && b < TW && i < nx && j < ny) {
        const float g = G[(a + 1) * gs + b + 1];
        const float d = F[(a + 2) * fs + b + 2] - V[(a + 1) * vs + b + 1];
        *sA = fmaf(g, d, *sA);
        *sB = fmaf(g, g, *sB);
        *sF = fmaf(d, d, *sF);
    }
    // x-edge between (i - 1, j) and (i, j); y-edge between (i, j - 1) and (i, j)
    const bool own_x = a < TH && j < ny && i <= nx && (b < TW || i == nx);
    const bool own_y = b < TW && i < nx && j <= ny && (a < TH || j == ny);
    const float Tx = TX[(a + 1) * xs + b + 1], wx = own_x ? WX[(a + 1) * xs + b + 1] : 0.0f;
    const float Ty = TY[(a + 1) * ys + b + 1], wy = own_y ? WY[(a + 1) * ys + b + 1] : 0.0f;
    *sJ = fmaf(wx, Tx, *sJ);
    *sJ = fmaf(wy, Ty, *sJ);
    if (wout) {
        if (own_x) wout[(size_t)j * (nx + 1) + i] = wx;
        if (own_y) wout[(size_t)(ny + 1) * (nx + 1) + (size_t)j * (nx + 1) + i] = wy;
    }
    if (K && (own_x || own_y)) {
        const float *Fb = F + a * fs + b;       // Fb[r][c] = f at (i - 2 + c, j - 2 + r)
        const float *Gb = G + a * gs + b;       // Gb[r][c] = g at (i - 1 + c, j - 1 + r)
        const float f11 = Fb[fs + 1], f12 = Fb[fs + 2], f21 = Fb[2 * fs + 1], f22 = Fb[2 * fs + 2];
        const float g00 = Gb[0], g01 = Gb[1], g10 = Gb[gs], g11 = Gb[gs + 1];
        float aex = 0.0f, bex = 0.0f, aey = 0.0f, bey = 0.0f;
        if (own_x)
            edge_ab(f21, f22, Fb[3 * fs + 1], Fb[3 * fs + 2], f11, f12,
                    g10, g11, Gb[2 * gs], Gb[2 * gs + 1], g00, g01, &aex, &bex);
        if (own_y)
            edge_ab(f12, f22, Fb[fs + 3], Fb[2 * fs + 3], f11, f21,
                    g01, g11, Gb[2], Gb[gs + 2], g00, g10, &aey, &bey);
        trial_accum<KT, EDGES>(K, s_t, eps2, Tx, wx, aex, bex, Ty, wy, aey, bey, dJ);
    }
}

// One 32 x 8 tile's share of a GD iteration's sums (Eq. 9's energy and the Armijo trial
// changes), evaluated by 128 threads (vt = 0..127) from the tile's values in shared memory:
//   sA = sum <g, f - v>, sB = sum g^2, sF = sum (f - v)^2 over the tile's pixels,
//   sJ = sum w T and dJ[m] = sum w (T'(t_m) - T) over the tile's owned half-edges (the left
//   x-edge and the upper y-edge of every pixel, and the edges on the image's right / lower
//   border when the tile touches it).
// Thread vt takes the vertically adjacent positions (a, b) = (2 (vt / 32), vt % 32) and
// (a + 1, b) -- their stencils share most of their values -- then (vt < 8) the right-border
// x-edge of row vt, or (32 <= vt < 64) the lower-border y-edge of column vt - 32: every
// value is a fixed function of the tile, so the per-tile sums (FP32 per thread and warp)
// do not depend on which kernel or block evaluates the tile.
// Frames (row stride in elements): F[r][c] = f at pixel (X0 - 2 + c, Y0 - 2 + r);
// G[r][c] = g and V[r][c] = v at pixel (X0 - 1 + c, Y0 - 1 + r); TX / WX [r][c] = x-edge
// between pixel columns X0 - 2 + c and X0 - 1 + c in row Y0 - 1 + r; TY / WY [r][c] =
// y-edge between pixel rows Y0 - 2 + r and Y0 - 1 + r in column X0 - 1 + c.
template <int KT>
__device__ __forceinline__ void tile_sums(int vt, int X0, int Y0, int nx, int ny, const float *F, int fs,
                                          const float *G, int gs, const float *V, int vs,
                                          const float *TX, const float *WX, int xs,
                                          const float *TY, const float *WY, int ys, int K,
                                          const float *s_t, float eps2, float *wout,
                                          float *sA, float *sB, float *sF, float *sJ, float (&dJ)[KT]) {
    constexpr int TW = 32, TH = 8;
    const int a = 2 * (vt >> 5), b = vt & 31;
    tile_position<KT>(a, b, X0, Y0, nx, ny, F, fs, G, gs, V, vs, TX, WX, xs, TY, WY, ys, K, s_t, eps2,
                      wout, sA, sB, sF, sJ, dJ);
    tile_position<KT>(a + 1, b, X0, Y0, nx, ny, F, fs, G, gs, V, vs, TX, WX, xs, TY, WY, ys, K, s_t,
                      eps2, wout, sA, sB, sF, sJ, dJ);
    // edges on the image's right / lower border (only tiles that reach it own them)
    if (X0 + TW >= nx && vt < TH)             // column TW: only its x-edge can be owned
        tile_position<KT, 1>(vt, TW, X0, Y0, nx, ny, F, fs, G, gs, V, vs, TX, WX, xs, TY, WY, ys, K, s_t,
                             eps2, wout, sA, sB, sF, sJ, dJ);
    else if (Y0 + TH >= ny && vt >= 32 && vt < 32 + TW)    // row TH: only its y-edge
        tile_position<KT, 2>(TH, vt - 32, X0, Y0, nx, ny, F, fs, G, gs, V, vs, TX, WX, xs, TY, WY, ys, K,
                             s_t, eps2, wout, sA, sB, sF, sJ, dJ);
}

}  // namespace eptv
