// 3-D cone-beam EPTV (the paper's method, which is 2-D, extended to a circular cone-beam
// scan with a flat detector; see eptv.h for the conventions).  Same algorithm as the 2-D
// path (Sec. 2.2: CGLS for (P1), GD with Armijo for (P2), clamp).
// Rays are parametrised by their depth along the central ray, counted from the plane
// through the rotation axis (D' = D - sid).  The x and y plane crossings of a ray then
// depend only on its view and detector column, the z plane crossings only on its detector
// row, and its length through a voxel is F * (D' interval) with F = |a| = sqrt(1 + (u^2 +
// w^2) / sdd^2) per detector pixel: P = diag(F) L', and both kernels below compute the
// entries of L' with the same canonical formula from the same tables.  Kernels:
//   K31  P:   ray-driven Siddon in 3-D.  A warp holds 32 adjacent detector columns of one
//             detector row; the SEG warps of a block split the ray's range along its major
//             axis (x or y).  The ray walks one cell per loop step: the cell's length is
//             its exit (the nearest of its three exit planes) minus its entry (the
//             previous cell's exit), the canonical min(exit planes) - max(entry planes) of
//             eptv_internal.cuh, and the lanes advance by selects, never branching apart.
//   K32  P^T: voxel-driven gather, the exact transpose L'^T diag(F): a thread owns ZP
//             voxels stacked in z (2 or 4); per view, the stack's corners bound the
//             detector columns and rows whose rays can cross it; per column, the x-y chord
//             through the stack; per row, the stack's plane parameters clamped to the
//             chord give each voxel's canonical length.
//   (P2) voxel-major kernels (the 2-D half-edges extended to faces, Eqs. 5, 9, A2, A3 in
//             3-D): the face magnitudes for sigma, the gradient with the energy sums, all
//             Armijo trial steps with the step decision, and the step / clamp; a thread
//             marches a column segment in z with the voxel's 19-value neighbourhood in
//             registers.  The block sums go through the exact, order-independent
//             reduction of eptv_internal.cuh; the step decision is FP64 in parallel lanes.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "eptv_internal.cuh"
#include "kernels.cuh"

namespace eptv {

// Per (view, column): the x, y of the ray's point at depth sid (D' = 0) and 1 / a_x,
// 1 / a_y, a = (central direction) + (u / sdd) e_u + (w / sdd) e_z the ray's direction per
// unit depth (a_x, a_y do not depend on w).  One 128-bit load.
struct __align__(16) ColRec3 { float qx, qy, ix, iy; };
// Per detector row: the z of the point at depth sid (w sid / sdd) and 1 / a_z = sdd / w.
struct __align__(8) RowRec3 { float qz, iz; };
// Records padded to 32 bytes and 16-byte aligned, so that one is two 128-bit loads.
struct __align__(16) ViewRec3 { float sx, sy, cx, cy, ux, uy, pad0, pad1; };  // source, central dir, e_u

struct Cone {
    int nx, ny, nz, nv, nu, nrow;                   // nv views, nu x nrow detector
    float dx, dy, dz, x0, y0, z0;
    float du, dw, uc, wc;                           // column index = u / du + uc, row = w / dw + wc
    float inv_du, inv_dw;                           // 1 / du, 1 / dw (candidate bounds only)
    float sdd, sid;
    float rxy;                                      // >= half-diagonal of the volume in x-y
    int band_max;                                   // >= rows of any z slab's band (K32)
    long long n_vox, n_rays;
    const ColRec3 *col;                             // [view][column]
    const RowRec3 *row;                             // [row]
    const float *fac;                               // F = |a| per detector pixel, [row][column]
    const ViewRec3 *view;
};

__device__ __forceinline__ float c3_len(float lo_a, float hi_a, float lo_b, float hi_b, float lo_c,
                                        float hi_c) {
    return fmaxf(0.0f, __fsub_rn(fminf(fminf(hi_a, hi_b), hi_c), fmaxf(fmaxf(lo_a, lo_b), lo_c)));
}

// ------------------------------------------------------------------ K31: projector

template <int SEG>
__global__ void __launch_bounds__(32 * SEG, 40 / SEG)
k31_project(Cone C, const float *__restrict__ f, const float *__restrict__ y_resid, float *__restrict__ out,
            double *__restrict__ partials, SliceDev *S, int fin)
{
    const double gamma_pre = threadIdx.x == 0 ? fin_gamma(S->sc, fin) : 0.0;
    __shared__ float red[SEG][33];
    __shared__ double rsm[2 * SEG];
    __shared__ double res[2];
    __shared__ int last_flag;
    const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
    const int nub = (C.nu + 31) >> 5;
    const int row_id = blockIdx.x / nub;                  // view * nrow + detector row
    const int iu = (blockIdx.x - row_id * nub) * 32 + lane;
    const int view = row_id / C.nrow, iv = row_id - view * C.nrow;
    const long long ri = (long long)row_id * C.nu + iu;
    float acc = 0.0f;
    if (iu < C.nu) {
        const ColRec3 Qc = C.col[view * C.nu + iu];
        const RowRec3 Qr = C.row[iv];
        struct { float px, py, pz, ix, iy, iz; } R = {Qc.qx, Qc.qy, Qr.qz, Qc.ix, Qc.iy, Qr.iz};
        // major axis M (x or y), minor axes m (the other) and z
        const bool ymaj = fabsf(R.ix) * C.dx >= fabsf(R.iy) * C.dy;
        float PM, iM, M0, dM, Pm, im, m0, dm;
        int nM, nm, sM, sm;                               // index strides of M and m
        if (ymaj) {
            PM = R.py; iM = R.iy; M0 = C.y0; dM = C.dy; nM = C.ny; sM = C.nx;
            Pm = R.px; im = R.ix; m0 = C.x0; dm = C.dx; nm = C.nx; sm = 1;
        } else {
            PM = R.px; iM = R.ix; M0 = C.x0; dM = C.dx; nM = C.nx; sM = 1;
            Pm = R.py; im = R.iy; m0 = C.y0; dm = C.dy; nm = C.ny; sm = C.nx;
        }
        float iz = R.iz;
        if (iM < 0.0f) { iM = -iM; im = -im; iz = -iz; }  // march with t increasing along M
        const int sgm = im > 0.0f ? 1 : -1, sgz = iz > 0.0f ? 1 : -1;
        const int ohm = sgm > 0 ? 1 : 0, olm = 1 - ohm, ohz = sgz > 0 ? 1 : 0, olz = 1 - ohz;
        const long long sz = (long long)C.nx * C.ny;
        // the ray's parameter range inside the minor-axis slabs of the volume
        const float tmA = cross_t(grid_line(0.0f, dm, m0), Pm, im);
        const float tmB = cross_t(grid_line((float)nm, dm, m0), Pm, im);
        const float tzA = cross_t(grid_line(0.0f, C.dz, C.z0), R.pz, iz);
        const float tzB = cross_t(grid_line((float)C.nz, C.dz, C.z0), R.pz, iz);
        const float t_lo = fmaxf(fminf(tmA, tmB), fminf(tzA, tzB));
        const float t_hi = fminf(fmaxf(tmA, tmB), fmaxf(tzA, tzB));
        const float tM0 = cross_t(grid_line(0.0f, dM, M0), PM, iM);
        const float tMn = cross_t(grid_line((float)nM, dM, M0), PM, iM);
        if (t_lo < t_hi && t_hi > tM0 && t_lo < tMn) {
            const float dMinv = 1.0f / iM;
            auto slab_of = [&](float t) {                  // largest r with t_M(r) <= t
                int r = (int)floorf(__fdividef(PM + t * dMinv - M0, dM));
                r = min(max(r, 0), nM - 1);
                for (int it = 0; it < 4 && r > 0 && cross_t(grid_line((float)r, dM, M0), PM, iM) > t; ++it) --r;
                for (int it = 0; it < 4 && r < nM - 1 && cross_t(grid_line((float)(r + 1), dM, M0), PM, iM) <= t; ++it) ++r;
                return r;
            };
            const int r_first = (t_lo <= tM0) ? 0 : slab_of(t_lo);
            const int r_last = (t_hi >= tMn) ? nM - 1 : slab_of(t_hi);
            const int nr = r_last - r_first + 1;
            const int chunk = (nr + SEG - 1) / SEG;
            const int rs = r_first + seg * chunk, re = min(rs + chunk - 1, r_last);
            if (rs <= re) {
                float ta = cross_t(grid_line((float)rs, dM, M0), PM, iM);
                const float t0 = fmaxf(ta, t_lo);
                // minor cells containing t0 (lo(c) <= t0 < hi(c)), m then z
                auto cell_of = [&](float P, float inv, float o, float d, int n, int sg, int ol, int oh) {
                    int c = (int)floorf(__fdividef(P + t0 / inv - o, d));
                    c = min(max(c, 0), n - 1);
                    for (int it = 0; it < 4; ++it) {
                        const float lo = cross_t(grid_line((float)(c + ol), d, o), P, inv);
                        const int cn = c - sg;
                        if (lo > t0 && cn >= 0 && cn < n) c = cn; else break;
                    }
                    for (int it = 0; it < 4; ++it) {
                        const float hi = cross_t(grid_line((float)(c + oh), d, o), P, inv);
                        const int cn = c + sg;
                        if (hi <= t0 && cn >= 0 && cn < n) c = cn; else break;
                    }
                    return c;
                };
                int cm = cell_of(Pm, im, m0, dm, nm, sgm, olm, ohm);
                int cz = cell_of(R.pz, iz, C.z0, C.dz, C.nz, sgz, olz, ohz);
                float lom = cross_t(grid_line((float)(cm + olm), dm, m0), Pm, im);
                float him = cross_t(grid_line((float)(cm + ohm), dm, m0), Pm, im);
                float loz = cross_t(grid_line((float)(cz + olz), C.dz, C.z0), R.pz, iz);
                float hiz = cross_t(grid_line((float)(cz + ohz), C.dz, C.z0), R.pz, iz);
                // The slab interval is clipped to the volume's (m, z) extent [t_lo, t_hi]:
                // plane parameters are monotone in the plane index, so for a cell inside the
                // volume the clipping changes neither its largest entry nor its smallest
                // exit plane and the clipped length is bit-identical to the canonical
                // six-plane formula; a cell outside gets length exactly 0.  The cell's
                // offset in the volume is carried along (32 bits: n_vox < 2^31).
                //
                // One loop iteration per cell: the walk leaves the cell through the nearest
                // of its M, m and z exit planes (M last on a tie with the clipped M exit,
                // m before z on a tie), so the lanes of a warp step together for as many
                // iterations as their longest walk, instead of each slab costing the warp
                // its lane with the most crossings.  A cell's largest entry plane is the
                // previous cell's exit (entry planes only grow along the walk, and the one
                // just crossed is the largest): tin = max(tin, exit) is the canonical max of
                // the three entry planes, exactly, for every cell inside the volume, and
                // beyond the volume's exit both give length 0.  The next crossing of each
                // axis is evaluated every step (three FMA-pipe triples, no operand selects)
                // and the one crossed is kept by selects, so the lanes never branch apart.
                // A cell's load is issued one step before its product is added (the
                // additions keep the walk's order).  Cells of nonzero length are inside the volume
                // (outside it every length is 0, see above); the clamp of the offset only
                // keeps the load in bounds.
                const int step_m = sgm * sm, step_z = sgz * (int)sz;
                const float sgm_f = (float)sgm, sgz_f = (float)sgz;
                const unsigned last_vox = (unsigned)(C.n_vox - 1);
                int idx = cz * (int)sz + rs * sM + cm * sm;
                float tin = fmaxf(fmaxf(t0, lom), loz);
                float tbc = fminf(cross_t(grid_line((float)(rs + 1), dM, M0), PM, iM), t_hi);
                float kM = (float)(rs + 2);                       // next plane index, per axis
                float km = (float)(cm + ohm) + sgm_f;
                float kz = (float)(cz + ohz) + sgz_f;
                const float kend = (float)(re + 2);               // M plane after the last slab's exit
                const int cap = (re - rs + 1) + nm + C.nz + 2;    // each step moves one index
                float pl = 0.0f, pv = 0.0f;
                for (int it = 0; it < cap; ++it) {
                    const float mn = fminf(him, hiz);
                    const float ex = fminf(tbc, mn);
                    const float lc = fmaxf(0.0f, __fsub_rn(ex, tin));
                    const float v = lc > 0.0f ? __ldg(f + min((unsigned)idx, last_vox)) : 0.0f;
                    acc = fmaf(pl, pv, acc);
                    pl = lc; pv = v;
                    tin = fmaxf(tin, ex);
                    const bool adv_M = !(mn < tbc);
                    if (adv_M && kM == kend) break;
                    const float tnM = cross_t(grid_line(kM, dM, M0), PM, iM);
                    const float tnm = cross_t(grid_line(km, dm, m0), Pm, im);
                    const float tnz = cross_t(grid_line(kz, C.dz, C.z0), R.pz, iz);
                    const bool adv_m = !adv_M && him <= hiz;
                    const bool adv_z = !adv_M && !adv_m;
                    tbc = adv_M ? fminf(tnM, t_hi) : tbc;
                    kM += adv_M ? 1.0f : 0.0f;
                    him = adv_m ? tnm : him;
                    km += adv_m ? sgm_f : 0.0f;
                    hiz = adv_z ? tnz : hiz;
                    kz += adv_z ? sgz_f : 0.0f;
                    idx += adv_M ? sM : (adv_m ? step_m : step_z);
                }
                acc = fmaf(pl, pv, acc);
            }
        }
    }
    red[seg][lane] = acc;
    __syncthreads();
    float sq = 0.0f, ysum = 0.0f;
    if (seg == 0 && iu < C.nu) {
        float tot = 0.0f;
#pragma unroll
        for (int w = 0; w < SEG; ++w) tot += red[w][lane];
        tot *= __ldg(C.fac + iv * C.nu + iu);              // L' -> P
        const float o = y_resid ? __ldg(y_resid + ri) - tot : tot;
        out[ri] = o;
        sq = o * o;
        ysum = o;
    }
    if (fin == FIN_NONE) return;
    float vals[2] = {sq, ysum};
    block_sum_to<2, 32 * SEG>(vals, partials + (size_t)blockIdx.x * 2, rsm);
    if (!reduce_slice<2, 32 * SEG>(*S, partials, 2, 0, gridDim.x, blockIdx.x, rsm, res, &last_flag)) return;
    if (threadIdx.x == 0) finalize(S->sc, fin, res[0], res[1], gamma_pre);
}

// ------------------------------------------------------------------ K32: back projector

// ys = F * y per ray (the diag(F) of P^T = L'^T diag(F)); grid.y = view
__global__ void __launch_bounds__(256)
k32_scale(const float *__restrict__ y, const float *__restrict__ fac, int npix, float *__restrict__ ys)
{
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= npix) return;
    const long long r = (long long)blockIdx.y * npix + i;
    ys[r] = __ldg(y + r) * __ldg(fac + i);
}

// Thread = ZP voxels stacked in z, (ix, iy, ZP iz_b + q), q < ZP; block = 256 (ix, iy) of
// one z block iz_b (grid.y).  A voxel's detector columns do not depend on z, and a
// column's x-y chord through the stack (its x and y plane parameters) does not depend on
// the row, so the stack shares, per view, its corner projections and, per column, the
// chord.  The z planes of a row depend on the row alone and all threads of a block have
// the same z planes: the block tabulates, in shared memory, each row's parameter interval
// through each voxel of the stack, for the band of rows that can meet its slab at any
// depth of the volume.
constexpr int kZPair = 2;                                   // smallest stack (grid and workspace bounds)
constexpr int kZStackMax = 4;                               // tallest stack (row bands)

// first and last detector row of the band of the slab [Za, Zb]: depths of the volume
// sid + D', |D'| <= rxy; half a row of margin (the per-column bounds use 0.01)
__device__ __forceinline__ void k32_band(const Cone &C, float Za, float Zb, int &b0, int &b1) {
    const float ka = __fdividef(C.sdd, C.sid - C.rxy), kb = __fdividef(C.sdd, C.sid + C.rxy);
    const float wlo = fminf(Za * ka, Za * kb), whi = fmaxf(Zb * ka, Zb * kb);
    b0 = max(0, (int)ceilf(fmaf(wlo, C.inv_dw, C.wc) - 0.5f));
    b1 = min(C.nrow - 1, (int)floorf(fmaf(whi, C.inv_dw, C.wc) + 0.5f));
    b1 = min(b1, b0 + C.band_max - 1);
}

template <int ZP>
__global__ void __launch_bounds__(256, 4)
k32_backproject(Cone C, const float *__restrict__ ys, float *__restrict__ out, double *__restrict__ partials,
                SliceDev *S, int fin)
{
    constexpr int NQ = ZP / 2;                              // float4 per row: the ZP + 1 plane parameters
    static_assert(4 * NQ >= ZP + 1, "plane parameters fit the row's words");
    const double gamma_pre = threadIdx.x == 0 ? fin_gamma(S->sc, fin) : 0.0;
    extern __shared__ float4 s_zt[];                       // [band][NQ]
    __shared__ double rsm[2 * 8];
    __shared__ double res[2];
    __shared__ int last_flag;
    const int iz0 = blockIdx.y * ZP;
    const int nzp = min(ZP, C.nz - iz0);                    // voxels of the stack inside
    float Z[ZP + 1];
#pragma unroll
    for (int q = 0; q <= ZP; ++q) Z[q] = grid_line((float)(iz0 + q), C.dz, C.z0);
    const float Ze = grid_line((float)(iz0 + nzp), C.dz, C.z0);
    int b0, b1;
    k32_band(C, Z[0], Ze, b0, b1);
    for (int r = b0 + (int)threadIdx.x; r <= b1; r += 256) {
        const RowRec3 Rr = C.row[r];
        float tz[4 * NQ];
#pragma unroll
        for (int q = 0; q < 4 * NQ; ++q) tz[q] = q <= ZP ? cross_t(Z[q], Rr.qz, Rr.iz) : 0.0f;
#pragma unroll
        for (int h = 0; h < NQ; ++h)
            s_zt[(r - b0) * NQ + h] = make_float4(tz[4 * h], tz[4 * h + 1], tz[4 * h + 2], tz[4 * h + 3]);
    }
    __syncthreads();
    const int pxy = blockIdx.x * 256 + threadIdx.x;         // iy * nx + ix
    float acc[ZP];
#pragma unroll
    for (int q = 0; q < ZP; ++q) acc[q] = 0.0f;
    const bool valid = pxy < C.nx * C.ny;
    if (valid) {
        const int iy = pxy / C.nx, ix = pxy - iy * C.nx;
        const float X0 = grid_line((float)ix, C.dx, C.x0), X1 = grid_line((float)(ix + 1), C.dx, C.x0);
        const float Y0 = grid_line((float)iy, C.dy, C.y0), Y1 = grid_line((float)(iy + 1), C.dy, C.y0);
        const long long view_sz = (long long)C.nrow * C.nu;
        for (int v = 0; v < C.nv; ++v) {
            const ViewRec3 V = C.view[v];
            float umin = 3e38f, umax = -3e38f, dmin = 3e38f, dmax = -3e38f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float px = (c & 1) ? X1 : X0, py = (c & 2) ? Y1 : Y0;
                const float wx = px - V.sx, wy = py - V.sy;
                const float depth = V.cx * wx + V.cy * wy;            // along the central ray
                const float u = __fdividef((V.ux * wx + V.uy * wy) * C.sdd, depth);
                umin = fminf(umin, u); umax = fmaxf(umax, u);
                dmin = fminf(dmin, depth); dmax = fmaxf(dmax, depth);
            }
            const int iu0 = max(0, (int)ceilf(fmaf(umin, C.inv_du, C.uc) - 0.01f));
            const int iu1 = min(C.nu - 1, (int)floorf(fmaf(umax, C.inv_du, C.uc) + 0.01f));
            // rows whose rays are inside [Z0, Ze] at some depth of the stack's x-y column:
            // w = z sdd / depth, depth in [dmin, dmax] (the corners' depths bound every
            // chord's; the margin covers their rounding).  The same rows serve every
            // column of the view, so the lanes of a warp (one slab, nearly equal depths)
            // walk the same rows; rows outside a chord's own range add exact zeros.
            const float ka = __fdividef(C.sdd, dmin), kb = __fdividef(C.sdd, dmax);
            const float wlo = fminf(Z[0] * ka, Z[0] * kb), whi = fmaxf(Ze * ka, Ze * kb);
            const int iv0 = max(b0, (int)ceilf(fmaf(wlo, C.inv_dw, C.wc) - 0.01f));
            const int iv1 = min(b1, (int)floorf(fmaf(whi, C.inv_dw, C.wc) + 0.01f));
            const ColRec3 *colv = C.col + v * C.nu;
            const float *ysv = ys + v * view_sz;
            for (int iu = iu0; iu <= iu1; ++iu) {
                const ColRec3 Q = colv[iu];
                const float ax = cross_t(X0, Q.qx, Q.ix), bx = cross_t(X1, Q.qx, Q.ix);
                const float ay = cross_t(Y0, Q.qy, Q.iy), by = cross_t(Y1, Q.qy, Q.iy);
                const float lo_xy = fmaxf(fminf(ax, bx), fminf(ay, by));
                const float hi_xy = fminf(fmaxf(ax, bx), fmaxf(ay, by));
                if (!(lo_xy < hi_xy)) continue;
                const float *ycol = ysv + iu;
                // Voxel q of the stack spans the row's plane parameters tz[q], tz[q + 1]
                // (a = their min, b = their max).  With c = min(max(tz, lo_xy), hi_xy),
                // |c[q + 1] - c[q]| is bit for bit the canonical six-plane length
                // max(0, min(hi_xy, b) - max(lo_xy, a)): where the intervals meet the two
                // clamped ends are min(hi_xy, b) and max(lo_xy, a) themselves, elsewhere
                // both ends clamp to the same bound (lo_xy < hi_xy here).  ZP + 1 clamps
                // instead of two min / max per voxel.
                for (int iv = iv0; iv <= iv1; ++iv) {
                    const float yv = __ldg(ycol + iv * C.nu);
                    float c[4 * NQ];
#pragma unroll
                    for (int h = 0; h < NQ; ++h) {
                        const float4 zt = s_zt[(iv - b0) * NQ + h];
                        c[4 * h] = zt.x; c[4 * h + 1] = zt.y; c[4 * h + 2] = zt.z; c[4 * h + 3] = zt.w;
                    }
#pragma unroll
                    for (int q = 0; q <= ZP; ++q) c[q] = fminf(fmaxf(c[q], lo_xy), hi_xy);
#pragma unroll
                    for (int q = 0; q < ZP; ++q) acc[q] = fmaf(fabsf(__fsub_rn(c[q + 1], c[q])), yv, acc[q]);
                }
            }
        }
        const long long nxy = (long long)C.nx * C.ny;
        const long long vox = (long long)iz0 * nxy + pxy;
#pragma unroll
        for (int q = 0; q < ZP; ++q)
            if (q < nzp) out[vox + q * nxy] = acc[q];
    }
    if (fin == FIN_NONE) return;
    const int nblk = gridDim.x * gridDim.y, lb = blockIdx.y * gridDim.x + blockIdx.x;
    float sq = 0.0f;
#pragma unroll
    for (int q = 0; q < ZP; ++q)
        if (valid && q < nzp) sq = fmaf(acc[q], acc[q], sq);
    float vals[1] = {sq};
    block_sum_to<1, 256>(vals, partials + (size_t)lb * 2, rsm);
    if (threadIdx.x == 0) partials[(size_t)lb * 2 + 1] = 0.0;
    if (!reduce_slice<2, 256>(*S, partials, 2, 0, nblk, lb, rsm, res, &last_flag)) return;
    if (threadIdx.x == 0) finalize(S->sc, fin, res[0], res[1], gamma_pre);
}

// ------------------------------------------------------------------ CGLS vectors

// y += sign * sc[which] * x
__global__ void __launch_bounds__(256)
k3v_axpy(float *__restrict__ y, const float *__restrict__ x, long long n, const double *__restrict__ sc,
         int which, float sign)
{
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const float a = sign * (float)sc[which];
    y[i] = fmaf(a, x[i], y[i]);
}

// u += a s; then (more) s = t + b s
__global__ void __launch_bounds__(256)
k3v_update_us(float *__restrict__ u, float *__restrict__ s, const float *__restrict__ t, long long n,
              const double *__restrict__ sc, int more)
{
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const float a = (float)sc[SC_A], b = (float)sc[SC_B];
    const float sv = s[i];
    u[i] = fmaf(a, sv, u[i]);
    if (more) s[i] = fmaf(b, sv, t[i]);
}

// ------------------------------------------------------------------ (P2) in 3-D

// Faces: family d (0: x, 1: y, 2: z) at (i, j, k) lies between voxel (i, j, k) - e_d ("a")
// and (i, j, k) ("b"); x-faces (nx+1) ny nz, y-faces nx (ny+1) nz, z-faces nx ny (nz+1).
// Voxel p = (i, j, k) owns the lower face of each family (a = p - e_d, b = p) and, on the
// volume's last plane of that family, the upper one (a = p, b = p + e_d): every face has
// one owner.  A face's stencil (Eq. A3 extended to 3-D: its two voxels and their four
// neighbours along each transverse axis) stays inside the 3 x 3 x 3 neighbourhood of
// either voxel beside it -- the centre, its 6 face and 12 edge neighbours -- so the
// kernels below take one voxel per thread, load those 19 values once (0 outside the
// volume) and evaluate all six faces from registers.
struct Vol {
    int nx, ny, nz;
    long long nfx, nfy, nfz, nf;
};

// The 19 values of x around voxel (i, j, k) at linear index p (corners unused, 0):
// N[dk + 1][dj + 1][di + 1].
__device__ __forceinline__ void load_nbhd(const float *__restrict__ x, const Vol &V, int i, int j, int k,
                                          long long p, float (&N)[3][3][3]) {
    const bool inner = i >= 1 && i <= V.nx - 2 && j >= 1 && j <= V.ny - 2 && k >= 1 && k <= V.nz - 2;
    const long long sy = V.nx, sz = (long long)V.nx * V.ny;
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk)
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
            for (int di = -1; di <= 1; ++di) {
                float val = 0.0f;
                if (abs(di) + abs(dj) + abs(dk) <= 2) {
                    const bool in = inner || (i + di >= 0 && i + di < V.nx && j + dj >= 0 && j + dj < V.ny &&
                                              k + dk >= 0 && k + dk < V.nz);
                    if (in) val = __ldg(x + p + di + dj * sy + dk * sz);
                }
                N[dk + 1][dj + 1][di + 1] = val;
            }
}

// The stencil of face (family D, UP: the upper face of the centre voxel, else the lower)
// in the neighbourhood N: a, b and, for the transverse axes t1 < t2, a +- e_t, b +- e_t.
template <int D, int UP>
struct FaceAt {
    static constexpr int ax = (D == 0 && !UP) ? -1 : 0, ay = (D == 1 && !UP) ? -1 : 0,
                         az = (D == 2 && !UP) ? -1 : 0;
    static constexpr int bx = ax + (D == 0), by = ay + (D == 1), bz = az + (D == 2);
    static constexpr int T1 = (D == 0) ? 1 : 0, T2 = (D == 2) ? 1 : 2;
    __device__ static __forceinline__ float at(const float (&N)[3][3][3], int x, int y, int z) {
        return N[z + 1][y + 1][x + 1];
    }
    // values: [0] a, [1] b, [2] a + e_t1, [3] b + e_t1, [4] a - e_t1, [5] b - e_t1, then t2
    __device__ static __forceinline__ void values(const float (&N)[3][3][3], float (&s)[10]) {
        constexpr int u1x = T1 == 0, u1y = T1 == 1, u1z = T1 == 2;
        constexpr int u2x = T2 == 0, u2y = T2 == 1, u2z = T2 == 2;
        s[0] = at(N, ax, ay, az);
        s[1] = at(N, bx, by, bz);
        s[2] = at(N, ax + u1x, ay + u1y, az + u1z);
        s[3] = at(N, bx + u1x, by + u1y, bz + u1z);
        s[4] = at(N, ax - u1x, ay - u1y, az - u1z);
        s[5] = at(N, bx - u1x, by - u1y, bz - u1z);
        s[6] = at(N, ax + u2x, ay + u2y, az + u2z);
        s[7] = at(N, bx + u2x, by + u2y, bz + u2z);
        s[8] = at(N, ax - u2x, ay - u2y, az - u2z);
        s[9] = at(N, bx - u2x, by - u2y, bz - u2z);
    }
};

// D = b - a and T^2 = eps^2 + D^2 + sum over t1, t2 of (cp^2 + cm^2) / 2 (Eq. A3 in 3-D:
// mc = (a + b) / 2, cp = (a + e_t + b + e_t) / 2 - mc, cm = mc - (a - e_t + b - e_t) / 2)
// from the stencil s of FaceAt::values.  Explicitly rounded (and explicitly fused)
// operations: the two voxels beside a face evaluate it to the same bits.
__device__ __forceinline__ float face_T2(float eps2, const float (&s)[10], float *D) {
    const float d = __fsub_rn(s[1], s[0]);
    const float mc = __fmul_rn(0.5f, __fadd_rn(s[0], s[1]));
    float t2 = __fmaf_rn(d, d, eps2);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const float cp = __fmaf_rn(0.5f, __fadd_rn(s[2 + 4 * t], s[3 + 4 * t]), -mc);
        const float cm = __fmaf_rn(-0.5f, __fadd_rn(s[4 + 4 * t], s[5 + 4 * t]), mc);
        t2 = __fmaf_rn(__fmul_rn(0.5f, cp), cp, t2);      // 0.5 cp is exact
        t2 = __fmaf_rn(__fmul_rn(0.5f, cm), cm, t2);
    }
    *D = d;
    return t2;
}

// The Armijo decomposition of one face along -t g (weights frozen):
// T'^2 = T^2 - 2 t a + t^2 b, a = D dD + 1/2 sum (cp dcp + cm dcm), b = dD^2 + 1/2 sum
// (dcp^2 + dcm^2), the d-quantities the same differences of g (stencils sf, sg).
__device__ __forceinline__ void face_ab(const float (&sf)[10], const float (&sg)[10], float *ae, float *be) {
    const float D = sf[1] - sf[0], dD = sg[1] - sg[0];
    const float mc = 0.5f * (sf[0] + sf[1]), gc = 0.5f * (sg[0] + sg[1]);
    float a = D * dD, b = dD * dD;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const float cp = 0.5f * (sf[2 + 4 * t] + sf[3 + 4 * t]) - mc, cm = mc - 0.5f * (sf[4 + 4 * t] + sf[5 + 4 * t]);
        const float dcp = 0.5f * (sg[2 + 4 * t] + sg[3 + 4 * t]) - gc, dcm = gc - 0.5f * (sg[4 + 4 * t] + sg[5 + 4 * t]);
        a += 0.5f * (cp * dcp + cm * dcm);
        b += 0.5f * (dcp * dcp + dcm * dcm);
    }
    *ae = a;
    *be = b;
}

// T, w (Eq. 5 with 1 / sigma^2 = inv_s2, or 1) and q = w D / T of a face from its D, T^2.
__device__ __forceinline__ void face_Twq(int mode, float inv_s2, float D, float t2, float *T, float *w,
                                         float *q) {
    const float rs = rsqrtf(t2);                // t2 >= eps^2 > 0
    *T = __fmul_rn(t2, rs);
    *w = (mode == EPTV_WEIGHTS_ONE) ? 1.0f : __expf(__fmul_rn(-t2, inv_s2));
    *q = __fmul_rn(__fmul_rn(*w, D), rs);
}

// compensated (Kahan) running sum of one thread's terms: the grid-stride kernels below
// give each thread tens of voxels, and the compensation keeps the thread's sum within a
// few units in the last place, as a single FP32 term would be
__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

__device__ __forceinline__ void vox_pos(const Vol &V, long long p, int &i, int &j, int &k) {
    const int pi = (int)p, q = pi / V.nx;          // n_vox < 2^31
    i = pi - q * V.nx;
    k = q / V.ny;
    j = q - k * V.ny;
}

// T of every face of x (for sigma), one slot per face: the owner's lower faces at
// 3 p + d, the upper faces of the last planes after them (x: ny nz, y: nx nz, z: nx ny)
__global__ void __launch_bounds__(256)
k3tv_face_T(Vol V, const float *__restrict__ x, float eps2, float *__restrict__ T)
{
    const long long nvox = (long long)V.nx * V.ny * V.nz;
    const long long p = (long long)blockIdx.x * 256 + threadIdx.x;
    if (p >= nvox) return;
    int i, j, k;
    vox_pos(V, p, i, j, k);
    float N[3][3][3];
    load_nbhd(x, V, i, j, k, p, N);
    float s[10], D, t2;
    FaceAt<0, 0>::values(N, s); t2 = face_T2(eps2, s, &D); T[3 * p + 0] = __fmul_rn(t2, rsqrtf(t2));
    FaceAt<1, 0>::values(N, s); t2 = face_T2(eps2, s, &D); T[3 * p + 1] = __fmul_rn(t2, rsqrtf(t2));
    FaceAt<2, 0>::values(N, s); t2 = face_T2(eps2, s, &D); T[3 * p + 2] = __fmul_rn(t2, rsqrtf(t2));
    const long long up0 = 3 * nvox, up1 = up0 + (long long)V.ny * V.nz, up2 = up1 + (long long)V.nx * V.nz;
    if (i == V.nx - 1) {
        FaceAt<0, 1>::values(N, s); t2 = face_T2(eps2, s, &D);
        T[up0 + (long long)k * V.ny + j] = __fmul_rn(t2, rsqrtf(t2));
    }
    if (j == V.ny - 1) {
        FaceAt<1, 1>::values(N, s); t2 = face_T2(eps2, s, &D);
        T[up1 + (long long)k * V.nx + i] = __fmul_rn(t2, rsqrtf(t2));
    }
    if (k == V.nz - 1) {
        FaceAt<2, 1>::values(N, s); t2 = face_T2(eps2, s, &D);
        T[up2 + (long long)j * V.nx + i] = __fmul_rn(t2, rsqrtf(t2));
    }
}

// The grad and trial kernels march in z: a work item is a column (i, j) and up to kZChunk
// consecutive voxels of it, and the thread keeps the 19-value neighbourhood in registers
// as it moves up -- the plane below and the centre plane shift down, and only the centre
// plane's four in-plane diagonals and the cross of the new plane above are loaded: 9
// loads per voxel instead of 19, and no index division per voxel.  Items run with x
// fastest, so a warp's loads are consecutive in x.
constexpr int kZChunk = 16;

// In-plane neighbours of column (i, j) inside the volume.
struct ColIn {
    bool xm, xp, ym, yp;
};

// Values around column (i, j) of the plane starting at pl (null: a plane outside the
// volume, all 0): the cross (P[dj + 1][di + 1] with |di| + |dj| <= 1) and the diagonals.
__device__ __forceinline__ void plane_cross(const float *pl, int nx, const ColIn &m, float (&P)[3][3]) {
    P[1][1] = pl ? __ldg(pl) : 0.0f;
    P[1][0] = (pl && m.xm) ? __ldg(pl - 1) : 0.0f;
    P[1][2] = (pl && m.xp) ? __ldg(pl + 1) : 0.0f;
    P[0][1] = (pl && m.ym) ? __ldg(pl - nx) : 0.0f;
    P[2][1] = (pl && m.yp) ? __ldg(pl + nx) : 0.0f;
}
__device__ __forceinline__ void plane_diag(const float *pl, int nx, const ColIn &m, float (&P)[3][3]) {
    P[0][0] = (pl && m.ym && m.xm) ? __ldg(pl - nx - 1) : 0.0f;
    P[0][2] = (pl && m.ym && m.xp) ? __ldg(pl - nx + 1) : 0.0f;
    P[2][0] = (pl && m.yp && m.xm) ? __ldg(pl + nx - 1) : 0.0f;
    P[2][2] = (pl && m.yp && m.xp) ? __ldg(pl + nx + 1) : 0.0f;
}

// Column (i, j) of plane k of x (null outside the volume).
__device__ __forceinline__ const float *plane_ptr(const float *x, const Vol &V, int i, int j, int k) {
    return (k >= 0 && k < V.nz) ? x + ((long long)k * V.ny + j) * V.nx + i : nullptr;
}

// The window N[dk + 1][dj + 1][di + 1] of x around (i, j, k0): the crosses of planes
// k0 - 1 and k0 + 1 and all of plane k0.
__device__ __forceinline__ void zwin_start(const float *x, const Vol &V, int i, int j, int k0, const ColIn &m,
                                           float (&N)[3][3][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) N[a][b][c] = 0.0f;
    plane_cross(plane_ptr(x, V, i, j, k0 - 1), V.nx, m, N[0]);
    const float *p0 = plane_ptr(x, V, i, j, k0);
    plane_cross(p0, V.nx, m, N[1]);
    plane_diag(p0, V.nx, m, N[1]);
    plane_cross(plane_ptr(x, V, i, j, k0 + 1), V.nx, m, N[2]);
}

// The window moved from (i, j, k) to (i, j, k + 1).
__device__ __forceinline__ void zwin_step(const float *x, const Vol &V, int i, int j, int k, const ColIn &m,
                                          float (&N)[3][3][3]) {
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            N[0][b][c] = N[1][b][c];
            N[1][b][c] = N[2][b][c];
        }
    plane_diag(plane_ptr(x, V, i, j, k + 1), V.nx, m, N[1]);
    plane_cross(plane_ptr(x, V, i, j, k + 2), V.nx, m, N[2]);
}

// Work item -> column (i, j), first plane k0 and the in-plane masks (two divisions per item).
__device__ __forceinline__ void zitem(const Vol &V, long long it, int &i, int &j, int &k0, ColIn &m) {
    const long long r = it / V.nx;
    i = (int)(it - r * V.nx);
    const long long c = r / V.ny;
    j = (int)(r - c * V.ny);
    k0 = (int)c * kZChunk;
    m.xm = i > 0;
    m.xp = i < V.nx - 1;
    m.ym = j > 0;
    m.yp = j < V.ny - 1;
}

// One face of the centre voxel: q, and w T.
template <int D, int UP>
__device__ __forceinline__ float face_q(const float (&N)[3][3][3], int mode, float eps2, float inv_s2, float *wT) {
    float s[10], Dv, T, w, q;
    FaceAt<D, UP>::values(N, s);
    const float t2 = face_T2(eps2, s, &Dv);
    face_Twq(mode, inv_s2, Dv, t2, &T, &w, &q);
    *wT = w * T;
    return q;
}

// g = lambda (f - v) - div q (Eq. 9 with Eq. A2: q = w D / T of the voxel's six faces,
// w with sigma = sc[SC_SIGMA]), and the sums J = sum w T over the faces (each by its
// owner), A = g.(f - v), B = g.g, F = |f - v|^2 (to sc[SC_Q0 .. SC_Q0 + 3]).  Along the
// column, a voxel's lower z-face is the upper one of the voxel below: evaluated once.
__global__ void __launch_bounds__(256, 4)
k3tv_grad(Vol V, const float *__restrict__ f, const float *__restrict__ v, float eps2, int mode, float lam,
          float *__restrict__ g, double *__restrict__ partials, SliceDev *S)
{
    __shared__ double rsm[4 * 8];
    __shared__ double res[4];
    __shared__ int last_flag;
    const float sig = (float)S->sc[SC_SIGMA];
    const float inv_s2 = 1.0f / (sig * sig);
    float J = 0.f, A = 0.f, B = 0.f, F = 0.f, cJ = 0.f, cA = 0.f, cB = 0.f, cF = 0.f;
    const long long n_items = (long long)V.nx * V.ny * ((V.nz + kZChunk - 1) / kZChunk);
    for (long long it = (long long)blockIdx.x * 256 + threadIdx.x; it < n_items; it += (long long)gridDim.x * 256) {
        int i, j, k0;
        ColIn m;
        zitem(V, it, i, j, k0, m);
        const int k1 = min(k0 + kZChunk, V.nz);
        float N[3][3][3];
        zwin_start(f, V, i, j, k0, m, N);
        float wT, qz0 = face_q<2, 0>(N, mode, eps2, inv_s2, &wT);
        float wTz0 = wT;
        const long long plane = (long long)V.nx * V.ny;
        long long p = (long long)k0 * plane + (long long)j * V.nx + i;
        for (int k = k0; k < k1; ++k, p += plane) {
            if (k > k0) zwin_step(f, V, i, j, k - 1, m, N);
            float wa, wb;
            const float qx0 = face_q<0, 0>(N, mode, eps2, inv_s2, &wa);
            kahan_add(J, cJ, wa);
            const float qx1 = face_q<0, 1>(N, mode, eps2, inv_s2, &wb);
            if (i == V.nx - 1) kahan_add(J, cJ, wb);
            const float qy0 = face_q<1, 0>(N, mode, eps2, inv_s2, &wa);
            kahan_add(J, cJ, wa);
            const float qy1 = face_q<1, 1>(N, mode, eps2, inv_s2, &wb);
            if (j == V.ny - 1) kahan_add(J, cJ, wb);
            kahan_add(J, cJ, wTz0);
            const float qz1 = face_q<2, 1>(N, mode, eps2, inv_s2, &wb);
            if (k == V.nz - 1) kahan_add(J, cJ, wb);
            const float div = (qx1 - qx0) + (qy1 - qy0) + (qz1 - qz0);
            const float d = N[1][1][1] - __ldg(v + p);
            const float gv = lam * d - div;
            g[p] = gv;
            kahan_add(A, cA, gv * d);
            kahan_add(B, cB, gv * gv);
            kahan_add(F, cF, d * d);
            qz0 = qz1;
            wTz0 = wb;
        }
    }
    float vals[4] = {J - cJ, A - cA, B - cB, F - cF};
    block_sum_to<4, 256>(vals, partials + (size_t)blockIdx.x * kPartialStride, rsm);
    if (!reduce_slice<4, 256>(*S, partials, kPartialStride, 0, gridDim.x, blockIdx.x, rsm, res, &last_flag)) return;
    if (threadIdx.x < 4) S->sc[SC_Q0 + threadIdx.x] = res[threadIdx.x];      // J, A, B, F
}

// dJ_m += w (T'_m - T) of one owned face in the cancellation-free form
// t (t b - 2 a) / (T' + T), T'^2 = T^2 + t (t b - 2 a), for the trial steps s_t[0 .. K).
template <int KT, int D, int UP>
__device__ __forceinline__ void trial_face(const float (&NF)[3][3][3], const float (&NG)[3][3][3], int mode,
                                           float eps2, float inv_s2, int K, const float *s_t, float (&dJ)[KT],
                                           float (&cJ)[KT]) {
    float sf[10], sg[10], Dv, T, w, q, ae, be;
    FaceAt<D, UP>::values(NF, sf);
    FaceAt<D, UP>::values(NG, sg);
    const float t2 = face_T2(eps2, sf, &Dv);
    face_Twq(mode, inv_s2, Dv, t2, &T, &w, &q);
    face_ab(sf, sg, &ae, &be);
    const float T2 = T * T;
#pragma unroll
    for (int m = 0; m < KT; ++m) {
        if (m < K) {
            const float t = s_t[m];
            const float num = t * fmaf(t, be, -2.0f * ae);
            const float T2n = fmaxf(T2 + num, eps2);
            const float Tn = T2n * rsqrtf(T2n);
            kahan_add(dJ[m], cJ[m], w * __fdividef(num, Tn + T));
        }
    }
}

// All Armijo trials of one GD iteration over the faces each voxel owns (weights and T
// frozen at f, evaluated as k3tv_grad evaluates them), then the decision from the sums
// k3tv_grad left in sc[SC_Q0 ..]: the first trial with
// E(f - t g) <= E(f) - c t |g|^2, E = lambda/2 |f - v|^2 + J.
template <int KT>
__global__ void __launch_bounds__(256, 3)
k3tv_trials(Vol V, const float *__restrict__ f, const float *__restrict__ g, const ParamsDev *__restrict__ P,
            int K, int first, int mode, double *__restrict__ partials, SliceDev *S)
{
    __shared__ float s_t[KT];
    __shared__ double s_td[KT];
    __shared__ double rsm[KT * 8];
    __shared__ double tot[KT];
    __shared__ int last_flag;
    if (threadIdx.x == 0) {
        double t;
        if (P->step_rule == EPTV_STEP_FIXED) t = P->t_fixed;
        else t = fmin(P->armijo_grow * S->sc[SC_TPREV], P->t_max > 0.0 ? P->t_max : 1.0 / P->lambda);
        for (int m = 0; m < KT; ++m) {
            s_t[m] = (float)t;
            s_td[m] = (double)(float)t;
            t *= P->armijo_shrink;
        }
    }
    __syncthreads();
    const float eps2 = (float)(P->eps * P->eps);
    const float sig = (float)S->sc[SC_SIGMA];
    const float inv_s2 = 1.0f / (sig * sig);
    float dJ[KT], cJ[KT];
#pragma unroll
    for (int m = 0; m < KT; ++m) dJ[m] = cJ[m] = 0.0f;
    const long long n_items = (long long)V.nx * V.ny * ((V.nz + kZChunk - 1) / kZChunk);
    for (long long it = (long long)blockIdx.x * 256 + threadIdx.x; K > 0 && it < n_items;
         it += (long long)gridDim.x * 256) {
        int i, j, k0;
        ColIn m;
        zitem(V, it, i, j, k0, m);
        const int k1 = min(k0 + kZChunk, V.nz);
        float NF[3][3][3], NG[3][3][3];
        zwin_start(f, V, i, j, k0, m, NF);
        zwin_start(g, V, i, j, k0, m, NG);
        for (int k = k0; k < k1; ++k) {
            if (k > k0) {
                zwin_step(f, V, i, j, k - 1, m, NF);
                zwin_step(g, V, i, j, k - 1, m, NG);
            }
            trial_face<KT, 0, 0>(NF, NG, mode, eps2, inv_s2, K, s_t, dJ, cJ);
            trial_face<KT, 1, 0>(NF, NG, mode, eps2, inv_s2, K, s_t, dJ, cJ);
            trial_face<KT, 2, 0>(NF, NG, mode, eps2, inv_s2, K, s_t, dJ, cJ);
            if (i == V.nx - 1) trial_face<KT, 0, 1>(NF, NG, mode, eps2, inv_s2, K, s_t, dJ, cJ);
            if (j == V.ny - 1) trial_face<KT, 1, 1>(NF, NG, mode, eps2, inv_s2, K, s_t, dJ, cJ);
            if (k == V.nz - 1) trial_face<KT, 2, 1>(NF, NG, mode, eps2, inv_s2, K, s_t, dJ, cJ);
        }
    }
#pragma unroll
    for (int m = 0; m < KT; ++m) dJ[m] -= cJ[m];
    block_sum_to<KT, 256>(dJ, partials + (size_t)blockIdx.x * kPartialStride, rsm);
    if (!reduce_slice<KT, 256>(*S, partials, kPartialStride, 0, gridDim.x, blockIdx.x, rsm, tot, &last_flag))
        return;
    if (threadIdx.x < 32) {
        double *sc = S->sc;
        const double J = sc[SC_Q0], A = sc[SC_Q0 + 1], Bg = sc[SC_Q0 + 2], F = sc[SC_Q0 + 3];
        const double lamd = P->lambda;
        const double E0 = 0.5 * lamd * F + J;
        const bool armijo = P->step_rule != EPTV_STEP_FIXED;
        double dl = 0.0;
        bool pass = false, nonfinite = false;
        if (armijo && threadIdx.x < K) {
            const double t = s_td[threadIdx.x];
            dl = lamd * (-t * A + 0.5 * t * t * Bg) + tot[threadIdx.x];
            nonfinite = !isfinite(dl);
            pass = dl <= -P->armijo_c * t * Bg;
        }
        const unsigned pass_mask = __ballot_sync(0xffffffffu, pass);
        const unsigned bad_mask = __ballot_sync(0xffffffffu, nonfinite);
        const int acc_m = pass_mask ? __ffs(pass_mask) - 1 : -1;
        const double dE = __shfl_sync(0xffffffffu, dl, acc_m >= 0 ? acc_m : 0);
        if (threadIdx.x == 0) {
            bool bad = !isfinite(E0) || !isfinite(A) || !isfinite(Bg);
            {
                if (first) sc[SC_E_FIRST] = E0;
                if (P->step_rule == EPTV_STEP_FIXED) {
                    const double t = s_td[0];
                    sc[SC_TSTEP] = t;
                    sc[SC_E_LAST] = E0 + lamd * (-t * A + 0.5 * t * t * Bg) + (K > 0 ? tot[0] : 0.0);
                    sc[SC_NACC_P2] += 1.0;
                } else {
                    const unsigned seen = acc_m >= 0 ? ((2u << acc_m) - 1u) : ((1u << K) - 1u);
                    if (bad_mask & seen) bad = true;
                    if (acc_m >= 0) {
                        sc[SC_TSTEP] = s_td[acc_m];
                        sc[SC_TPREV] = s_td[acc_m];
                        sc[SC_E_LAST] = E0 + dE;
                        sc[SC_NACC_P2] += 1.0;
                    } else {
                        sc[SC_TSTEP] = 0.0;
                        sc[SC_TPREV] = s_td[K - 1] * P->armijo_shrink / P->armijo_grow;
                        sc[SC_E_LAST] = E0;
                        sc[SC_NFAIL] += 1.0;
                        sc[SC_NFAIL_P2] += 1.0;
                    }
                }
            }
            if (bad) sc[SC_NONFINITE] = 1.0;
        }
    }
}

// f_out = f - sc[SC_TSTEP] g, clamped at 0 when clamp (the last step of a (P2) solve)
__global__ void __launch_bounds__(256)
k3tv_apply(const float *__restrict__ f, const float *__restrict__ g, float *__restrict__ out, long long n,
           const double *__restrict__ sc, int clamp)
{
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    float x = fmaf(-(float)sc[SC_TSTEP], g[i], f[i]);
    if (clamp) x = fmaxf(x, 0.0f);
    out[i] = x;
}

__global__ void k3_set_sigma(const float *__restrict__ val, double floor_, SliceDev *S) {
    S->sc[SC_SIGMA] = fmax((double)*val, floor_);
}

__global__ void k3_set_scalar(SliceDev *S, int which, double value) { S->sc[which] = value; }

__global__ void __launch_bounds__(256) k3_clamp(float *__restrict__ x, long long n) {
    const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
    if (i < n) x[i] = fmaxf(x[i], 0.0f);
}

// ------------------------------------------------------------------ host side

static unsigned nblk_of(long long n, int per) { return (unsigned)((n + per - 1) / per); }
static unsigned nblk_capped(long long n, int per, unsigned cap) { return std::max(1u, std::min(nblk_of(n, per), cap)); }

}  // namespace eptv

using namespace eptv;

struct eptv3_geometry {
    eptv3_geometry_desc desc;
    std::vector<double> angles;
    Cone C;
    Vol V;
    int k31_seg = 8;
    int k32_zp = 4;                                      // voxels per K32 thread (2 or 4)
    unsigned red_blocks = 1184;   // grid of the grid-stride reducing kernels: 8 blocks per SM
    ColRec3 *col = nullptr;
    RowRec3 *row = nullptr;
    float *fac = nullptr;
    float *ys = nullptr;                                 // F * y for K32
    ViewRec3 *view = nullptr;
    float *u = nullptr, *s = nullptr, *t = nullptr, *fa = nullptr, *fb = nullptr, *g = nullptr;
    float *y = nullptr, *r = nullptr, *q = nullptr;
    float *Tsel = nullptr, *sel = nullptr;
    double *partials = nullptr, *sc = nullptr;
    unsigned long long *acc = nullptr;
    unsigned int *ctr = nullptr;
    SliceDev *d_sd = nullptr;
    ParamsDev *d_params = nullptr;
    std::vector<void *> allocs;
};

static int c3_fail(int code, const std::string &m) { return report_error(code, m.c_str()); }

#define C3CU(call)                                                                         \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return c3_fail(EPTV_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
static int c3_alloc(eptv3_geometry *g, T **p, size_t count) {
    void *q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return c3_fail(EPTV_ERR_NOMEM, "cudaMalloc failed for the cone-beam workspace");
    }
    g->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return 0;
}

static float c3_inv(double c) {
    if (std::fabs(c) < 1e-30) return c < 0 ? -1e30f : 1e30f;
    return (float)(1.0 / c);
}

static void c3_project(const eptv3_geometry *g, const float *f, const float *y_resid, float *out, int fin,
                       cudaStream_t st) {
    const unsigned nb = (unsigned)((long long)g->C.nv * g->C.nrow * ((g->C.nu + 31) / 32));
    switch (g->k31_seg) {
    case 2: k31_project<2><<<nb, 64, 0, st>>>(g->C, f, y_resid, out, g->partials, g->d_sd, fin); break;
    case 4: k31_project<4><<<nb, 128, 0, st>>>(g->C, f, y_resid, out, g->partials, g->d_sd, fin); break;
    case 16: k31_project<16><<<nb, 512, 0, st>>>(g->C, f, y_resid, out, g->partials, g->d_sd, fin); break;
    default: k31_project<8><<<nb, 256, 0, st>>>(g->C, f, y_resid, out, g->partials, g->d_sd, fin); break;
    }
}

static void c3_backproject(const eptv3_geometry *g, const float *y, float *out, int fin, cudaStream_t st) {
    const int npix = g->C.nu * g->C.nrow;
    k32_scale<<<dim3(nblk_of(npix, 256), (unsigned)g->C.nv), 256, 0, st>>>(y, g->fac, npix, g->ys);
    const int zp = g->k32_zp;
    const dim3 grid(nblk_of((long long)g->C.nx * g->C.ny, 256), (unsigned)((g->C.nz + zp - 1) / zp));
    const size_t smem = sizeof(float4) * (size_t)g->C.band_max * (zp / 2);
    if (zp == 4) k32_backproject<4><<<grid, 256, smem, st>>>(g->C, g->ys, out, g->partials, g->d_sd, fin);
    else k32_backproject<2><<<grid, 256, smem, st>>>(g->C, g->ys, out, g->partials, g->d_sd, fin);
}

// (P1): M CGLS iterations on g->u (App. I), data g->y
static void c3_cgls(const eptv3_geometry *g, int M, cudaStream_t st) {
    const long long nv = g->C.n_vox, nr = g->C.n_rays;
    c3_project(g, g->u, g->y, g->r, FIN_NONE, st);                       // r = y - P u
    c3_backproject(g, g->r, g->s, FIN_GAMMA0, st);                       // s = P^T r, gamma
    for (int m = 0; m < M; ++m) {
        c3_project(g, g->s, nullptr, g->q, FIN_QQ_TO_A, st);             // q = P s, a
        const bool more = m + 1 < M;
        if (more) {
            k3v_axpy<<<nblk_of(nr, 256), 256, 0, st>>>(g->r, g->q, nr, g->sc, SC_A, -1.0f);
            c3_backproject(g, g->r, g->t, FIN_B, st);                    // t = P^T r, b
        }
        k3v_update_us<<<nblk_of(nv, 256), 256, 0, st>>>(g->u, g->s, g->t, nv, g->sc, more ? 1 : 0);
    }
}

// (P2) on v = g->fa (the CGLS result copied there), result clamped into `out`
static int c3_p2(const eptv3_geometry *g, const eptv_params *p, const float *v, float *out, cudaStream_t st) {
    const Vol &V = g->V;
    const long long nv = g->C.n_vox;
    const float eps2 = (float)(p->eps * p->eps);
    // sigma: k-th smallest face magnitude of v
    k3tv_face_T<<<nblk_of(nv, 256), 256, 0, st>>>(V, v, eps2, g->Tsel);
    const long long rank = std::min<long long>(std::max<long long>((long long)std::ceil(p->sigma_q * V.nf), 1), V.nf);
    const char *err = "";
    int rc = select_kth_noalloc(g->Tsel, (long)V.nf, (long)rank, g->sel, st, &err);
    if (rc) return c3_fail(rc, err);
    k3_set_sigma<<<1, 1, 0, st>>>(g->sel, p->sigma_floor, g->d_sd);
    k3_set_scalar<<<1, 1, 0, st>>>(g->d_sd, SC_NFAIL_P2, 0.0);
    k3_set_scalar<<<1, 1, 0, st>>>(g->d_sd, SC_NACC_P2, 0.0);
    const int K = p->step_rule == EPTV_STEP_FIXED ? 1 : p->max_trials;
    const int mode = p->weights_mode == EPTV_WEIGHTS_ONE ? EPTV_WEIGHTS_ONE : EPTV_WEIGHTS_EPTV;
    const float *cur = v;
    for (int n = 0; n < p->n_gd; ++n) {
        float *nxt = (n == p->n_gd - 1) ? out : ((cur == g->fb) ? g->u : g->fb);
        if (nxt == v) nxt = g->fb;
        const unsigned nbv = nblk_capped((long long)V.nx * V.ny * ((V.nz + kZChunk - 1) / kZChunk), 256, g->red_blocks);
        k3tv_grad<<<nbv, 256, 0, st>>>(V, cur, v, eps2, mode, (float)p->lambda, g->g, g->partials, g->d_sd);
        if (K <= 1) k3tv_trials<1><<<nbv, 256, 0, st>>>(V, cur, g->g, g->d_params, K, n == 0, mode, g->partials, g->d_sd);
        else if (K <= 4) k3tv_trials<4><<<nbv, 256, 0, st>>>(V, cur, g->g, g->d_params, K, n == 0, mode, g->partials, g->d_sd);
        else if (K <= 8) k3tv_trials<8><<<nbv, 256, 0, st>>>(V, cur, g->g, g->d_params, K, n == 0, mode, g->partials, g->d_sd);
        else k3tv_trials<16><<<nbv, 256, 0, st>>>(V, cur, g->g, g->d_params, K, n == 0, mode, g->partials, g->d_sd);
        k3tv_apply<<<nblk_of(nv, 256), 256, 0, st>>>(cur, g->g, nxt, nv, g->sc, n == p->n_gd - 1 ? 1 : 0);
        cur = nxt;
    }
    if (p->n_gd == 0) {
        C3CU(cudaMemcpyAsync(out, v, sizeof(float) * nv, cudaMemcpyDeviceToDevice, st));
        k3_clamp<<<nblk_of(nv, 256), 256, 0, st>>>(out, nv);
    }
    C3CU(cudaGetLastError());
    return 0;
}

static int c3_read_sc(const eptv3_geometry *g, double *h, cudaStream_t st) {
    C3CU(cudaMemcpyAsync(h, g->sc, sizeof(double) * kScalarStride, cudaMemcpyDeviceToHost, st));
    C3CU(cudaStreamSynchronize(st));
    return 0;
}

static int c3_upload_params(const eptv3_geometry *g, const eptv_params *p, cudaStream_t st) {
    ParamsDev pd;
    fill_params(p, &pd);
    C3CU(cudaMemcpyAsync(g->d_params, &pd, sizeof pd, cudaMemcpyHostToDevice, st));
    return 0;
}

extern "C" {

int eptv3_create_geometry(const eptv3_geometry_desc *d, eptv3_geometry **out) {
    if (!d || !out) return c3_fail(EPTV_ERR_ARG, "NULL argument");
    *out = nullptr;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || d->n_views < 1 || d->nu < 1 || d->nv < 1)
        return c3_fail(EPTV_ERR_ARG, "sizes must be >= 1");
    if (!(d->dx > 0 && d->dy > 0 && d->dz > 0 && d->du > 0 && d->dv > 0))
        return c3_fail(EPTV_ERR_ARG, "pitches must be > 0");
    const double R = 0.5 * std::sqrt(d->nx * d->dx * d->nx * d->dx + d->ny * d->dy * d->ny * d->dy);
    const double rxy = R * (1.0 + 1e-5);                  // every depth of the volume is in sid -+ rxy
    if (!(d->sid > rxy * (1.0 + 1e-5)) || !(d->sdd > d->sid))
        return c3_fail(EPTV_ERR_ARG, "need sdd > sid > half-diagonal");
    const long long n_vox = (long long)d->nx * d->ny * d->nz;
    const long long n_rays = (long long)d->n_views * d->nu * d->nv;
    if (n_vox > (1LL << 31) - 1 || n_rays > (1LL << 31) - 1) return c3_fail(EPTV_ERR_ARG, "volume or scan too large");
    eptv3_geometry *g = new eptv3_geometry();
    g->desc = *d;
    if (d->angles) {
        g->angles.assign(d->angles, d->angles + d->n_views);
        g->desc.angles = g->angles.data();
    }
    if (d->n_views > 65535 || (d->nz + kZPair - 1) / kZPair > 65535) {
        delete g;
        return c3_fail(EPTV_ERR_ARG, "at most 65535 views and 131070 slices");
    }
    // ray tables in FP64, stored FP32.  Depth parametrisation: the ray's displacement per
    // unit depth is a = (central direction) + (u / sdd) e_u + (w / sdd) e_z, its point at
    // depth sid is (u e_u + w e_z) sid / sdd (the source plus sid times the central
    // direction is on the rotation axis), and F = |a|
    const int npix = d->nu * d->nv;
    std::vector<ColRec3> cols((size_t)d->n_views * d->nu);
    std::vector<RowRec3> rows((size_t)d->nv);
    std::vector<float> fac((size_t)npix);
    std::vector<ViewRec3> views((size_t)d->n_views);
    const double m_inv = d->sid / d->sdd;
    for (int iv = 0; iv < d->nv; ++iv) {
        const double w = (iv - (d->nv - 1) / 2.0 + d->v_off) * d->dv;
        rows[iv] = RowRec3{(float)(w * m_inv), c3_inv(w / d->sdd)};
        for (int iu = 0; iu < d->nu; ++iu) {
            const double u = (iu - (d->nu - 1) / 2.0 + d->u_off) * d->du;
            fac[(size_t)iv * d->nu + iu] = (float)std::sqrt(1.0 + (u * u + w * w) / (d->sdd * d->sdd));
        }
    }
    for (int k = 0; k < d->n_views; ++k) {
        const double th = d->angles ? d->angles[k] : 2.0 * M_PI * k / d->n_views;
        const double c = std::cos(th), s = std::sin(th);
        const double Sx = d->sid * c, Sy = d->sid * s;
        views[k] = ViewRec3{(float)Sx, (float)Sy, (float)-c, (float)-s, (float)-s, (float)c, 0.0f, 0.0f};
        for (int iv = 0; iv < d->nv; ++iv) {
            const double w = (iv - (d->nv - 1) / 2.0 + d->v_off) * d->dv;
            for (int iu = 0; iu < d->nu; ++iu) {
                const double u = (iu - (d->nu - 1) / 2.0 + d->u_off) * d->du;
                const double ux = -d->sdd * c - u * s, uy = -d->sdd * s + u * c, uz = w;
                const bool zmaj = std::fabs(uz) / d->dz >= std::max(std::fabs(ux) / d->dx, std::fabs(uy) / d->dy);
                if (zmaj) {
                    delete g;
                    return c3_fail(EPTV_ERR_ARG, "cone too wide: a ray crosses z planes faster than x and y planes");
                }
            }
        }
        for (int iu = 0; iu < d->nu; ++iu) {
            const double u = (iu - (d->nu - 1) / 2.0 + d->u_off) * d->du;
            const double ax = -c - u / d->sdd * s, ay = -s + u / d->sdd * c;
            cols[(size_t)k * d->nu + iu] = ColRec3{(float)(-s * u * m_inv), (float)(c * u * m_inv), c3_inv(ax), c3_inv(ay)};
        }
    }
    Cone &C = g->C;
    C.nx = d->nx; C.ny = d->ny; C.nz = d->nz; C.nv = d->n_views; C.nu = d->nu; C.nrow = d->nv;
    C.dx = (float)d->dx; C.dy = (float)d->dy; C.dz = (float)d->dz;
    C.x0 = (float)(-0.5 * d->nx * d->dx); C.y0 = (float)(-0.5 * d->ny * d->dy); C.z0 = (float)(-0.5 * d->nz * d->dz);
    C.du = (float)d->du; C.dw = (float)d->dv;
    C.inv_du = (float)(1.0 / d->du); C.inv_dw = (float)(1.0 / d->dv);
    C.uc = (float)((d->nu - 1) / 2.0 - d->u_off); C.wc = (float)((d->nv - 1) / 2.0 - d->v_off);
    C.sdd = (float)d->sdd; C.sid = (float)d->sid;
    C.rxy = (float)rxy;
    {   // K32's row bands (the kernel's formula in FP64; each end may move by a row in FP32),
        // for the tallest stack: a shorter stack's slab lies inside one of its slabs
        int bmax = 0;
        for (int iz0 = 0; iz0 < d->nz; iz0 += kZStackMax) {
            const int nzp = std::min(kZStackMax, d->nz - iz0);
            const double Za = -0.5 * d->nz * d->dz + iz0 * d->dz, Zb = Za + nzp * d->dz;
            const double ka = d->sdd / (d->sid - rxy), kb = d->sdd / (d->sid + rxy);
            const double wlo = std::min(Za * ka, Za * kb), whi = std::max(Zb * ka, Zb * kb);
            const double wc = (d->nv - 1) / 2.0 - d->v_off;
            const int b0 = std::max(0, (int)std::ceil(wlo / d->dv + wc - 0.5));
            const int b1 = std::min(d->nv - 1, (int)std::floor(whi / d->dv + wc + 0.5));
            bmax = std::max(bmax, b1 - b0 + 1);
        }
        C.band_max = std::min(d->nv, bmax + 2);
        if (C.band_max < 1) C.band_max = 1;
    }
    C.n_vox = n_vox; C.n_rays = n_rays;
    Vol &V = g->V;
    V.nx = d->nx; V.ny = d->ny; V.nz = d->nz;
    V.nfx = (long long)(d->nx + 1) * d->ny * d->nz;
    V.nfy = (long long)d->nx * (d->ny + 1) * d->nz;
    V.nfz = (long long)d->nx * d->ny * (d->nz + 1);
    V.nf = V.nfx + V.nfy + V.nfz;
    if (V.nf > (1LL << 31) - 1) {
        delete g;
        return c3_fail(EPTV_ERR_ARG, "volume too large: 2^31 or more faces");
    }
    // grid of the grid-stride reducing kernels: 8 resident 256-thread blocks of 32 registers per SM
    {
        int dev = 0, n_sm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n_sm > 0)
            g->red_blocks = 8u * (unsigned)n_sm;
        cudaGetLastError();
    }
    // workspace
    const long long blk_k31 = (long long)d->n_views * d->nv * ((d->nu + 31) / 32);
    const long long blk_face = (V.nf + 255) / 256, blk_vox = (n_vox + 255) / 256;
    const long long blk_k32 = ((long long)d->nx * d->ny + 255) / 256 * ((d->nz + kZPair - 1) / kZPair);
    int rc = 0;
    auto A = [&](auto **p, size_t n) { if (!rc) rc = c3_alloc(g, p, n); };
    A(&g->col, cols.size()); A(&g->row, rows.size()); A(&g->fac, fac.size()); A(&g->view, (size_t)d->n_views);
    A(&g->ys, (size_t)n_rays);
    for (float **p : {&g->u, &g->s, &g->t, &g->fa, &g->fb, &g->g}) A(p, (size_t)n_vox);
    for (float **p : {&g->y, &g->r, &g->q}) A(p, (size_t)n_rays);
    A(&g->Tsel, (size_t)V.nf);
    A(&g->sel, 1);
    A(&g->partials, (size_t)std::max(std::max(blk_k31, blk_k32) * 2, std::max(blk_face, blk_vox) * kPartialStride));
    A(&g->acc, (size_t)kPartialStride * kAccCopies * kAccStride);
    A(&g->ctr, 1);
    A(&g->sc, kScalarStride);
    A(&g->d_sd, 1);
    A(&g->d_params, 1);
    if (rc) { eptv3_destroy_geometry(g); return rc; }
    const size_t band_bytes = sizeof(float4) * (size_t)C.band_max;        // per pair of voxels
    if (band_bytes > 100 * 1024) {
        eptv3_destroy_geometry(g);
        return c3_fail(EPTV_ERR_ARG, "detector row band of a z slab too tall for the back projector");
    }
    if (band_bytes > 24 * 1024 &&
        (cudaFuncSetAttribute(k32_backproject<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)band_bytes) != cudaSuccess ||
         cudaFuncSetAttribute(k32_backproject<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * band_bytes)) != cudaSuccess)) {
        cudaGetLastError();
        eptv3_destroy_geometry(g);
        return c3_fail(EPTV_ERR_CUDA, "cannot raise the back projector's shared memory");
    }
    C.col = g->col; C.row = g->row; C.fac = g->fac; C.view = g->view;
    SliceDev sd;
    memset(&sd, 0, sizeof sd);
    sd.ctr = g->ctr; sd.acc = g->acc; sd.sc = g->sc;
    if (cudaMemcpy(g->col, cols.data(), sizeof(ColRec3) * cols.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->row, rows.data(), sizeof(RowRec3) * rows.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->fac, fac.data(), sizeof(float) * fac.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->view, views.data(), sizeof(ViewRec3) * views.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->d_sd, &sd, sizeof sd, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(g->ctr, 0, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(g->acc, 0, sizeof(unsigned long long) * kPartialStride * kAccCopies * kAccStride) != cudaSuccess ||
        cudaMemset(g->sc, 0, sizeof(double) * kScalarStride) != cudaSuccess) {
        eptv3_destroy_geometry(g);
        return c3_fail(EPTV_ERR_CUDA, "upload of the cone-beam tables failed");
    }
    *out = g;
    return 0;
}

void eptv3_destroy_geometry(eptv3_geometry *g) {
    if (!g) return;
    cudaDeviceSynchronize();
    for (void *p : g->allocs) cudaFree(p);
    delete g;
}

int eptv3_set_tuning(eptv3_geometry *g, int seg) {
    if (!g || (seg != 2 && seg != 4 && seg != 8 && seg != 16)) return c3_fail(EPTV_ERR_ARG, "seg must be 2, 4, 8 or 16");
    g->k31_seg = seg;
    return 0;
}

int eptv3_set_backprojector_stack(eptv3_geometry *g, int zp) {
    if (!g || (zp != 2 && zp != 4)) return c3_fail(EPTV_ERR_ARG, "zp must be 2 or 4");
    g->k32_zp = zp;
    return 0;
}

int eptv3_project(const eptv3_geometry *g, const float *d_f, float *d_y, void *stream) {
    if (!g || !d_f || !d_y) return c3_fail(EPTV_ERR_ARG, "NULL argument");
    c3_project(g, d_f, nullptr, d_y, FIN_NONE, (cudaStream_t)stream);
    C3CU(cudaGetLastError());
    return 0;
}

int eptv3_backproject(const eptv3_geometry *g, const float *d_y, float *d_f, void *stream) {
    if (!g || !d_f || !d_y) return c3_fail(EPTV_ERR_ARG, "NULL argument");
    c3_backproject(g, d_y, d_f, FIN_NONE, (cudaStream_t)stream);
    C3CU(cudaGetLastError());
    return 0;
}

int eptv3_cgls(const eptv3_geometry *g, int M, const float *d_y, float *d_u, void *stream) {
    if (!g || !d_y || !d_u) return c3_fail(EPTV_ERR_ARG, "NULL argument");
    if (M < 0) return c3_fail(EPTV_ERR_ARG, "M < 0");
    cudaStream_t st = (cudaStream_t)stream;
    C3CU(cudaMemcpyAsync(g->y, d_y, sizeof(float) * g->C.n_rays, cudaMemcpyDeviceToDevice, st));
    C3CU(cudaMemcpyAsync(g->u, d_u, sizeof(float) * g->C.n_vox, cudaMemcpyDeviceToDevice, st));
    c3_cgls(g, M, st);
    C3CU(cudaGetLastError());
    C3CU(cudaMemcpyAsync(d_u, g->u, sizeof(float) * g->C.n_vox, cudaMemcpyDeviceToDevice, st));
    return 0;
}

int eptv3_tv_step(const eptv3_geometry *g, const eptv_params *p, const float *d_v, float *d_f,
                  double *t_prev_io, eptv_stats *out_opt, void *stream) {
    if (!g || !d_v || !d_f) return c3_fail(EPTV_ERR_ARG, "NULL argument");
    int rc = check_params(p);
    if (rc) return rc;
    if (p->weights_mode == EPTV_WEIGHTS_PRIOR) return c3_fail(EPTV_ERR_ARG, "PRIOR weights are 2-D only");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = c3_upload_params(g, p, st))) return rc;
    const double t0 = (t_prev_io && *t_prev_io > 0.0) ? *t_prev_io : (p->t_init > 0.0 ? p->t_init : 1.0 / p->lambda);
    k3_set_scalar<<<1, 1, 0, st>>>(g->d_sd, SC_TPREV, t0);
    k3_set_scalar<<<1, 1, 0, st>>>(g->d_sd, SC_NONFINITE, 0.0);
    k3_set_scalar<<<1, 1, 0, st>>>(g->d_sd, SC_NFAIL, 0.0);
    C3CU(cudaMemcpyAsync(g->fa, d_v, sizeof(float) * g->C.n_vox, cudaMemcpyDeviceToDevice, st));
    if ((rc = c3_p2(g, p, g->fa, d_f, st))) return rc;
    double sc[kScalarStride];
    if ((rc = c3_read_sc(g, sc, st))) return rc;
    if (sc[SC_NONFINITE] != 0.0) return c3_fail(EPTV_ERR_NONFINITE, "non-finite value in the (P2) solve");
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
    return 0;
}

int eptv3_reconstruct(const eptv3_geometry *g, const eptv_params *p, const float *d_y, float *d_f,
                      eptv_report *rep_opt, void *stream) {
    if (!g || !d_y || !d_f) return c3_fail(EPTV_ERR_ARG, "NULL argument");
    int rc = check_params(p);
    if (rc) return rc;
    if (p->weights_mode == EPTV_WEIGHTS_PRIOR) return c3_fail(EPTV_ERR_ARG, "PRIOR weights are 2-D only");
    cudaStream_t st = (cudaStream_t)stream;
    const long long nv = g->C.n_vox;
    if ((rc = c3_upload_params(g, p, st))) return rc;
    C3CU(cudaMemcpyAsync(g->y, d_y, sizeof(float) * g->C.n_rays, cudaMemcpyDeviceToDevice, st));
    C3CU(cudaMemcpyAsync(g->u, d_f, sizeof(float) * nv, cudaMemcpyDeviceToDevice, st));
    k3_clamp<<<nblk_of(nv, 256), 256, 0, st>>>(g->u, nv);
    k3_set_scalar<<<1, 1, 0, st>>>(g->d_sd, SC_TPREV, p->t_init > 0.0 ? p->t_init : 1.0 / p->lambda);
    k3_set_scalar<<<1, 1, 0, st>>>(g->d_sd, SC_NONFINITE, 0.0);
    k3_set_scalar<<<1, 1, 0, st>>>(g->d_sd, SC_NFAIL, 0.0);
    for (int k = 0; k < p->n_outer; ++k) {
        c3_cgls(g, p->cgls_iters, st);                                   // v = CGLS_M(u) in u
        C3CU(cudaMemcpyAsync(g->fa, g->u, sizeof(float) * nv, cudaMemcpyDeviceToDevice, st));
        if ((rc = c3_p2(g, p, g->fa, g->u, st))) return rc;              // (P2) + clamp -> u
    }
    C3CU(cudaMemcpyAsync(d_f, g->u, sizeof(float) * nv, cudaMemcpyDeviceToDevice, st));
    if (rep_opt) {
        double sc[kScalarStride];
        if ((rc = c3_read_sc(g, sc, st))) return rc;
        if (sc[SC_NONFINITE] != 0.0) return c3_fail(EPTV_ERR_NONFINITE, "non-finite value during the reconstruction");
        rep_opt->n_outer = p->n_outer;
        rep_opt->sigma_last = sc[SC_SIGMA];
        rep_opt->t_prev = sc[SC_TPREV];
        rep_opt->n_fail = (int)sc[SC_NFAIL];
        rep_opt->status = rep_opt->n_fail ? EPTV_WARN_LINESEARCH : EPTV_OK;
        rep_opt->n_launches = 0;
    }
    return 0;
}

int eptv3_report_energy(const eptv3_geometry *g, const eptv_params *p, double sigma_ref, const float *d_f,
                        const float *d_y, double *h_energy, void *stream) {
    if (!g || !d_f || !d_y || !h_energy) return c3_fail(EPTV_ERR_ARG, "NULL argument");
    int rc = check_params(p);
    if (rc) return rc;
    if (!(sigma_ref > 0.0)) return c3_fail(EPTV_ERR_ARG, "sigma_ref must be > 0");
    cudaStream_t st = (cudaStream_t)stream;
    c3_project(g, d_f, d_y, g->q, FIN_NORM, st);                         // |y - P f|^2 -> SC_NORM
    k3_set_scalar<<<1, 1, 0, st>>>(g->d_sd, SC_SIGMA, sigma_ref);
    const int mode = p->weights_mode == EPTV_WEIGHTS_ONE ? EPTV_WEIGHTS_ONE : EPTV_WEIGHTS_EPTV;
    // J at f (k3tv_grad with v = f; its g goes to the workspace)
    const long long n_items = (long long)g->V.nx * g->V.ny * ((g->V.nz + kZChunk - 1) / kZChunk);
    k3tv_grad<<<nblk_capped(n_items, 256, g->red_blocks), 256, 0, st>>>(g->V, d_f, d_f, (float)(p->eps * p->eps), mode,
                                                                         (float)p->lambda, g->g, g->partials, g->d_sd);
    C3CU(cudaGetLastError());
    double sc[kScalarStride];
    if ((rc = c3_read_sc(g, sc, st))) return rc;
    *h_energy = 0.5 * p->mu * sc[SC_NORM] + sc[SC_Q0];
    return 0;
}

}  // extern "C"
