// K1: fan-beam forward projection y = P f (Eq. 1), p_ij = exact intersection length of
// ray i with pixel j (Siddon, Sec. 2.1), one ray per lane, ray-driven gather.
//
// B300 layout: a block is 32 adjacent bins of one view (one per lane) times SEG warps;
// warp w marches rows [r_w, r_{w+1}) of its lane's ray.  Adjacent bins of one view are
// ~0.7 pixel apart, so the 32 lanes of a warp read a narrow band of one image row per
// step (1-2 cache lines): the gather is coalesced without staging.  Rays that cross
// columns faster than rows ("shallow") march over columns instead, reading the
// transposed copy of the image when the producer kernel wrote one.
//
// Per row the march visits at most two pixels (three only for a ray within rounding of
// 45 degrees, where the third piece is an FP32 sliver and is dropped): the segment
// lengths are min(exit planes) - max(entry planes) with the canonical plane
// parameters of eptv_internal.cuh, bit-identical to the back projector's.
// The SEG partial sums of a ray are combined in shared memory in a fixed order.
#include <type_traits>

#include "eptv_internal.cuh"
#include "kernels.cuh"

namespace eptv {

// HAS_T: the launch supplies the transposed image (every call of the CGLS does), so a
// shallow ray marches over the transposed copy and the column stride is 1 for every ray.
// At most 64 registers (8 blocks of 4 warps per SM): SEG = 4 then fits the 512^2
// workload's 1120 blocks in one wave, with no spills.
template <int SEG, bool HAS_T>
__global__ void __launch_bounds__(32 * SEG, 32 / SEG)
k1_project(const SliceDev *__restrict__ sls, TileMap map, ProjArgs a, double *__restrict__ partials)
{
    pdl_wait();
    __shared__ float red[SEG][33];
    __shared__ double rsm[2 * SEG];
    __shared__ double res[2];
    __shared__ int last_flag;

    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const int nb = S.nb;
    const double gamma_pre = threadIdx.x == 0 ? fin_gamma(S.sc, a.fin) : 0.0;
    const int nbb = (nb + 31) >> 5;
    // work unit (view, group of 32 bins) of this block: heaviest first, so that the blocks
    // dispatched last are the short ones and the SMs finish together
    const int unit = S.k1_order ? __ldg(S.k1_order + local) : local;
    const int v = unit / nbb;
    const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
    const int k = (unit - v * nbb) * 32 + lane;

    const float *img, *imgT;
    float *out;
    if (a.img_override) { img = a.img_override; imgT = a.imgT_override; }
    else if (a.img == IMG_U) { img = S.u; imgT = a.no_T ? nullptr : S.uT; }
    else { img = S.s; imgT = a.no_T ? nullptr : S.sT; }
    if (a.out_override) out = a.out_override;
    else out = (a.out == SINO_R) ? S.r : S.q;

    float acc = 0.0f;
    RayRec R = {0.0f, 0.0f, 0.0f, 0.0f};
    bool lane_sliver = false;
    if (k < nb) {
        R = S.ray[v * nb + k];
        // a second column crossing within one row (an FP32 sliver) needs a ray within
        // rounding of the diagonal: columns crossed per row = |iM| dM / (|im| dm) >= 0.99
        const float cx = fabsf(R.ix) * S.dx, cy = fabsf(R.iy) * S.dy;
        lane_sliver = fminf(cx, cy) >= 0.99f * fmaxf(cx, cy);
    }
    const bool any_sliver = __any_sync(0xffffffffu, lane_sliver);   // warp-uniform branch below
    if (k < nb) {
        const bool steep = fabsf(R.ix) * S.dx >= fabsf(R.iy) * S.dy;
        float PM, iM, M0, dM, Pm, im, m0, dm;
        int nM, nm;
        const float *base;
        int sM, sm;
        if (steep) {
            PM = R.py; iM = R.iy; M0 = S.y0; dM = S.dy; nM = S.ny;
            Pm = R.px; im = R.ix; m0 = S.x0; dm = S.dx; nm = S.nx;
            base = img; sM = S.nx; sm = 1;
        } else {
            PM = R.px; iM = R.ix; M0 = S.x0; dM = S.dx; nM = S.nx;
            Pm = R.py; im = R.iy; m0 = S.y0; dm = S.dy; nm = S.ny;
            if (HAS_T) { base = imgT; sM = S.ny; sm = 1; }
            else { base = img; sM = 1; sm = S.nx; }
        }
        if (iM < 0.0f) { iM = -iM; im = -im; }   // march with t increasing along the major axis
        const int sgn = (im > 0.0f) ? 1 : -1;
        const int off_hi = sgn > 0 ? 1 : 0, off_lo = 1 - off_hi;

        // ray's parameter range inside the minor-axis slab of the image
        const float tmA = cross_t(grid_line(0.0f, dm, m0), Pm, im);
        const float tmB = cross_t(grid_line((float)nm, dm, m0), Pm, im);
        const float tm_lo = fminf(tmA, tmB), tm_hi = fmaxf(tmA, tmB);
        const float tM0 = cross_t(grid_line(0.0f, dM, M0), PM, iM);
        const float tMn = cross_t(grid_line((float)nM, dM, M0), PM, iM);
        const float dMinv = 1.0f / iM;           // major direction component (> 0)
        const float dmdir = 1.0f / im;

        if (tm_hi > tM0 && tm_lo < tMn && tm_lo < tm_hi) {
            // row containing parameter t: largest r in [0, nM-1] with t_M(r) <= t
            auto row_of = [&](float t) {
                int r = (int)floorf(__fdividef(PM + t * dMinv - M0, dM));
                r = min(max(r, 0), nM - 1);
                for (int it = 0; it < 4 && r > 0 && cross_t(grid_line((float)r, dM, M0), PM, iM) > t; ++it) --r;
                for (int it = 0; it < 4 && r < nM - 1 && cross_t(grid_line((float)(r + 1), dM, M0), PM, iM) <= t; ++it) ++r;
                return r;
            };
            const int r_first = (tm_lo <= tM0) ? 0 : row_of(tm_lo);
            const int r_last = (tm_hi >= tMn) ? nM - 1 : row_of(tm_hi);
            const int nr = r_last - r_first + 1;
            const int chunk = (nr + SEG - 1) / SEG;
            const int rs = r_first + seg * chunk;
            const int re = min(rs + chunk - 1, r_last);
            if (rs <= re) {
                float ta = cross_t(grid_line((float)rs, dM, M0), PM, iM);
                const float t_start = fmaxf(ta, tm_lo);
                // column containing t_start: lo(c) <= t_start < hi(c)
                int c = (int)floorf(__fdividef(Pm + t_start * dmdir - m0, dm));
                c = min(max(c, 0), nm - 1);
                for (int it = 0; it < 4; ++it) {
                    const float lo = cross_t(grid_line((float)(c + off_lo), dm, m0), Pm, im);
                    const int cn = c - sgn;
                    if (lo > t_start && cn >= 0 && cn < nm) c = cn; else break;
                }
                for (int it = 0; it < 4; ++it) {
                    const float hi = cross_t(grid_line((float)(c + off_hi), dm, m0), Pm, im);
                    const int cn = c + sgn;
                    if (hi <= t_start && cn >= 0 && cn < nm) c = cn; else break;
                }
                float lo0 = cross_t(grid_line((float)(c + off_lo), dm, m0), Pm, im);
                float hi0 = cross_t(grid_line((float)(c + off_hi), dm, m0), Pm, im);
                float fr = (float)(rs + 1);
                const float fsgn = (float)sgn;
                float f1 = (float)(c + sgn + off_hi);     // plane beyond the next column (exact)
                const float *rowp = base + (size_t)rs * sM;
                // The row interval is clipped to the image's minor-axis extent
                // [tm_lo, tm_hi]: a column inside the image has both planes inside that
                // extent, so its length is bit-identical to the unclipped slab formula,
                // and a column outside the image gets length exactly 0 -- so the column
                // index only needs clamping for the address.
                float tac = fmaxf(ta, tm_lo);
                // one row of the march: lengths of the (at most) two columns the ray
                // crosses in this row and their offsets from the row start.  SLIVER: the
                // warp holds a ray within rounding of the diagonal, which can cross a
                // second column plane inside one row (without one, that cannot happen:
                // the columns crossed per row are below 0.99, far beyond FP32 error)
                auto step = [&](auto sliver, float &l0, float &l1, int &o0, int &o1) {
                    const float tb = cross_t(grid_line(fr, dM, M0), PM, iM);
                    const float tbc = fminf(tb, tm_hi);
                    fr += 1.0f;
                    const int c1 = c + sgn;
                    const float hi1 = cross_t(grid_line(f1, dm, m0), Pm, im);
                    l0 = seg_len(lo0, hi0, tac, tbc);
                    l1 = seg_len(hi0, hi1, tac, tbc);
                    o0 = min(max(c, 0), nm - 1) * sm;
                    o1 = c1 * sm;                // used only when l1 > 0 (column inside)
                    if (hi0 < tb) {
                        c = c1; lo0 = hi0; hi0 = hi1; f1 += fsgn;
                        if (decltype(sliver)::value && hi1 < tb) {   // FP32 sliver near 45 degrees
                            c += sgn; lo0 = hi1;
                            hi0 = cross_t(grid_line((float)(c + off_hi), dm, m0), Pm, im);
                            f1 += fsgn;
                        }
                    }
                    tac = fmaxf(tb, tm_lo);
                };
                // rows in groups of kRows: the plane arithmetic of the group first, then
                // all its gathers (independent, in flight together), then the products
                // in row order (the same sum as a row-by-row march)
                auto march = [&](auto sliver) {
                    constexpr int kRows = 4;
                    int r = rs;
                    for (; r + kRows - 1 <= re; r += kRows) {
                        float l0[kRows], l1[kRows], v0[kRows], v1[kRows];
                        int o0[kRows], o1[kRows];
#pragma unroll
                        for (int u = 0; u < kRows; ++u) step(sliver, l0[u], l1[u], o0[u], o1[u]);
#pragma unroll
                        for (int u = 0; u < kRows; ++u) {
                            v0[u] = __ldg(rowp + u * sM + o0[u]);
                            v1[u] = 0.0f;
                            if (l1[u] > 0.0f) v1[u] = __ldg(rowp + u * sM + o1[u]);
                        }
#pragma unroll
                        for (int u = 0; u < kRows; ++u) {
                            acc = fmaf(l0[u], v0[u], acc);
                            acc = fmaf(l1[u], v1[u], acc);
                        }
                        rowp += kRows * sM;
                    }
                    for (; r <= re; ++r) {
                        float l0, l1;
                        int o0, o1;
                        step(sliver, l0, l1, o0, o1);
                        const float v0 = __ldg(rowp + o0);
                        float v1 = 0.0f;
                        if (l1 > 0.0f) v1 = __ldg(rowp + o1);
                        acc = fmaf(l0, v0, acc);
                        acc = fmaf(l1, v1, acc);
                        rowp += sM;
                    }
                };
                if (any_sliver) march(std::true_type{});
                else march(std::false_type{});
            }
        }
    }

    red[seg][lane] = acc;
    __syncthreads();
    float sq = 0.0f, ysum = 0.0f;
    if (seg == 0) {
        float tot = 0.0f;
#pragma unroll
        for (int w = 0; w < SEG; ++w) tot += red[w][lane];
        if (k < nb) {
            const int idx = v * nb + k;
            float o = tot;
            if (a.resid) o = __ldg((a.y_override ? a.y_override : S.y) + idx) - tot;
            out[idx] = o;
            sq = o * o;
            ysum = o;
        }
    }
    if (a.fin == FIN_NONE) return;

    // block reduction of |out|^2 (warp 0 holds the values)
    const int nblk = __ldg(map.start + si + 1) - __ldg(map.start + si);
    const int b0 = __ldg(map.start + si);
    if (seg == 0) {
        float s1 = warp_sum(sq), s2 = warp_sum(ysum);
        if (lane == 0) {
            partials[(size_t)blockIdx.x * 2 + 0] = (double)s1;
            partials[(size_t)blockIdx.x * 2 + 1] = (double)s2;
        }
    }
    if (!reduce_slice<2, 32 * SEG>(S, partials, 2, b0, nblk, local, rsm, res, &last_flag)) return;
    if (threadIdx.x == 0) finalize(S.sc, a.fin, res[0], res[1], gamma_pre);
}

void launch_project(const Batch &B, const ProjArgs &a, cudaStream_t st) {
    const int nblk = B.blocks(FAM_K1);
    if (nblk == 0) return;
    ++g_launch_count;
    // the kernel reads the transposed image exactly when this holds
    const bool has_t = a.img_override ? (a.imgT_override != nullptr) : !a.no_T;
    const TileMap m = B.map(FAM_K1);
#define K1_LAUNCH(SEGv)                                                                            \
    (has_t ? launch_pdl(k1_project<SEGv, true>, nblk, 32 * SEGv, 0, st, B.d_sd, m, a, B.d_partials) \
           : launch_pdl(k1_project<SEGv, false>, nblk, 32 * SEGv, 0, st, B.d_sd, m, a, B.d_partials))
    switch (B.k1_seg) {
    case 4: K1_LAUNCH(4); break;
    case 16: K1_LAUNCH(16); break;
    default: K1_LAUNCH(8); break;
    }
#undef K1_LAUNCH
}

}  // namespace eptv
