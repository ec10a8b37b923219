// K2: f = P^T y, the exact transpose of the projector, as a scatter-free pixel-driven
// gather (the paper rejects the ray-driven scatter for its write conflicts, Sec. 2.3).
//
// A block covers a kTileW x kTileH (32 x 8) pixel tile, so a 512^2 image gives ~7 tiles
// per SM (an even share in one wave).  A thread owns a 4 x kRowsPT pixel block (float4
// rows) and every VG-th view; the VG partial sums of a block are added in group order
// (deterministic).  For every view the thread bounds the fan angles of its block from
// the block's corners (tan-space min/max, then atan), visits the bins whose rays can
// cross it, and recomputes each p_ij with the canonical plane parameters of
// eptv_internal.cuh -- the same FP32 operations as the projector, so <P x, y> =
// <x, P^T y> holds up to summation order.  The 5 column planes and kRowsPT + 1 row planes
// of a candidate ray are shared by the block's pixels.  Optionally also writes the
// transposed image (for the projector's shallow rays) and reduces |f|^2.
//
// EQ11 = true: the paper's pixel-driven back projector instead (Eq. 11, Sec. 2.3,
// derived in App. III), an approximation of the transpose:
//   [P^T y](u, v) = (du dv / dbeta) sum_theta y^theta(beta*) / l(u, v),
// beta* = fan angle of the line from the source through the pixel centre, l its length,
// y linearly interpolated between the two bins around beta* (bins off the detector read
// 0).  Flat detector (bins uniform in t = tan beta): weight (du dv / dt) (1 + t*^2) / l.
#include "eptv_internal.cuh"
#include "kernels.cuh"

namespace eptv {

constexpr int kRowsPT = 2;                                   // pixel rows per thread
constexpr int kBlocksPT = (kTileW / 4) * (kTileH / kRowsPT);  // 4 x kRowsPT blocks per tile

template <int VG, bool EQ11>
__global__ void __launch_bounds__(kBlocksPT * VG, EQ11 ? 0 : 1024 / (kBlocksPT * VG))
k2_backproject(const SliceDev *__restrict__ sls, TileMap map, BackArgs a, double *__restrict__ partials)
{
    pdl_wait();
    constexpr int NT = kBlocksPT * VG, R = kRowsPT;
    __shared__ float4 part[VG > 1 ? VG - 1 : 1][R][kBlocksPT];
    __shared__ float tr[kTileH][kTileW + 1];
    __shared__ double rsm[2 * (NT / 32)];
    __shared__ double res[2];
    __shared__ int last_flag;

    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const int nx = S.nx, ny = S.ny, nb = S.nb;
    const double gamma_pre = threadIdx.x == 0 ? fin_gamma(S.sc, a.fin) : 0.0;
    const int tiles_x = (nx + kTileW - 1) / kTileW;
    const int tyb = local / tiles_x, txb = local - tyb * tiles_x;
    const int blk = threadIdx.x % kBlocksPT, vg = threadIdx.x / kBlocksPT;
    const int lx = blk % (kTileW / 4), ly = blk / (kTileW / 4);
    const int i0 = txb * kTileW + lx * 4, j0 = tyb * kTileH + ly * R;

    const float *sino = a.in_override ? a.in_override : S.r;
    float acc[R][4];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = 0.0f;

    if (EQ11 && j0 < ny && i0 < nx) {
        float xc[4], yc[R];
#pragma unroll
        for (int q = 0; q < 4; ++q) xc[q] = grid_line((float)(i0 + q) + 0.5f, S.dx, S.x0);
#pragma unroll
        for (int r = 0; r < R; ++r) yc[r] = grid_line((float)(j0 + r) + 0.5f, S.dy, S.y0);
        const float inv_db = S.inv_dbeta, kc = S.kc;
        const bool arc = S.detector == EPTV_DETECTOR_ARC;
        for (int v = vg; v < S.nv; v += VG) {
            const ViewRec V = S.view[v];
            const float *sv = sino + (size_t)v * nb;
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float wx = xc[q] - V.sx, wy = yc[r] - V.sy;
                const float cr = V.cx * wy - V.cy * wx;          // l sin(beta*)
                const float dt = V.cx * wx + V.cy * wy;          // l cos(beta*)
                const float rl = rsqrtf(wx * wx + wy * wy);       // 1 / l
                float u, w;
                if (arc) {
                    u = atan2f(cr, dt) * inv_db + kc;
                    w = rl;
                } else {
                    const float t = __fdividef(cr, dt);
                    u = t * inv_db + kc;
                    w = fmaf(t, t, 1.0f) * rl;
                }
                if (dt > 0.0f && u > -1.0f && u < (float)nb) {
                    const float fk = floorf(u);
                    const int k0 = (int)fk;
                    const float fr = u - fk;
                    float y0 = 0.0f, y1 = 0.0f;
                    if (k0 >= 0) y0 = __ldg(sv + k0);
                    if (k0 + 1 < nb) y1 = __ldg(sv + k0 + 1);
                    acc[r][q] = fmaf(fmaf(fr, y1 - y0, y0), w, acc[r][q]);
                }
            }
        }
        const float scale = S.dx * S.dy * inv_db;
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[r][q] *= scale;
    }
    if (!EQ11 && j0 < ny && i0 < nx) {
        float X[5], Y[R + 1];
#pragma unroll
        for (int q = 0; q < 5; ++q) X[q] = grid_line((float)(i0 + q), S.dx, S.x0);
#pragma unroll
        for (int r = 0; r <= R; ++r) Y[r] = grid_line((float)(j0 + r), S.dy, S.y0);
        // corners of the block's part inside the image (pixels beyond the edge are not
        // written, so their bins need not be visited)
        const float Xe = grid_line((float)(i0 + min(4, nx - i0)), S.dx, S.x0);
        const float Ye = grid_line((float)(j0 + min(R, ny - j0)), S.dy, S.y0);
        const float inv_db = S.inv_dbeta, kc = S.kc;
        const bool arc = S.detector == EPTV_DETECTOR_ARC;

        for (int v = vg; v < S.nv; v += VG) {
            const ViewRec V = S.view[v];
            // tan of the fan angle of each corner as seen from the source
            float tmin = 3.0e38f, tmax = -3.0e38f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float px = (c & 1) ? Xe : X[0];
                const float py = (c & 2) ? Ye : Y[0];
                const float wx = px - V.sx, wy = py - V.sy;
                const float num = V.cx * wy - V.cy * wx;
                const float den = V.cx * wx + V.cy * wy;
                const float tt = __fdividef(num, den);
                tmin = fminf(tmin, tt);
                tmax = fmaxf(tmax, tt);
            }
            float ulo, uhi;
            if (arc) { ulo = atanf(tmin) * inv_db + kc; uhi = atanf(tmax) * inv_db + kc; }
            else { ulo = tmin * inv_db + kc; uhi = tmax * inv_db + kc; }
            const int klo = max(0, (int)ceilf(ulo - 0.01f));
            const int khi = min(nb - 1, (int)floorf(uhi + 0.01f));
            const RayRec *rr = S.ray + (size_t)v * nb;
            const float *sv = sino + (size_t)v * nb;
            for (int k = klo; k <= khi; ++k) {
                const RayRec Rr = rr[k];
                const float yv = __ldg(sv + k);
                float ty[R + 1], tx[5];
#pragma unroll
                for (int r = 0; r <= R; ++r) ty[r] = cross_t(Y[r], Rr.py, Rr.iy);
#pragma unroll
                for (int q = 0; q < 5; ++q) tx[q] = cross_t(X[q], Rr.px, Rr.ix);
                // the column planes clamped to the row's slab [rlo, rhi]: pixel q's length
                // |c[q + 1] - c[q]| is bit for bit seg_len(min, max of tx[q], tx[q + 1],
                // rlo, rhi) (where the column meets the slab its clamped planes are those
                // min / max, elsewhere both clamp to one bound) -- 5 clamps per row
                // instead of two min / max pairs per pixel
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float rlo = fminf(ty[r], ty[r + 1]), rhi = fmaxf(ty[r], ty[r + 1]);
                    float c[5];
#pragma unroll
                    for (int q = 0; q < 5; ++q) c[q] = fminf(fmaxf(tx[q], rlo), rhi);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        acc[r][q] = fmaf(fabsf(__fsub_rn(c[q + 1], c[q])), yv, acc[r][q]);
                }
            }
        }
    }

    // combine the view groups in order (group 0 owns the block's output)
    if (VG > 1) {
        if (vg > 0) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                part[vg - 1][r][blk] = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
        }
        __syncthreads();
        if (vg == 0) {
#pragma unroll
            for (int gi = 0; gi < VG - 1; ++gi)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float4 p = part[gi][r][blk];
                    acc[r][0] += p.x; acc[r][1] += p.y; acc[r][2] += p.z; acc[r][3] += p.w;
                }
        }
    }

    float *out;
    float *outT = nullptr;
    if (a.out_override) out = a.out_override;
    else if (a.out == 0) { out = S.s; if (a.write_T) outT = S.sT; }
    else if (a.out == 1) out = S.t;
    else { out = S.u; if (a.write_T) outT = S.uT; }

    float sq = 0.0f;
    if (vg == 0 && i0 < nx) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = j0 + r;
            if (j >= ny) break;
            float *p = out + (size_t)j * nx + i0;
            if (i0 + 3 < nx && ((nx & 3) == 0) && ((((uintptr_t)p) & 15) == 0)) {
                *reinterpret_cast<float4 *>(p) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) if (i0 + q < nx) p[q] = acc[r][q];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) if (i0 + q < nx) sq = fmaf(acc[r][q], acc[r][q], sq);
        }
    }
    if (outT) {
        if (vg == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) tr[ly * R + r][lx * 4 + q] = acc[r][q];
        }
        __syncthreads();
        constexpr int kRowGroups = kTileH / 4;          // 4 rows of one column per thread
        for (int idx = threadIdx.x; idx < kTileW * kRowGroups; idx += NT) {
            const int ii = idx / kRowGroups, jj0 = (idx % kRowGroups) * 4;
            const int gi = txb * kTileW + ii;
            if (gi < nx) {
                for (int q = 0; q < 4; ++q) {
                    const int gj = tyb * kTileH + jj0 + q;
                    if (gj < ny) outT[(size_t)gi * ny + gj] = tr[jj0 + q][ii];
                }
            }
        }
    }
    if (a.fin == FIN_NONE) return;

    const int b0 = __ldg(map.start + si);
    const int nblk = __ldg(map.start + si + 1) - b0;
    float vals[1] = {sq};
    block_sum_to<1, NT>(vals, partials + (size_t)blockIdx.x * 2, rsm);
    if (threadIdx.x == 0) partials[(size_t)blockIdx.x * 2 + 1] = 0.0;
    if (!reduce_slice<2, NT>(S, partials, 2, b0, nblk, local, rsm, res, &last_flag)) return;
    if (threadIdx.x == 0) finalize(S.sc, a.fin, res[0], res[1], gamma_pre);
}

void launch_backproject(const Batch &B, const BackArgs &a, cudaStream_t st) {
    const int nblk = B.blocks(FAM_K2);
    if (nblk == 0) return;
    ++g_launch_count;
    const TileMap m = B.map(FAM_K2);
    const bool eq11 = B.bp_eq11 || a.eq11;
#define K2_LAUNCH(VGv)                                                                                  \
    (eq11 ? launch_pdl(k2_backproject<VGv, true>, nblk, kBlocksPT * VGv, 0, st, B.d_sd, m, a, B.d_partials) \
          : launch_pdl(k2_backproject<VGv, false>, nblk, kBlocksPT * VGv, 0, st, B.d_sd, m, a, B.d_partials))
    switch (B.k2_vg) {
    case 1: K2_LAUNCH(1); break;
    case 2: K2_LAUNCH(2); break;
    case 8: K2_LAUNCH(8); break;
    case 16: K2_LAUNCH(16); break;
    default: K2_LAUNCH(4); break;
    }
#undef K2_LAUNCH
}

}  // namespace eptv
