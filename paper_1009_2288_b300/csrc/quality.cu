// Image-quality metrics of Sec. 3 (not part of the iteration; used to compare results):
//   Eq. (12)  relative error e = |f - f*|^2 / |f*|^2
//   Eq. (13)  edge correlation c of the binary Sobel edge maps of f and f*: an edge is an
//             interior pixel whose squared Sobel magnitude gx^2 + gy^2 exceeds
//             s^2 times its mean over the interior (no thinning)
//   Eq. (14)  SNR = 10 log10(E(P)^2 / E([P - E(P)]^2)) over a rectangle P of f
// Two launches over 32 x 32 tiles: the FP64 sums (squared error, |f*|^2, the two mean
// Sobel energies, the ROI moments), then the edge decisions and their counts.  The Sobel
// magnitudes are formed in FP64 from the FP32 pixels with explicitly rounded operations in
// a fixed order, so an edge decision is the same as an FP64 evaluation of the definition.
#include <math.h>

#include "eptv_internal.cuh"
#include "kernels.cuh"

namespace eptv {

// gx^2 + gy^2 at interior pixel (i, j), FP64: gx = (f[j-1][i+1] + 2 f[j][i+1] + f[j+1][i+1])
// - (f[j-1][i-1] + 2 f[j][i-1] + f[j+1][i-1]), gy likewise along the columns.
__device__ __forceinline__ double sobel2(const float *__restrict__ f, int nx, int i, int j) {
    auto at = [&](int ii, int jj) { return (double)__ldg(f + (size_t)jj * nx + ii); };
    const double gx = __dsub_rn(__dadd_rn(__dadd_rn(at(i + 1, j - 1), __dmul_rn(2.0, at(i + 1, j))), at(i + 1, j + 1)),
                                __dadd_rn(__dadd_rn(at(i - 1, j - 1), __dmul_rn(2.0, at(i - 1, j))), at(i - 1, j + 1)));
    const double gy = __dsub_rn(__dadd_rn(__dadd_rn(at(i - 1, j + 1), __dmul_rn(2.0, at(i, j + 1))), at(i + 1, j + 1)),
                                __dadd_rn(__dadd_rn(at(i - 1, j - 1), __dmul_rn(2.0, at(i, j - 1))), at(i + 1, j - 1)));
    return __dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy));
}

template <int NV>
__device__ __forceinline__ void block_sum_d(const double (&v)[NV], double *out, double *smem /* NV * 8 */) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double a = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) smem[k * 8 + w] = a;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double acc = 0.0;
        for (int i = 0; i < 8; ++i) acc += smem[threadIdx.x * 8 + i];
        out[threadIdx.x] = acc;
    }
}

// Pass 1: sums |f - r|^2, |r|^2, sum of Sobel energies of f and r over the interior,
// ROI sum and sum of squares of f -> sc[SC_Q0 .. SC_Q0 + 5].
__global__ void __launch_bounds__(256)
k_quality_sums(const SliceDev *__restrict__ sls, TileMap map, const float *__restrict__ f,
               const float *__restrict__ r, int rx0, int ry0, int rw, int rh, double *__restrict__ partials)
{
    __shared__ double rsm[6 * 8];
    __shared__ double res[6];
    __shared__ int last_flag;
    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const int nx = S.nx, ny = S.ny;
    const int tiles_x = (nx + 31) >> 5;
    const int tyb = local / tiles_x, txb = local - tyb * tiles_x;
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = txb * 32 + lx, j = tyb * 32 + ly + 8 * q;
        if (i >= nx || j >= ny) continue;
        const double fv = (double)__ldg(f + (size_t)j * nx + i);
        const bool interior = i > 0 && j > 0 && i < nx - 1 && j < ny - 1;
        if (r) {
            const double rv = (double)__ldg(r + (size_t)j * nx + i);
            const double d = fv - rv;
            v[0] += d * d;
            v[1] += rv * rv;
            if (interior) v[3] += sobel2(r, nx, i, j);
        }
        if (interior) v[2] += sobel2(f, nx, i, j);
        if (i >= rx0 && i < rx0 + rw && j >= ry0 && j < ry0 + rh) {
            v[4] += fv;
            v[5] += fv * fv;
        }
    }
    const int b0 = __ldg(map.start + si);
    const int nblk = __ldg(map.start + si + 1) - b0;
    block_sum_d<6>(v, partials + (size_t)blockIdx.x * kPartialStride, rsm);
    if (!reduce_slice<6, 256>(S, partials, kPartialStride, b0, nblk, local, rsm, res, &last_flag)) return;
    if (threadIdx.x < 6) S.sc[SC_Q0 + threadIdx.x] = res[threadIdx.x];
}

// Pass 2: edge maps with thresholds scale2 x (mean Sobel energy of pass 1); counts of
// edges of f, of r and of both -> sc[SC_Q0 + 6 .. SC_Q0 + 8]; optional byte maps.
__global__ void __launch_bounds__(256)
k_quality_edges(const SliceDev *__restrict__ sls, TileMap map, const float *__restrict__ f,
                const float *__restrict__ r, double scale2, unsigned char *__restrict__ bf,
                unsigned char *__restrict__ br, double *__restrict__ partials)
{
    __shared__ double rsm[3 * 8];
    __shared__ double res[3];
    __shared__ int last_flag;
    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const int nx = S.nx, ny = S.ny;
    const double n_int = (double)(nx - 2) * (double)(ny - 2);
    const double tf = scale2 * (S.sc[SC_Q0 + 2] / n_int);
    const double tr = scale2 * (S.sc[SC_Q0 + 3] / n_int);
    const int tiles_x = (nx + 31) >> 5;
    const int tyb = local / tiles_x, txb = local - tyb * tiles_x;
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    double v[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = txb * 32 + lx, j = tyb * 32 + ly + 8 * q;
        if (i >= nx || j >= ny) continue;
        const bool interior = i > 0 && j > 0 && i < nx - 1 && j < ny - 1;
        const bool ef = interior && sobel2(f, nx, i, j) > tf;
        const bool er = r && interior && sobel2(r, nx, i, j) > tr;
        v[0] += ef ? 1.0 : 0.0;
        v[1] += er ? 1.0 : 0.0;
        v[2] += (ef && er) ? 1.0 : 0.0;
        if (bf) bf[(size_t)j * nx + i] = ef ? 1 : 0;
        if (br) br[(size_t)j * nx + i] = er ? 1 : 0;
    }
    const int b0 = __ldg(map.start + si);
    const int nblk = __ldg(map.start + si + 1) - b0;
    block_sum_d<3>(v, partials + (size_t)blockIdx.x * kPartialStride, rsm);
    if (!reduce_slice<3, 256>(S, partials, kPartialStride, b0, nblk, local, rsm, res, &last_flag)) return;
    if (threadIdx.x < 3) S.sc[SC_Q0 + 6 + threadIdx.x] = res[threadIdx.x];
}

void launch_quality(const Batch &B, const float *f, const float *r, int rx0, int ry0, int rw, int rh,
                    double scale2, unsigned char *bf, unsigned char *br, cudaStream_t st) {
    const int nblk = B.blocks(FAM_IMG);
    if (nblk == 0) return;
    g_launch_count += 2;
    k_quality_sums<<<nblk, 256, 0, st>>>(B.d_sd, B.map(FAM_IMG), f, r, rx0, ry0, rw, rh, B.d_partials);
    k_quality_edges<<<nblk, 256, 0, st>>>(B.d_sd, B.map(FAM_IMG), f, r, scale2, bf, br, B.d_partials);
}

}  // namespace eptv
