// K3: CGLS vector updates (App. I).  The scalars a = |P^T r|^2 / |P s|^2 and
// b = |P^T r'|^2 / |P^T r|^2 are formed on the device by the reductions fused into the
// projector / back projector (FP64), so the whole (P1) loop runs without a host sync.
#include "eptv_internal.cuh"
#include "kernels.cuh"

namespace eptv {

thread_local long long g_launch_count = 0;

// r -= a q (step 3)
__global__ void __launch_bounds__(256)
k3_update_r(const SliceDev *__restrict__ sls, TileMap map)
{
    pdl_wait();
    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const float a = (float)S.sc[SC_A];
    const int base = local * 1024 + threadIdx.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = base + q * 256;
        if (i < S.n_rays) S.r[i] = fmaf(-a, S.q[i], S.r[i]);
    }
}

// u += a s (step 2); if update_s: s = t + b s (step 5) and the transposed copy of s.
__global__ void __launch_bounds__(256)
k3_update_us(const SliceDev *__restrict__ sls, TileMap map, int update_s)
{
    __shared__ float tile[32][33];
    pdl_wait();
    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const int nx = S.nx, ny = S.ny;
    const int tiles_x = (nx + 31) >> 5;
    const int tyb = local / tiles_x, txb = local - tyb * tiles_x;
    const float a = (float)S.sc[SC_A];
    const float b = (float)S.sc[SC_B];
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    const int i = txb * 32 + lx;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int jj = ly + 8 * q;
        const int j = tyb * 32 + jj;
        if (i < nx && j < ny) {
            const size_t p = (size_t)j * nx + i;
            const float s = S.s[p];
            S.u[p] = fmaf(a, s, S.u[p]);
            if (update_s) {
                const float sn = fmaf(b, s, S.t[p]);
                S.s[p] = sn;
                tile[jj][lx] = sn;
            }
        }
    }
    if (!update_s || S.sT == nullptr) return;
    __syncthreads();
    // transposed store: sT[i][j]
    const int jx = txb * 32;   // block's first column -> rows of sT
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int ii = ly + 8 * q;           // column within the tile
        const int gi = jx + ii;
        const int gj = tyb * 32 + lx;
        if (gi < nx && gj < ny) S.sT[(size_t)gi * ny + gj] = tile[lx][ii];
    }
}

void launch_cgls_update_r(const Batch &B, cudaStream_t st) {
    const int nblk = B.blocks(FAM_SINO);
    if (nblk) { ++g_launch_count; launch_pdl(k3_update_r, nblk, 256, 0, st, B.d_sd, B.map(FAM_SINO)); }
}

void launch_cgls_update_us(const Batch &B, int update_s, cudaStream_t st) {
    const int nblk = B.blocks(FAM_IMG);
    if (nblk) { ++g_launch_count; launch_pdl(k3_update_us, nblk, 256, 0, st, B.d_sd, B.map(FAM_IMG), update_s); }
}

// Small helpers: set one scalar of every slice; advance the outer-iteration counter.
__global__ void k_set_scalar(const SliceDev *__restrict__ sls, int n, int which, double value) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) sls[s].sc[which] = value;
}

void launch_set_scalar(const Batch &B, int which, double value, cudaStream_t st) {
    ++g_launch_count;
    k_set_scalar<<<(B.n + 63) / 64, 64, 0, st>>>(B.d_sd, B.n, which, value);
}

// dst = transpose of src ([ny][nx] -> [nx][ny]) for every slice (single-slice calls).
__global__ void __launch_bounds__(256)
k_transpose(const SliceDev *__restrict__ sls, TileMap map, const float *src, float *dst)
{
    __shared__ float tile[32][33];
    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const int nx = S.nx, ny = S.ny;
    const int tiles_x = (nx + 31) >> 5;
    const int tyb = local / tiles_x, txb = local - tyb * tiles_x;
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int jj = ly + 8 * q, j = tyb * 32 + jj, i = txb * 32 + lx;
        if (i < nx && j < ny) tile[jj][lx] = src[(size_t)j * nx + i];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int ii = ly + 8 * q;
        const int gi = txb * 32 + ii, gj = tyb * 32 + lx;
        if (gi < nx && gj < ny) dst[(size_t)gi * ny + gj] = tile[lx][ii];
    }
}

void launch_transpose(const Batch &B, const float *src, float *dst, cudaStream_t st) {
    const int nblk = B.blocks(FAM_IMG);
    if (nblk) { ++g_launch_count; k_transpose<<<nblk, 256, 0, st>>>(B.d_sd, B.map(FAM_IMG), src, dst); }
}

}  // namespace eptv
