// Stored-matrix operator (Sec. 2.3): for small problems the paper keeps P as a sparse
// matrix and applies P and P^T as sparse matrix-vector products.  Here both are built
// once per geometry, on the device, as CSR matrices whose nonzeros are the canonical
// p_ij of eptv_internal.cuh (the values the on-the-fly back projector K2 forms), and are
// applied by SpMV kernels that stream the matrix from HBM while the vector they gather
// from stays in L2.
//
// Layout of each matrix: ptr [rows + 1] (int32), col [nnz] (int32), val [nnz] (FP32).
// Every row is padded to a multiple of 4 entries (val 0, col = the row's last column) so
// that one lane reads 4 entries with one 16-byte load of each array.
//   P^T: rows = pixels j = iy nx + ix, columns = rays i = v nb + k in increasing order.
//   P:   rows = rays, columns = pixels in increasing order -- the exact transpose of P^T
//        (same values, same set of nonzeros), made by a counting transpose and a
//        per-row sort, so the layout does not depend on the order of atomic updates.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "eptv_internal.cuh"
#include "kernels.cuh"

namespace eptv {

// ---------------------------------------------------------------- build

// Row j of P^T: the rays of every view whose fan angle can reach pixel j (the corner
// bound of K2, 0.01 bins of margin), each with the canonical slab length; only lengths
// > 0 are kept.  FILL = false writes the padded row length, FILL = true the entries.
template <bool FILL>
__global__ void __launch_bounds__(256)
k_pt_rows(const SliceDev *__restrict__ sd, int *__restrict__ cnt, const int *__restrict__ ptr,
          int *__restrict__ col, float *__restrict__ val)
{
    const SliceDev &S = *sd;
    const int pix = blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= S.n_pix) return;
    const int iy = pix / S.nx, ix = pix - iy * S.nx;
    const float X0 = grid_line((float)ix, S.dx, S.x0), X1 = grid_line((float)(ix + 1), S.dx, S.x0);
    const float Y0 = grid_line((float)iy, S.dy, S.y0), Y1 = grid_line((float)(iy + 1), S.dy, S.y0);
    const bool arc = S.detector == EPTV_DETECTOR_ARC;
    const int nb = S.nb;
    int n = 0;
    const int base = FILL ? ptr[pix] : 0;
    const int cap = FILL ? ptr[pix + 1] - base : 0;     // the row's allocation
    int last = 0;
    for (int v = 0; v < S.nv; ++v) {
        const ViewRec V = S.view[v];
        float tmin = 3.0e38f, tmax = -3.0e38f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float px = (c & 1) ? X1 : X0;
            const float py = (c & 2) ? Y1 : Y0;
            // explicit roundings: the counting and the filling pass must enumerate the
            // same bins, whatever contraction the compiler would choose in each
            const float wx = __fsub_rn(px, V.sx), wy = __fsub_rn(py, V.sy);
            const float num = __fsub_rn(__fmul_rn(V.cx, wy), __fmul_rn(V.cy, wx));
            const float den = __fadd_rn(__fmul_rn(V.cx, wx), __fmul_rn(V.cy, wy));
            const float tt = __fdiv_rn(num, den);
            tmin = fminf(tmin, tt);
            tmax = fmaxf(tmax, tt);
        }
        float ulo, uhi;
        if (arc) {
            ulo = __fmaf_rn(atanf(tmin), S.inv_dbeta, S.kc);
            uhi = __fmaf_rn(atanf(tmax), S.inv_dbeta, S.kc);
        } else {
            ulo = __fmaf_rn(tmin, S.inv_dbeta, S.kc);
            uhi = __fmaf_rn(tmax, S.inv_dbeta, S.kc);
        }
        const int klo = max(0, (int)ceilf(ulo - 0.01f));
        const int khi = min(nb - 1, (int)floorf(uhi + 0.01f));
        for (int k = klo; k <= khi; ++k) {
            const RayRec R = S.ray[(size_t)v * nb + k];
            const float ta = cross_t(Y0, R.py, R.iy), tb = cross_t(Y1, R.py, R.iy);
            const float t0 = cross_t(X0, R.px, R.ix), t1 = cross_t(X1, R.px, R.ix);
            const float len = seg_len(fminf(t0, t1), fmaxf(t0, t1), fminf(ta, tb), fmaxf(ta, tb));
            if (len > 0.0f) {
                if (FILL && n < cap) {
                    col[base + n] = v * nb + k;
                    val[base + n] = len;
                }
                last = v * nb + k;
                ++n;
            }
        }
    }
    const int n4 = (n + 3) & ~3;
    if (FILL) {
        for (int q = n; q < min(n4, cap); ++q) { col[base + q] = last; val[base + q] = 0.0f; }
    } else {
        cnt[pix] = n4;
    }
}

// Exclusive prefix sum of n ints by one block (setup only): out[i] = sum in[0..i),
// out[n] = total; *total64 receives the total in 64 bits (the caller checks it fits).
__global__ void __launch_bounds__(1024)
k_scan_exclusive(const int *__restrict__ in, int *__restrict__ out, int n, long long *__restrict__ total64)
{
    __shared__ long long wsum[32];
    __shared__ long long carry_s;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 4096) {
        long long v[4], s = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = base + tid * 4 + q;
            v[q] = (i < n) ? (long long)in[i] : 0;
            s += v[q];
        }
        long long incl = s;          // inclusive scan of the thread sums
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            long long x = wsum[lane], xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long t = __shfl_up_sync(0xffffffffu, xi, o);
                if (lane >= o) xi += t;
            }
            wsum[lane] = xi - x;     // exclusive prefix of the warp sums
        }
        __syncthreads();
        long long run = carry_s + wsum[w] + incl - s;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = base + tid * 4 + q;
            if (i < n) out[i] = (int)run;
            run += v[q];
        }
        __syncthreads();
        if (tid == 1023) carry_s = run;
        __syncthreads();
    }
    if (tid == 0) {
        out[n] = (int)carry_s;
        *total64 = carry_s;
    }
}

// Nonzeros per column of P^T (= per row of P); padding entries have val 0.
__global__ void __launch_bounds__(256)
k_count_cols(int rows, const int *__restrict__ ptr, const int *__restrict__ col,
             const float *__restrict__ val, int *__restrict__ cnt)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    for (int e = ptr[r]; e < ptr[r + 1]; ++e)
        if (val[e] != 0.0f) atomicAdd(cnt + col[e], 1);
}

__global__ void __launch_bounds__(256)
k_pad4(int n, const int *__restrict__ cnt, int *__restrict__ cnt4)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cnt4[i] = (cnt[i] + 3) & ~3;
}

// Entry (r, c, v) of P^T goes to row c of P at ptrT[c] + (arrival order); each row is
// sorted afterwards.
__global__ void __launch_bounds__(256)
k_scatter_t(int rows, const int *__restrict__ ptr, const int *__restrict__ col,
            const float *__restrict__ val, const int *__restrict__ ptrT, int *__restrict__ cursor,
            int *__restrict__ colT, float *__restrict__ valT)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    for (int e = ptr[r]; e < ptr[r + 1]; ++e) {
        const float v = val[e];
        if (v == 0.0f) continue;
        const int c = col[e];
        const int pos = ptrT[c] + atomicAdd(cursor + c, 1);
        colT[pos] = r;
        valT[pos] = v;
    }
}

constexpr int kMaxStoredRow = 4096;

// One block per row of P: bitonic sort of the row's (column, value) pairs by column in
// shared memory, then the padding entries.
__global__ void __launch_bounds__(256)
k_sort_rows(int rows, const int *__restrict__ ptr, const int *__restrict__ cnt,
            int *__restrict__ col, float *__restrict__ val)
{
    __shared__ int key[kMaxStoredRow];
    __shared__ float sv[kMaxStoredRow];
    const int r = blockIdx.x;
    if (r >= rows) return;
    const int b = ptr[r], n = cnt[r], n4 = ptr[r + 1] - b;
    int N = 1;
    while (N < n) N <<= 1;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        key[i] = (i < n) ? col[b + i] : 0x7fffffff;
        sv[i] = (i < n) ? val[b + i] : 0.0f;
    }
    __syncthreads();
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool asc = (i & k) == 0;
                    if ((key[i] > key[ixj]) == asc) {
                        const int tk = key[i]; key[i] = key[ixj]; key[ixj] = tk;
                        const float tv = sv[i]; sv[i] = sv[ixj]; sv[ixj] = tv;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        col[b + i] = (i < n) ? key[i] : (n > 0 ? key[n - 1] : 0);
        val[b + i] = (i < n) ? sv[i] : 0.0f;
    }
}

// ---------------------------------------------------------------- SpMV

// y = P x: one warp per ray; each lane streams 4 entries per step (16-byte loads of col
// and val, evict-first), gathers x from L2, the warp sums in a fixed shuffle tree.
// Same output selection, residual mode and fused |out|^2 reduction as K1.
__global__ void __launch_bounds__(256)
k_spmv_p(const SliceDev *__restrict__ sls, TileMap map, ProjArgs a, unsigned int *__restrict__ counters,
         double *__restrict__ partials)
{
    __shared__ double rsm[2 * 8];
    __shared__ double res[2];
    __shared__ int last_flag;
    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = local * 8 + warp;
    const float *x = a.img_override ? a.img_override : (a.img == IMG_U ? S.u : S.s);
    float *out = a.out_override ? a.out_override : (a.out == SINO_R ? S.r : S.q);
    float sq = 0.0f, ysum = 0.0f;
    if (row < S.n_rays) {
        const int b = __ldg(S.p_ptr + row) >> 2, e = __ldg(S.p_ptr + row + 1) >> 2;
        const int4 *c4 = reinterpret_cast<const int4 *>(S.p_col);
        const float4 *v4 = reinterpret_cast<const float4 *>(S.p_val);
        float acc = 0.0f;
        for (int gi = b + lane; gi < e; gi += 32) {
            const int4 c = __ldcs(c4 + gi);
            const float4 v = __ldcs(v4 + gi);
            acc = fmaf(v.x, __ldg(x + c.x), acc);
            acc = fmaf(v.y, __ldg(x + c.y), acc);
            acc = fmaf(v.z, __ldg(x + c.z), acc);
            acc = fmaf(v.w, __ldg(x + c.w), acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            float o = acc;
            if (a.resid) o = __ldg((a.y_override ? a.y_override : S.y) + row) - acc;
            out[row] = o;
            sq = o * o;
            ysum = o;
        }
    }
    if (a.fin == FIN_NONE) return;
    const int b0 = __ldg(map.start + si);
    const int nblk = __ldg(map.start + si + 1) - b0;
    float vals[2] = {sq, ysum};
    block_sum_to<2, 256>(vals, partials + (size_t)blockIdx.x * 2, rsm);
    if (!last_block_of_slice(counters + si, nblk, &last_flag)) return;
    last_block_sum<2, 256>(partials, 2, b0, nblk, rsm, res);
    if (threadIdx.x == 0) finalize(S.sc, a.fin, res[0], res[1]);
}

// x = P^T y: 8 lanes per pixel row (rows hold ~2 rays per view), 32 pixels per block.
// Same output selection and fused |out|^2 reduction as K2 (no transposed copy: the
// stored operator never reads one).
__global__ void __launch_bounds__(256)
k_spmv_pt(const SliceDev *__restrict__ sls, TileMap map, BackArgs a, unsigned int *__restrict__ counters,
          double *__restrict__ partials)
{
    __shared__ double rsm[2 * 8];
    __shared__ double res[2];
    __shared__ int last_flag;
    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const int sub = threadIdx.x & 7;
    const int row = local * 32 + (threadIdx.x >> 3);
    const float *in = a.in_override ? a.in_override : S.r;
    float *out;
    if (a.out_override) out = a.out_override;
    else if (a.out == 0) out = S.s;
    else if (a.out == 1) out = S.t;
    else out = S.u;
    float acc = 0.0f;
    if (row < S.n_pix) {
        const int b = __ldg(S.pt_ptr + row) >> 2, e = __ldg(S.pt_ptr + row + 1) >> 2;
        const int4 *c4 = reinterpret_cast<const int4 *>(S.pt_col);
        const float4 *v4 = reinterpret_cast<const float4 *>(S.pt_val);
        for (int gi = b + sub; gi < e; gi += 8) {
            const int4 c = __ldcs(c4 + gi);
            const float4 v = __ldcs(v4 + gi);
            acc = fmaf(v.x, __ldg(in + c.x), acc);
            acc = fmaf(v.y, __ldg(in + c.y), acc);
            acc = fmaf(v.z, __ldg(in + c.z), acc);
            acc = fmaf(v.w, __ldg(in + c.w), acc);
        }
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    float sq = 0.0f;
    if (sub == 0 && row < S.n_pix) {
        out[row] = acc;
        sq = acc * acc;
    }
    if (a.fin == FIN_NONE) return;
    const int b0 = __ldg(map.start + si);
    const int nblk = __ldg(map.start + si + 1) - b0;
    float vals[1] = {sq};
    block_sum_to<1, 256>(vals, partials + (size_t)blockIdx.x * 2, rsm);
    if (threadIdx.x == 0) partials[(size_t)blockIdx.x * 2 + 1] = 0.0;
    if (!last_block_of_slice(counters + si, nblk, &last_flag)) return;
    last_block_sum<2, 256>(partials, 2, b0, nblk, rsm, res);
    if (threadIdx.x == 0) finalize(S.sc, a.fin, res[0], res[1]);
}

void launch_spmv_p(const Batch &B, const ProjArgs &a, cudaStream_t st) {
    const int nblk = B.blocks(FAM_SPMV_P);
    if (nblk == 0) return;
    ++g_launch_count;
    k_spmv_p<<<nblk, 256, 0, st>>>(B.d_sd, B.map(FAM_SPMV_P), a, B.d_counters, B.d_partials);
}

void launch_spmv_pt(const Batch &B, const BackArgs &a, cudaStream_t st) {
    const int nblk = B.blocks(FAM_SPMV_PT);
    if (nblk == 0) return;
    ++g_launch_count;
    k_spmv_pt<<<nblk, 256, 0, st>>>(B.d_sd, B.map(FAM_SPMV_PT), a, B.d_counters, B.d_partials);
}

// ---------------------------------------------------------------- build driver

static unsigned nb256(long long n) { return (unsigned)((n + 255) / 256); }

// Builds both matrices of the slice described by d_sd (device copy of `S`, whose ray and
// view tables are set).  Allocation goes through `alloc` (owned by the caller).  Returns
// cudaSuccess, or cudaErrorInvalidValue if a row of P is longer than kMaxStoredRow or the
// matrix has 2^31 or more stored entries.
cudaError_t build_stored(const SliceDev &S, const SliceDev *d_sd, StoredAlloc alloc, void *ctx,
                         StoredMatrices *m, cudaStream_t st) {
    const int n_pix = S.n_pix, n_rays = S.n_rays;
    int *cnt = nullptr, *cnt4 = nullptr, *cursor = nullptr;
    long long *tot = nullptr;
    cudaError_t e;
    long long h_tot = 0;
#define TRY(x) do { e = (x); if (e != cudaSuccess) goto done; } while (0)
    TRY(cudaMalloc(&cnt, sizeof(int) * (size_t)(std::max(n_pix, n_rays) + 1)));
    TRY(cudaMalloc(&cnt4, sizeof(int) * (size_t)(n_rays + 1)));
    TRY(cudaMalloc(&cursor, sizeof(int) * (size_t)n_rays));
    TRY(cudaMalloc(&tot, sizeof(long long)));
    // P^T: padded row lengths, offsets, entries
    TRY(alloc(ctx, (void **)&m->pt_ptr, sizeof(int) * ((size_t)n_pix + 1)));
    k_pt_rows<false><<<nb256(n_pix), 256, 0, st>>>(d_sd, cnt, nullptr, nullptr, nullptr);
    k_scan_exclusive<<<1, 1024, 0, st>>>(cnt, m->pt_ptr, n_pix, tot);
    TRY(cudaMemcpyAsync(&h_tot, tot, sizeof h_tot, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    if (h_tot >= (1LL << 31) - 4) { e = cudaErrorInvalidValue; goto done; }
    m->nnz_pt = h_tot;
    TRY(alloc(ctx, (void **)&m->pt_col, sizeof(int) * (size_t)std::max(h_tot, 4LL)));
    TRY(alloc(ctx, (void **)&m->pt_val, sizeof(float) * (size_t)std::max(h_tot, 4LL)));
    k_pt_rows<true><<<nb256(n_pix), 256, 0, st>>>(d_sd, nullptr, m->pt_ptr, m->pt_col, m->pt_val);
    // P = (P^T)^T: counts per ray, padded offsets, scatter, sort each row
    TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n_rays, st));
    TRY(cudaMemsetAsync(cursor, 0, sizeof(int) * (size_t)n_rays, st));
    k_count_cols<<<nb256(n_pix), 256, 0, st>>>(n_pix, m->pt_ptr, m->pt_col, m->pt_val, cnt);
    k_pad4<<<nb256(n_rays), 256, 0, st>>>(n_rays, cnt, cnt4);
    TRY(alloc(ctx, (void **)&m->p_ptr, sizeof(int) * ((size_t)n_rays + 1)));
    k_scan_exclusive<<<1, 1024, 0, st>>>(cnt4, m->p_ptr, n_rays, tot);
    TRY(cudaMemcpyAsync(&h_tot, tot, sizeof h_tot, cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    if (h_tot >= (1LL << 31) - 4) { e = cudaErrorInvalidValue; goto done; }
    m->nnz_p = h_tot;
    {
        // the longest row must fit the sort's shared memory
        int max_row = 0;
        std::vector<int> h(n_rays);
        TRY(cudaMemcpy(h.data(), cnt, sizeof(int) * (size_t)n_rays, cudaMemcpyDeviceToHost));
        for (int v : h) max_row = std::max(max_row, v);
        if (max_row > kMaxStoredRow) { e = cudaErrorInvalidValue; goto done; }
    }
    TRY(alloc(ctx, (void **)&m->p_col, sizeof(int) * (size_t)std::max(h_tot, 4LL)));
    TRY(alloc(ctx, (void **)&m->p_val, sizeof(float) * (size_t)std::max(h_tot, 4LL)));
    k_scatter_t<<<nb256(n_pix), 256, 0, st>>>(n_pix, m->pt_ptr, m->pt_col, m->pt_val, m->p_ptr, cursor,
                                              m->p_col, m->p_val);
    k_sort_rows<<<n_rays, 256, 0, st>>>(n_rays, m->p_ptr, cnt, m->p_col, m->p_val);
    TRY(cudaGetLastError());
    TRY(cudaStreamSynchronize(st));
done:
#undef TRY
    cudaFree(cnt);
    cudaFree(cnt4);
    cudaFree(cursor);
    cudaFree(tot);
    return e;
}

}  // namespace eptv
