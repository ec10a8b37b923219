// Stored-matrix operator (Sec. 2.3): for small problems the paper keeps P as a sparse
// matrix and applies P and P^T as sparse matrix-vector products.  Here both are built
// once per geometry, on the device, as CSR matrices whose nonzeros are the canonical
// p_ij of eptv_internal.cuh (the values the on-the-fly back projector K2 forms), and are
// applied by SpMV kernels that stream the matrix from HBM while the vector they gather
// from stays in L2.
//
// Layout of each matrix: ptr [rows + 1] (int32), col [nnz] (int32), val [nnz] (FP32).
// Every row is padded to a multiple of 4 entries (val 0, col = the row's last column).
// The SpMV kernels read a SELL-32 copy of each (see below); the CSR form is what
// eptv_copy_matrix exports.
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

// Both kernels read a SELL-32 copy of their matrix (sliced ELLPACK): a slice holds 32
// rows, entry j of the row in lane l sits at sptr[s] + 32 j + l, and every row of slice s
// has slen[s] entries (zero-padded).  A lane owns a row, so each load of the stream is one
// 128-byte line per array, and the 32 rows gathered for at step j are neighbours -- the
// access pattern of the on-the-fly K1 / K2:
//   P:   slice s = rays 32 s .. 32 s + 31 (adjacent bins).  A shallow ray's columns are
//        stored as transposed pixel indices ix ny + iy (sorted in that order) and gathered
//        from the transposed image, like K1 does, so adjacent bins meet adjacent words.
//   P^T: slice (iy, sx) = pixels ix = 32 sx .. 32 sx + 31 of image row iy.
// A lane sums its row in entry order (deterministic).
// Layout within a slice: chunks of kSellChunk entries per lane, lane-interleaved, so that a
// lane's next kSellChunk entries are one 16-byte word (one 128-bit load of columns and one
// of values) and a warp's loads of one chunk are a contiguous 512 bytes.
constexpr int kSellChunk = 4;
__host__ __device__ __forceinline__ int sell_index(int j, int lane) {
    return (j / kSellChunk) * (32 * kSellChunk) + lane * kSellChunk + (j % kSellChunk);
}

__device__ __forceinline__ bool ray_is_steep(const RayRec &R, float dx, float dy) {
    return fabsf(R.ix) * dx >= fabsf(R.iy) * dy;      // the K1 criterion
}

// Row index of lane l of slice sl: linear slicing (width 0: rows 32 sl + l) or row-aligned
// slicing of an image with rows of `width` entries; -1 for a lane past the end.
__device__ __forceinline__ int sell_row(int sl, int l, int rows, int width) {
    if (width == 0) {
        const int r = sl * 32 + l;
        return r < rows ? r : -1;
    }
    const int spr = (width + 31) >> 5;
    const int iy = sl / spr, ix = (sl - iy * spr) * 32 + l;
    return (ix < width && iy * width < rows) ? iy * width + ix : -1;
}

// L2 policies for the matrix stream: a matrix larger than L2 passes through it on every
// product, evicting itself before reuse, so its entries are read evict_first -- except a
// leading part that fits in half of L2, read evict_last, which then stays in L2 from one
// product to the next (the products of an outer iteration and of the iterations after it)
// and is not read from DRAM again.  The other half is left to everything else.
__device__ __forceinline__ unsigned long long l2_evict_last_policy() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ int4 ld_keep(const int4 *a, unsigned long long p) {
    int4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(a), "l"(p));
    return v;
}
__device__ __forceinline__ float4 ld_keep(const float4 *a, unsigned long long p) {
    float4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(a), "l"(p));
    return v;
}

// REMAP: columns are transposed pixel indices c = ix ny + iy to be read from the
// natural image (no transposed copy given): index (c % ny) nx + c / ny.
// PIPE (long rows): software-pipelined, the next chunk's loads are in flight while the
// current chunk gathers from the vector, so the stream does not wait for the gathers.
// Short rows (P^T) run faster without the extra prologue loads.  base: the slice's start
// plus 32 times the first entry (a multiple of kSellChunk); len: a multiple of kSellChunk.
// The lane sums its entries in order (the same sum as an entry-by-entry loop).  keep: the
// slice's entries are read evict_last (the short-row form only).
template <bool REMAP, bool PIPE>
__device__ __forceinline__ float sell_row_dot(const int *__restrict__ scol, const float *__restrict__ sval,
                                              int base, int len, int lane, const float *__restrict__ x,
                                              int nx, int ny, bool keep = false) {
    const int4 *pc = reinterpret_cast<const int4 *>(scol + base) + lane;
    const float4 *pv = reinterpret_cast<const float4 *>(sval + base) + lane;
    const int n_chunks = len / kSellChunk;
    auto gather = [&](int k) {
        if (REMAP) { const int ix = k / ny; k = (k - ix * ny) * nx + ix; }
        return __ldg(x + k);
    };
    float acc = 0.0f;
    if (!PIPE) {
        const unsigned long long pol = l2_evict_last_policy();
        for (int c = 0; c < n_chunks; ++c) {
            const int4 cc = keep ? ld_keep(pc + 32 * c, pol) : __ldcs(pc + 32 * c);
            const float4 vv = keep ? ld_keep(pv + 32 * c, pol) : __ldcs(pv + 32 * c);
            const float x0 = gather(cc.x), x1 = gather(cc.y), x2 = gather(cc.z), x3 = gather(cc.w);
            acc = fmaf(vv.x, x0, acc);
            acc = fmaf(vv.y, x1, acc);
            acc = fmaf(vv.z, x2, acc);
            acc = fmaf(vv.w, x3, acc);
        }
        return acc;
    }
    // guarded loads as if / else: the conditional-expression form compiled to a loop
    // that ran the back projection at half the speed
    int4 cc = make_int4(0, 0, 0, 0);
    float4 vv = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (n_chunks > 0) {
        cc = __ldcs(pc);
        vv = __ldcs(pv);
    }
    for (int c = 0; c < n_chunks; ++c) {
        int4 cn = make_int4(0, 0, 0, 0);
        float4 vn = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (c + 1 < n_chunks) {
            cn = __ldcs(pc + 32 * (c + 1));
            vn = __ldcs(pv + 32 * (c + 1));
        }
        const float x0 = gather(cc.x), x1 = gather(cc.y), x2 = gather(cc.z), x3 = gather(cc.w);
        acc = fmaf(vv.x, x0, acc);
        acc = fmaf(vv.y, x1, acc);
        acc = fmaf(vv.z, x2, acc);
        acc = fmaf(vv.w, x3, acc);
        cc = cn;
        vv = vn;
    }
    return acc;
}

// y = P x (rows = rays).  Rays are long (hundreds of entries) and few (a slice per 32
// rays), so a block of 8 warps shares one slice: warp w streams the w-th eighth of the
// slice's entries and the 8 partial sums are added in warp order.  Same image selection
// (with its transposed copy), output selection, residual mode and fused |out|^2
// reduction as K1.
__global__ void __launch_bounds__(256)
k_spmv_p(const SliceDev *__restrict__ sls, TileMap map, ProjArgs a, double *__restrict__ partials)
{
    pdl_wait();
    __shared__ float part[8][32];
    __shared__ double rsm[2 * 8];
    __shared__ double res[2];
    __shared__ int last_flag;
    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double gamma_pre = threadIdx.x == 0 ? fin_gamma(S.sc, a.fin) : 0.0;
    const int slice = local;
    const int row = slice * 32 + lane;
    const float *x, *xT;
    if (a.img_override) { x = a.img_override; xT = a.imgT_override; }
    else if (a.img == IMG_U) { x = S.u; xT = a.no_T ? nullptr : S.uT; }
    else { x = S.s; xT = a.no_T ? nullptr : S.sT; }
    float *out = a.out_override ? a.out_override : (a.out == SINO_R ? S.r : S.q);
    float acc = 0.0f;
    if (row < S.n_rays) {
        const int len = __ldg(S.p_slen + slice);                       // multiple of kSellChunk
        const int chunk = ((len + 7) / 8 + kSellChunk - 1) / kSellChunk * kSellChunk;
        const int j0 = min(len, warp * chunk), j1 = min(len, j0 + chunk);
        const int base = __ldg(S.p_sptr + slice) + 32 * j0;
        const bool steep = ray_is_steep(S.ray[row], S.dx, S.dy);
        if (steep || xT)     // one loop for the whole warp, lanes differ only in the source
            acc = sell_row_dot<false, true>(S.p_scol, S.p_sval, base, j1 - j0, lane, steep ? x : xT, S.nx, S.ny);
        else
            acc = sell_row_dot<true, true>(S.p_scol, S.p_sval, base, j1 - j0, lane, x, S.nx, S.ny);
    }
    part[warp][lane] = acc;
    __syncthreads();
    float sq = 0.0f, ysum = 0.0f;
    if (warp == 0 && row < S.n_rays) {
        float tot = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) tot += part[w][lane];
        float o = tot;
        if (a.resid) o = __ldg((a.y_override ? a.y_override : S.y) + row) - tot;
        out[row] = o;
        sq = o * o;
        ysum = o;
    }
    if (a.fin == FIN_NONE) return;
    const int b0 = __ldg(map.start + si);
    const int nblk = __ldg(map.start + si + 1) - b0;
    float vals[2] = {sq, ysum};
    block_sum_to<2, 256>(vals, partials + (size_t)blockIdx.x * 2, rsm);
    if (!reduce_slice<2, 256>(S, partials, 2, b0, nblk, local, rsm, res, &last_flag)) return;
    if (threadIdx.x == 0) finalize(S.sc, a.fin, res[0], res[1], gamma_pre);
}

// x = P^T y (rows = pixels).  A block covers a 32 x 8 pixel tile (warp = one image row of
// 32 pixels = one slice).  Same output selection, transposed copy (through a shared-memory
// tile, 8 consecutive rows per column) and fused |out|^2 reduction as K2.
__global__ void __launch_bounds__(256)
k_spmv_pt(const SliceDev *__restrict__ sls, TileMap map, BackArgs a, double *__restrict__ partials)
{
    pdl_wait();
    __shared__ float tile[8][33];
    __shared__ double rsm[2 * 8];
    __shared__ double res[2];
    __shared__ int last_flag;
    int local;
    const int si = find_slice(map, blockIdx.x, &local);
    const SliceDev &S = sls[si];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double gamma_pre = threadIdx.x == 0 ? fin_gamma(S.sc, a.fin) : 0.0;
    const int spr = (S.nx + 31) >> 5;
    const int ty = local / spr, sx = local - ty * spr;
    const int iy = ty * 8 + warp, ix = sx * 32 + lane;
    const int slice = iy * spr + sx;
    const float *in = a.in_override ? a.in_override : S.r;
    float *out, *outT = nullptr;
    if (a.out_override) out = a.out_override;
    else if (a.out == 0) { out = S.s; if (a.write_T) outT = S.sT; }
    else if (a.out == 1) out = S.t;
    else { out = S.u; if (a.write_T) outT = S.uT; }
    float acc = 0.0f;
    const bool valid = iy < S.ny && ix < S.nx;
    if (valid) {
        acc = sell_row_dot<false, false>(S.pt_scol, S.pt_sval, __ldg(S.pt_sptr + slice),
                                         __ldg(S.pt_slen + slice), lane, in, S.nx, S.ny,
                                         slice < S.pt_keep);
        out[(size_t)iy * S.nx + ix] = acc;
    }
    if (outT) {
        tile[warp][lane] = acc;
        __syncthreads();
        const int cx = threadIdx.x >> 3, ry = threadIdx.x & 7;
        const int gx = sx * 32 + cx, gy = ty * 8 + ry;
        if (gx < S.nx && gy < S.ny) outT[(size_t)gx * S.ny + gy] = tile[ry][cx];
    }
    if (a.fin == FIN_NONE) return;
    const int b0 = __ldg(map.start + si);
    const int nblk = __ldg(map.start + si + 1) - b0;
    float vals[1] = {valid ? acc * acc : 0.0f};
    block_sum_to<1, 256>(vals, partials + (size_t)blockIdx.x * 2, rsm);
    if (threadIdx.x == 0) partials[(size_t)blockIdx.x * 2 + 1] = 0.0;
    if (!reduce_slice<2, 256>(S, partials, 2, b0, nblk, local, rsm, res, &last_flag)) return;
    if (threadIdx.x == 0) finalize(S.sc, a.fin, res[0], res[1], gamma_pre);
}

void launch_spmv_p(const Batch &B, const ProjArgs &a, cudaStream_t st) {
    const int nblk = B.blocks(FAM_SPMV_P);
    if (nblk == 0) return;
    ++g_launch_count;
    launch_pdl(k_spmv_p, nblk, 256, 0, st, B.d_sd, B.map(FAM_SPMV_P), a, B.d_partials);
}

void launch_spmv_pt(const Batch &B, const BackArgs &a, cudaStream_t st) {
    const int nblk = B.blocks(FAM_SPMV_PT);
    if (nblk == 0) return;
    ++g_launch_count;
    launch_pdl(k_spmv_pt, nblk, 256, 0, st, B.d_sd, B.map(FAM_SPMV_PT), a, B.d_partials);
}

// ---------------------------------------------------------------- CSR -> SELL-32

// Real entries of each row of a padded CSR matrix (padding: < 4 trailing zeros).
__global__ void __launch_bounds__(256)
k_row_real(int rows, const int *__restrict__ ptr, const float *__restrict__ val, int *__restrict__ cnt)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int b = ptr[r];
    int e = ptr[r + 1];
    while (e > b && val[e - 1] == 0.0f) --e;
    cnt[r] = e - b;
}

// slen[s] = longest row of slice s rounded up to a multiple of kSellChunk; w[s] = 32 slen[s]
// (the slice's stored entries).
__global__ void __launch_bounds__(256)
k_slice_len(int n_sl, int rows, int width, const int *__restrict__ cnt, int *__restrict__ slen,
            int *__restrict__ w)
{
    const int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= n_sl) return;
    int m = 0;
    for (int l = 0; l < 32; ++l) {
        const int r = sell_row(sl, l, rows, width);
        if (r >= 0) m = max(m, cnt[r]);
    }
    m = (m + kSellChunk - 1) / kSellChunk * kSellChunk;
    slen[sl] = m;
    w[sl] = 32 * m;
}

// Row sell_row(s, l) of the CSR matrix into lane l of slice s; the padding repeats the
// row's last column with value 0 (lanes past the end: column 0).
__global__ void __launch_bounds__(256)
k_fill_sell(int n_sl, int rows, int width, const int *__restrict__ ptr, const int *__restrict__ cnt,
            const int *__restrict__ col, const float *__restrict__ val, const int *__restrict__ sptr,
            const int *__restrict__ slen, int *__restrict__ scol, float *__restrict__ sval)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int sl = (int)(t >> 5), l = (int)(t & 31);
    if (sl >= n_sl) return;
    const int r = sell_row(sl, l, rows, width);
    const int base = sptr[sl], len = slen[sl];
    const int n = (r >= 0) ? cnt[r] : 0;
    const int b = (r >= 0) ? ptr[r] : 0;
    const int last = n > 0 ? col[b + n - 1] : 0;
    for (int j = 0; j < len; ++j) {
        const int idx = base + sell_index(j, l);
        scol[idx] = (j < n) ? col[b + j] : last;
        sval[idx] = (j < n) ? val[b + j] : 0.0f;
    }
}

// Shallow rays of P (the K1 criterion): columns to transposed pixel indices ix ny + iy.
__global__ void __launch_bounds__(256)
k_transpose_shallow(const SliceDev *__restrict__ sd, const int *__restrict__ ptr, const int *__restrict__ cnt,
                    int *__restrict__ col)
{
    const SliceDev &S = *sd;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= S.n_rays) return;
    if (ray_is_steep(S.ray[r], S.dx, S.dy)) return;
    const int b = ptr[r];
    for (int e = b; e < b + cnt[r]; ++e) {
        const int c = col[e];
        const int iy = c / S.nx, ix = c - iy * S.nx;
        col[e] = ix * S.ny + iy;
    }
}

// ---------------------------------------------------------------- build driver

static unsigned nb256(long long n) { return (unsigned)((n + 255) / 256); }

// SELL-32 copy of a padded, row-sorted CSR matrix (width: 0 for linear slicing, else the
// image row length for row-aligned slicing; tmp_cnt: rows ints, tmp_w: slices + 1 ints,
// tot: one long long; all device scratch).
static cudaError_t to_sell(int rows, int width, const int *ptr, const int *col, const float *val,
                           StoredAlloc alloc, void *ctx, int **sptr, int **slen, int **scol, float **sval,
                           long long *total, int *tmp_cnt, int *tmp_w, long long *tot, cudaStream_t st) {
    const int n_sl = width ? (rows / width) * ((width + 31) / 32) : (rows + 31) / 32;
    cudaError_t e;
    if ((e = alloc(ctx, (void **)slen, sizeof(int) * (size_t)std::max(n_sl, 1))) != cudaSuccess) return e;
    if ((e = alloc(ctx, (void **)sptr, sizeof(int) * ((size_t)n_sl + 1))) != cudaSuccess) return e;
    k_row_real<<<nb256(rows), 256, 0, st>>>(rows, ptr, val, tmp_cnt);
    k_slice_len<<<nb256(n_sl), 256, 0, st>>>(n_sl, rows, width, tmp_cnt, *slen, tmp_w);
    k_scan_exclusive<<<1, 1024, 0, st>>>(tmp_w, *sptr, n_sl, tot);
    long long h_tot = 0;
    if ((e = cudaMemcpyAsync(&h_tot, tot, sizeof h_tot, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (h_tot >= (1LL << 31) - 32) return cudaErrorInvalidValue;
    *total = h_tot;
    if ((e = alloc(ctx, (void **)scol, sizeof(int) * (size_t)std::max(h_tot, 32LL))) != cudaSuccess) return e;
    if ((e = alloc(ctx, (void **)sval, sizeof(float) * (size_t)std::max(h_tot, 32LL))) != cudaSuccess) return e;
    k_fill_sell<<<nb256((long long)n_sl * 32), 256, 0, st>>>(n_sl, rows, width, ptr, tmp_cnt, col, val, *sptr,
                                                            *slen, *scol, *sval);
    return cudaGetLastError();
}

// Builds both matrices of the slice described by d_sd (device copy of `S`, whose ray and
// view tables are set).  Allocation goes through `alloc` (owned by the caller).  Returns
// cudaSuccess, or cudaErrorInvalidValue if a row of P is longer than kMaxStoredRow or the
// matrix has 2^31 or more stored entries.
cudaError_t build_stored(const SliceDev &S, const SliceDev *d_sd, StoredAlloc alloc, void *ctx,
                         StoredMatrices *m, cudaStream_t st) {
    const int n_pix = S.n_pix, n_rays = S.n_rays;
    int *cnt = nullptr, *cnt4 = nullptr, *cursor = nullptr, *w = nullptr, *tcol = nullptr;
    float *tval = nullptr;
    long long *tot = nullptr;
    cudaError_t e;
    long long h_tot = 0;
#define TRY(x) do { e = (x); if (e != cudaSuccess) goto done; } while (0)
    TRY(cudaMalloc(&cnt, sizeof(int) * (size_t)(std::max(n_pix, n_rays) + 1)));
    TRY(cudaMalloc(&cnt4, sizeof(int) * (size_t)(n_rays + 1)));
    TRY(cudaMalloc(&cursor, sizeof(int) * (size_t)n_rays));
    TRY(cudaMalloc(&tot, sizeof(long long)));
    // slice widths: (n_rays + 31) / 32 slices of P, ny * ceil(nx / 32) of P^T
    TRY(cudaMalloc(&w, sizeof(int) * (size_t)(std::max((n_rays + 31) / 32, S.ny * ((S.nx + 31) / 32)) + 2)));
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
    // SELL-32 copies for the SpMV kernels.  P: a copy whose shallow rows hold transposed
    // pixel indices, re-sorted; P^T: row-aligned slices of the image.
    TRY(cudaMalloc(&tcol, sizeof(int) * (size_t)std::max(m->nnz_p, 4LL)));
    TRY(cudaMalloc(&tval, sizeof(float) * (size_t)std::max(m->nnz_p, 4LL)));
    TRY(cudaMemcpyAsync(tcol, m->p_col, sizeof(int) * (size_t)m->nnz_p, cudaMemcpyDeviceToDevice, st));
    TRY(cudaMemcpyAsync(tval, m->p_val, sizeof(float) * (size_t)m->nnz_p, cudaMemcpyDeviceToDevice, st));
    k_transpose_shallow<<<nb256(n_rays), 256, 0, st>>>(d_sd, m->p_ptr, cnt, tcol);
    k_sort_rows<<<n_rays, 256, 0, st>>>(n_rays, m->p_ptr, cnt, tcol, tval);
    TRY(to_sell(n_rays, 0, m->p_ptr, tcol, tval, alloc, ctx, &m->p_sptr, &m->p_slen, &m->p_scol,
                &m->p_sval, &m->sell_p, cnt, w, tot, st));
    TRY(to_sell(n_pix, S.nx, m->pt_ptr, m->pt_col, m->pt_val, alloc, ctx, &m->pt_sptr, &m->pt_slen,
                &m->pt_scol, &m->pt_sval, &m->sell_pt, cnt, w, tot, st));
    TRY(cudaStreamSynchronize(st));
done:
#undef TRY
    cudaFree(cnt);
    cudaFree(cnt4);
    cudaFree(cursor);
    cudaFree(tot);
    cudaFree(w);
    cudaFree(tcol);
    cudaFree(tval);
    return e;
}

}  // namespace eptv
