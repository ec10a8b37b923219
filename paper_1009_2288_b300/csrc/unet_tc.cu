// 3x3 convolution of the learned warm-start network on the Blackwell tensor cores:
// tcgen05.mma (kind::f16, BF16 operands from shared memory, FP32 accumulator in tensor
// memory), implicit GEMM with
//   M = 128 output pixels of a tile, N = COUT output channels, K = 9 taps x CIN channels
// in 9 CIN/16 MMAs of 128 x COUT x 16 per tile.  The same kernel is the forward pass
// (weights [COUT][9][CIN]) and the data gradient (the mirrored, channel-swapped weights,
// CIN and COUT exchanged).
//
// A persistent block of 6 warps walks its tiles through two pipelines:
//   warp 4 loads each tile's input halo with TMA (cp.async.bulk.tensor, a 4-D tensor map
//     of the NHWC input; one box of 8 channels x the halo's columns x rows per 8-channel
//     chunk; the box reads zeros outside the image) into one of NS halo stages;
//   warp 5 issues the tile's MMAs into one of two accumulators in tensor memory and
//     commits them to the stage's "empty" and the accumulator's "full" mbarriers;
//   warps 0-3 read the accumulator back with tcgen05.ld (warp w: lanes 32w .. 32w + 31 =
//     its 32 pixels), add the bias, apply the ReLU, round to BF16, store into the output
//     channel slice, and release the accumulator.
// So the loads of the next tiles and the read-back of the previous one overlap the MMAs.
//
// Shared-memory operands use the canonical K-major layout without swizzle: "core
// matrices" of 8 rows x 16 bytes (8 channels), each 128 contiguous bytes.
//   B (weights, loaded once): byte (tap, ci, co) = ((tap CIN/8 + ci/8) COUT + co) 16 +
//     2 (ci % 8): N-direction stride 128 B, K-direction stride 16 COUT B.
//   A, tiles of one row segment (W a multiple of 128): per 8-channel chunk c8 one box of
//     3 halo rows x 130 columns at c8 A_C8 (A_C8 = the box rounded up to 128 bytes), byte
//     (r, px) = (r 130 + px) 16 within it: for tap (ky, kx) the 128 rows of A are the
//     columns px = m + kx of halo row ky -- a uniform 16-byte stride (M-direction stride
//     128 B, K-direction stride A_C8).
//   A, tiles of two rows (W = 64): three copies of the 4-row x 64-column halo, copy kx
//     shifted by kx - 1 columns: for tap (ky, kx) the 128 rows are the 128 consecutive
//     entries from row ky of copy kx.
//
// Every wait on an mbarrier is bounded: a role that waits longer than about a second sets
// the block's failure flag (the other roles stop at their next wait), the block sets the
// library's tensor-core error flag, frees its tensor memory and returns
// (eptv_unet_tc_status reports it).
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "eptv_internal.cuh"
#include "unet.cuh"

namespace eptv {

typedef __nv_bfloat16 bf16;

static __device__ unsigned int g_tc_error;     // 1: a bounded wait ran out

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of tcgen05.mma: start address, leading (K-direction)
// and stride (M/N-direction) byte offsets, all in 16-byte units; descriptor version 1,
// base offset 0, relative leading offsets, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 D, BF16 A and B, both K-major, N and M.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr long long kTcWaitCycles = 2000000000ll;   // ~1 s at 2 GHz
constexpr long long kTcWaitSpins = 1ll << 26;

__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}

// Bounded wait for the phase of the given parity to complete; false (and *fail set) if
// the bound ran out or another role of the block has failed.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity, volatile int *fail) {
    const long long t0 = clock64();
    for (long long s = 0; s < kTcWaitSpins; ++s) {
        if (mbar_try_wait(mbar, parity)) return true;
        if ((s & 63) == 63) {
            if (*fail) return false;
            if (clock64() - t0 > kTcWaitCycles) break;
        }
    }
    *fail = 1;
    return false;
}

// 4-D tiled TMA load of the NHWC input (channel, column, row, image) into shared memory,
// completing bytes on the mbarrier.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            int c3, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(dst), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(mbar))
        : "memory");
}

template <int CIN, int COUT, bool SHIFT>
struct TcShape {
    static constexpr int C8 = CIN / 8;
    static constexpr int HR = SHIFT ? 4 : 3;           // halo rows
    static constexpr int HW = SHIFT ? 64 : 130;        // pixels per halo row (per copy)
    static constexpr int NCOPY = SHIFT ? 3 : 1;
    static constexpr int TX_C8 = HR * HW * 16;         // bytes of one TMA box (8 channels)
    static constexpr int A_C8 = (TX_C8 + 127) / 128 * 128;   // box destinations 128-byte aligned
    static constexpr int A_COPY = C8 * A_C8;
    static constexpr int A_STAGE = NCOPY * A_COPY;
    static constexpr int TX = NCOPY * C8 * TX_C8;      // bytes landing per stage
    static constexpr int B_BYTES = 9 * C8 * COUT * 16;
    static constexpr int NS = (1024 + B_BYTES + 2 * A_STAGE <= 224 * 1024) ? 2 : 1;   // halo stages
    static constexpr int SMEM = 1024 + B_BYTES + NS * A_STAGE;
    static constexpr uint32_t NCOLS = 2 * COUT <= 32 ? 32 : (2 * COUT <= 64 ? 64 : (2 * COUT <= 128 ? 128 : 256));
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT >= 16 && COUT <= 128, "UMMA shape");
};

// 192 threads: warps 0-3 read the accumulators back (warp w: TMEM lanes 32w .. 32w + 31),
// warp 4 issues the TMA loads of the halo, warp 5 the MMAs.  Pipelines: halo stage s
// (full[s]: TMA bytes landed; empty[s]: the MMAs that read it are done) and accumulator b
// of two in tensor memory (tfull[b]: MMAs done; tempty[b]: the four epilogue warps read it).
template <int CIN, int COUT, bool SHIFT>
__global__ void __launch_bounds__(192, 1)
k_conv3x3_tc(const __grid_constant__ CUtensorMap xmap, int xo, int nimg, int H, int W,
             const bf16 *__restrict__ wt, const float *__restrict__ bias,
             bf16 *__restrict__ y, int ys, int yo, int relu, int vec16)
{
    using Sh = TcShape<CIN, COUT, SHIFT>;
    constexpr int C8 = Sh::C8, NS = Sh::NS;
    extern __shared__ unsigned char tc_smem_raw[];
    const uint32_t raw = smem_u32(tc_smem_raw);
    unsigned char *base = tc_smem_raw + (((raw + 1023u) & ~1023u) - raw);     // 1024-byte aligned
    unsigned char *sB = base;
    unsigned char *sA = base + Sh::B_BYTES;
    __shared__ __align__(8) uint64_t full[2], empty[2], tfull[2], tempty[2];
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_fail;
    __shared__ float s_bias[COUT];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // weights [COUT][9][CIN] -> B layout; bias
    for (int idx = tid; idx < COUT * 9 * C8; idx += 192) {
        const int co = idx / (9 * C8), rem = idx - co * 9 * C8, tap = rem / C8, c8 = rem - tap * C8;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(wt + ((size_t)co * 9 + tap) * CIN + c8 * 8));
        *reinterpret_cast<uint4 *>(sB + ((tap * C8 + c8) * COUT + co) * 16) = v;
    }
    for (int c = tid; c < COUT; c += 192) s_bias[c] = bias ? __ldg(bias + c) : 0.0f;
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(Sh::NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    const int tiles_per_img = SHIFT ? H / 2 : H * (W / 128);
    const int ntiles = nimg * tiles_per_img;
    if (warp == 4) {
        // ---- TMA producer: the halo of each tile, one box per 8-channel chunk (and copy)
        if (lane == 0) {
            int i = 0;
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
                const int s = i % NS;
                if (i >= NS && !mbar_wait(&empty[s], (uint32_t)((i / NS) - 1) & 1u, &s_fail)) break;
                const int n = tile / tiles_per_img, t = tile - n * tiles_per_img;
                const int r0 = SHIFT ? 2 * t : t / (W / 128);
                const int c0 = SHIFT ? 0 : (t - r0 * (W / 128)) * 128;
                mbar_expect_tx(&full[s], (uint32_t)Sh::TX);
                const uint32_t a = smem_u32(sA + s * Sh::A_STAGE);
                for (int kx = 0; kx < Sh::NCOPY; ++kx)
                    for (int c8 = 0; c8 < C8; ++c8)
                        tma_load_4d(a + kx * Sh::A_COPY + c8 * Sh::A_C8, &xmap, xo + 8 * c8,
                                    SHIFT ? kx - 1 : c0 - 1, r0 - 1, n, &full[s]);
            }
        }
    } else if (warp == 5) {
        // ---- MMA issuer: 9 taps x CIN / 16 MMAs of 128 x COUT x 16 per tile
        if (lane == 0) {
            constexpr uint32_t idesc = tc_idesc(128, COUT);
            const uint32_t b0 = smem_u32(sB);
            int i = 0;
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
                const int s = i % NS, b = i & 1;
                if (!mbar_wait(&full[s], (uint32_t)(i / NS) & 1u, &s_fail)) break;
                if (i >= 2 && !mbar_wait(&tempty[b], (uint32_t)((i / 2) - 1) & 1u, &s_fail)) break;
                tc_fence_after();
                const uint32_t a0 = smem_u32(sA + s * Sh::A_STAGE);
                const uint32_t d = tmem + (uint32_t)(b * COUT);
                uint32_t acc = 0;
#pragma unroll 1
                for (int tap = 0; tap < 9; ++tap) {
                    const int ky = tap / 3, kx = tap - 3 * (tap / 3);
#pragma unroll
                    for (int k16 = 0; k16 < CIN / 16; ++k16) {
                        const uint32_t aa = SHIFT ? a0 + kx * Sh::A_COPY + 2 * k16 * Sh::A_C8 + ky * Sh::HW * 16
                                                  : a0 + 2 * k16 * Sh::A_C8 + (ky * Sh::HW + kx) * 16;
                        const uint32_t bb = b0 + ((tap * C8 + 2 * k16) * COUT) * 16;
                        tc_mma(d, tc_desc(aa, Sh::A_C8, 128), tc_desc(bb, COUT * 16, 128), idesc, acc);
                        acc = 1;
                    }
                }
                tc_commit(&empty[s]);       // the halo stage is free once these MMAs are done
                tc_commit(&tfull[b]);       // and the accumulator is ready
            }
        }
    } else {
        // ---- epilogue: bias, ReLU, BF16 store of the tile's 128 pixels x COUT channels
        int i = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
            const int b = i & 1;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(&tfull[b], (uint32_t)(i / 2) & 1u, &s_fail);
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            tc_fence_after();
            const int n = tile / tiles_per_img, t = tile - n * tiles_per_img;
            const int r0 = SHIFT ? 2 * t : t / (W / 128);
            const int c0 = SHIFT ? 0 : (t - r0 * (W / 128)) * 128;
            const int p = warp * 32 + lane;
            const int gy = SHIFT ? r0 + p / 64 : r0, gx = SHIFT ? p % 64 : c0 + p;
            bf16 *yp = y + ((size_t)(n * H + gy) * W + gx) * ys + yo;
#pragma unroll
            for (int j = 0; j < COUT / 16; ++j) {
                float v[16];
                tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * COUT + j * 16), v);
                uint32_t pk[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float a = v[2 * q] + s_bias[j * 16 + 2 * q], c = v[2 * q + 1] + s_bias[j * 16 + 2 * q + 1];
                    if (relu) { a = fmaxf(a, 0.0f); c = fmaxf(c, 0.0f); }
                    const __nv_bfloat162 h = __floats2bfloat162_rn(a, c);
                    pk[q] = *reinterpret_cast<const uint32_t *>(&h);
                }
                if (vec16) {
                    *reinterpret_cast<uint4 *>(yp + j * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    *reinterpret_cast<uint4 *>(yp + j * 16 + 8) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) *reinterpret_cast<uint32_t *>(yp + j * 16 + 2 * q) = pk[q];
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
    }
    __syncthreads();
    if (s_fail && tid == 0) atomicOr(&g_tc_error, 1u);
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Sh::NCOLS) : "memory");
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static std::atomic<EncodeTiledFn> fn{nullptr};
    EncodeTiledFn f = fn.load();
    if (!f) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
            cudaGetLastError();
            return nullptr;
        }
        f = reinterpret_cast<EncodeTiledFn>(p);
        fn.store(f);
    }
    return f;
}

template <int CIN, int COUT, bool SHIFT>
static cudaError_t launch_tc(const bf16 *x, int n, int H, int W, int xs, int xo, const bf16 *wt,
                             const float *b, bf16 *y, int ys, int yo, int relu, cudaStream_t st) {
    using Sh = TcShape<CIN, COUT, SHIFT>;
    const void *fn = (const void *)&k_conv3x3_tc<CIN, COUT, SHIFT>;
    static int occ = 0;                  // per process; same value on every device
    if (!occ) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
        if (e != cudaSuccess) return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, 192, Sh::SMEM);
        if (e != cudaSuccess || o < 1) return e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
        occ = std::min(o, (int)(512 / Sh::NCOLS));          // tensor-memory columns per SM
    }
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    // the NHWC input as a 4-D tensor (channel, column, row, image); one box = 8 channels of
    // HW columns of HR rows; outside the image the box reads zeros
    CUtensorMap map;
    const cuuint64_t dims[4] = {(cuuint64_t)xs, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)n};
    const cuuint64_t strides[3] = {(cuuint64_t)xs * 2, (cuuint64_t)W * xs * 2, (cuuint64_t)H * W * xs * 2};
    const cuuint32_t box[4] = {8, (cuuint32_t)Sh::HW, (cuuint32_t)Sh::HR, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(x), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = n * (SHIFT ? H / 2 : H * (W / 128));
    const int grid = std::max(1, std::min(ntiles, occ * sms));
    const int vec16 = ((ys | yo) % 8 == 0) && ((((uintptr_t)y) & 15) == 0);
    ++g_launch_count;
    k_conv3x3_tc<CIN, COUT, SHIFT><<<grid, 192, Sh::SMEM, st>>>(map, xo, n, H, W, wt, b, y, ys, yo, relu, vec16);
    return cudaGetLastError();
}

// The tensor-core path for the layers whose rows it tiles: W a multiple of 128 (one row
// segment of 128 pixels per tile) or W = 64 with H even (two rows per tile), input channel
// stride and offset multiples of 8 (16-byte TMA boxes).  Returns cudaErrorNotSupported
// for the others (the caller then uses the mma.sync kernel).
cudaError_t unet_conv3x3_tc(const void *x, int n, int H, int W, int cin, int xs, int xo, const void *wt,
                            const float *b, int cout, void *y, int ys, int yo, int relu, cudaStream_t st,
                            bool all_shapes) {
    const bool row = W % 128 == 0, pair = W == 64 && H % 2 == 0;
    if ((!row && !pair) || (xs % 8) || (xo % 8) || (((uintptr_t)x) & 15)) return cudaErrorNotSupported;
    // measured on B300 (batch of 16): the 8-channel TMA boxes of the halo make the kernel
    // load-bound; it matches or beats the mma.sync kernel for rows of 128+ pixels with
    // CIN >= 32 or COUT >= 48, and loses on 16 -> 16 at 256^2 and on the single-stage
    // two-row tiles of 64-pixel rows, which therefore stay on mma.sync by default
    if (!all_shapes && !(row && (cin >= 32 || cout >= 48))) return cudaErrorNotSupported;
    const bf16 *X = static_cast<const bf16 *>(x);
    const bf16 *Wt = static_cast<const bf16 *>(wt);
    bf16 *Y = static_cast<bf16 *>(y);
#define TC_CASE(CI, CO)                                                                              \
    if (cin == CI && cout == CO)                                                                     \
        return row ? launch_tc<CI, CO, false>(X, n, H, W, xs, xo, Wt, b, Y, ys, yo, relu, st)        \
                   : launch_tc<CI, CO, true>(X, n, H, W, xs, xo, Wt, b, Y, ys, yo, relu, st);
    TC_CASE(16, 16) TC_CASE(16, 32) TC_CASE(32, 32) TC_CASE(32, 64) TC_CASE(64, 64)
    TC_CASE(96, 32) TC_CASE(48, 16) TC_CASE(32, 16) TC_CASE(64, 32) TC_CASE(32, 96)
    TC_CASE(16, 48) TC_CASE(64, 96)
#undef TC_CASE
    return cudaErrorNotSupported;
}

// Reads and clears the tensor-core error flag (1: a bounded wait ran out).
cudaError_t unet_tc_status(int *flag) {
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc_error, sizeof v);
    if (e != cudaSuccess) return e;
    if (v) {
        const unsigned int z = 0;
        e = cudaMemcpyToSymbol(g_tc_error, &z, sizeof z);
    }
    *flag = (int)v;
    return e;
}

}  // namespace eptv
