// Layer kernels of the learned warm-start network (a small U-Net; the paper has none):
// BF16 activations in NHWC layout ([n][H][W][channel stride], a layer may read or write a
// channel slice so that concatenation is free), FP32 master weights.
//
//   conv3x3 forward (and data gradient, with flipped / transposed weights): implicit GEMM
//     on the tensor cores with mma.sync m16n8k16 (BF16 in, FP32 accumulate).  A block
//     keeps all weights [COUT][9][CIN] in shared memory and walks 8 x 16 output tiles;
//     each tile's 10 x 18 input halo is staged in shared memory; a warp computes two
//     rows of 16 pixels (M = 16 per mma) for all output channels (N = COUT), K = 9 taps x
//     CIN.  Padded shared strides make every fragment load bank-conflict free.
//     Fused bias + ReLU + BF16 store into a channel slice of the output.
//   conv3x3 weight gradient: implicit GEMM on the tensor cores as well (M = output
//     channels, N = input channels, K = pixels), one warp per tap, register accumulators
//     over a block's pixel tiles, one FP32 atomic add per weight per block.
//   pooling / upsampling / ReLU backward / 1x1 head + loss / Adam: elementwise kernels.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "eptv_internal.cuh"
#include "unet.cuh"

namespace eptv {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                               uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

constexpr int kCvTH = 8, kCvTW = 16;                  // output tile
constexpr int kCvHP = kCvTH + 2, kCvWP = kCvTW + 2;   // halo tile

template <int CIN, int COUT>
constexpr int conv_smem_bytes() {
    return (kCvHP * kCvWP * (CIN + 8) + COUT * (9 * CIN + 8)) * 2;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(128)
k_conv3x3_mma(const bf16 *__restrict__ x, int nimg, int H, int W, int xs, int xo,
              const bf16 *__restrict__ wt, const float *__restrict__ bias,
              bf16 *__restrict__ y, int ys, int yo, int relu)
{
    constexpr int XS = CIN + 8;          // bf16 per staged pixel
    constexpr int WS = 9 * CIN + 8;      // bf16 per staged output channel
    constexpr int NT = COUT / 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16 *sx = reinterpret_cast<bf16 *>(smem_raw);
    bf16 *sw = sx + kCvHP * kCvWP * XS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;

    // all weights once per block
    constexpr int WV = 9 * CIN / 8;      // 16-byte vectors per output channel
    for (int idx = tid; idx < COUT * WV; idx += 128) {
        const int co = idx / WV, v = idx - co * WV;
        *reinterpret_cast<uint4 *>(sw + co * WS + v * 8) =
            __ldg(reinterpret_cast<const uint4 *>(wt + (size_t)co * 9 * CIN + v * 8));
    }
    const int tiles_x = (W + kCvTW - 1) / kCvTW, tiles_y = (H + kCvTH - 1) / kCvTH;
    const int ntiles = nimg * tiles_x * tiles_y;
    float bv[NT][2];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        bv[nt][0] = bias ? __ldg(bias + nt * 8 + 2 * t) : 0.0f;
        bv[nt][1] = bias ? __ldg(bias + nt * 8 + 2 * t + 1) : 0.0f;
    }

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int n = tile / (tiles_x * tiles_y);
        const int rem = tile - n * tiles_x * tiles_y;
        const int r0 = (rem / tiles_x) * kCvTH, c0 = (rem % tiles_x) * kCvTW;
        __syncthreads();                 // previous tile's reads of sx are done
        constexpr int XV = CIN / 8;
        for (int idx = tid; idx < kCvHP * kCvWP * XV; idx += 128) {
            const int p = idx / XV, v = idx - p * XV;
            const int ty = p / kCvWP, tx = p - ty * kCvWP;
            const int gy = r0 - 1 + ty, gx = c0 - 1 + tx;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (gy >= 0 && gy < H && gx >= 0 && gx < W)
                val = __ldg(reinterpret_cast<const uint4 *>(x + ((size_t)(n * H + gy) * W + gx) * xs + xo + v * 8));
            *reinterpret_cast<uint4 *>(sx + p * XS + v * 8) = val;
        }
        __syncthreads();

        float acc[2][NT][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.0f;

#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int ky = tap / 3, kx = tap - 3 * (tap / 3);
#pragma unroll
            for (int k0 = 0; k0 < CIN; k0 += 16) {
                uint32_t b[NT][2];
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const bf16 *wp = sw + (nt * 8 + g) * WS + tap * CIN + k0 + 2 * t;
                    b[nt][0] = *reinterpret_cast<const uint32_t *>(wp);
                    b[nt][1] = *reinterpret_cast<const uint32_t *>(wp + 8);
                }
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const int row = warp * 2 + mt + ky;
                    const bf16 *p0 = sx + (row * kCvWP + g + kx) * XS + k0 + 2 * t;
                    const bf16 *p1 = p0 + 8 * XS;
                    const uint32_t a0 = *reinterpret_cast<const uint32_t *>(p0);
                    const uint32_t a1 = *reinterpret_cast<const uint32_t *>(p1);
                    const uint32_t a2 = *reinterpret_cast<const uint32_t *>(p0 + 8);
                    const uint32_t a3 = *reinterpret_cast<const uint32_t *>(p1 + 8);
#pragma unroll
                    for (int nt = 0; nt < NT; ++nt) mma_bf16_16816(acc[mt][nt], a0, a1, a2, a3, b[nt][0], b[nt][1]);
                }
            }
        }
        // epilogue: bias, ReLU, BF16, store into the output channel slice
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int gy = r0 + warp * 2 + mt;
            if (gy >= H) continue;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int gx = c0 + g + 8 * half;
                if (gx >= W) continue;
                bf16 *yp = y + ((size_t)(n * H + gy) * W + gx) * ys + yo;
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    float v0 = acc[mt][nt][2 * half] + bv[nt][0];
                    float v1 = acc[mt][nt][2 * half + 1] + bv[nt][1];
                    if (relu) { v0 = fmaxf(v0, 0.0f); v1 = fmaxf(v1, 0.0f); }
                    *reinterpret_cast<__nv_bfloat162 *>(yp + nt * 8 + 2 * t) = __floats2bfloat162_rn(v0, v1);
                }
            }
        }
    }
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3,
                                              const bf16 *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

template <int CIN, int COUT>
constexpr int wgrad_smem_bytes() {
    return (kCvHP * kCvWP * (CIN + 8) + kCvTH * kCvTW * (COUT + 8)) * 2;
}

// dW[co][tap][ci] += sum_p dy[p][co] x[p + off(tap)][ci], db[co] += sum_p dy[p][co].
// Implicit GEMM on the tensor cores: M = output channels, N = input channels, K = pixels.
// The block walks 8 x 16 pixel tiles (stride gridDim.x); per tile the 10 x 18 input halo
// and the 8 x 16 output-gradient tile are staged in shared memory in their NHWC layout, and
// ldmatrix.trans turns 8-pixel x 8-channel blocks into the K-major fragments of the mma.
// Warp w owns tap w (9 warps): per tile row (K = 16 pixels) it multiplies the dy fragment
// of every 16-channel group by the halo row shifted by that tap.  Warp 4 (the centre tap)
// also multiplies dy by a ones fragment for the bias gradient.  FP32 accumulators stay in
// registers over all of the block's tiles and are added to dW once per block.  A block
// covers MG of the COUT / 16 output-channel groups (blockIdx.y picks which), so that a warp
// holds at most 64 accumulators.
template <int CIN, int COUT>
__host__ __device__ constexpr int wgrad_mgroups() {
    int mg = COUT / 16;
    while (mg > 1 && (mg * (CIN / 8) > 16 || (COUT / 16) % mg)) --mg;
    return mg;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(288, 1)
k_conv3x3_wgrad_mma(const bf16 *__restrict__ x, int nimg, int H, int W, int xs, int xo,
                    const bf16 *__restrict__ dy, int dys, int dyo,
                    float *__restrict__ dw, float *__restrict__ db)
{
    constexpr int XS = CIN + 8, DS = COUT + 8;
    constexpr int MT = wgrad_mgroups<CIN, COUT>(), NT = CIN / 8;
    const int m0 = blockIdx.y * MT;                          // first 16-channel group
    extern __shared__ __align__(16) unsigned char smem_raw[];
    bf16 *sx = reinterpret_cast<bf16 *>(smem_raw);          // [10 * 18][XS]
    bf16 *sd = sx + kCvHP * kCvWP * XS;                      // [8 * 16][DS]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const int tap = warp, ky = tap / 3, kx = tap - 3 * (tap / 3);
    const bool bias_warp = (db != nullptr) && tap == 4;

    float acc[MT][NT][4];
    float accb[MT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
        for (int q = 0; q < 4; ++q) accb[mt][q] = 0.0f;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.0f;
    }
    // per-lane ldmatrix row offsets: matrix q = lane / 8, row r = lane % 8
    const int q = lane >> 3, r = lane & 7;
    const int a_pix = r + (q >> 1) * 8, a_ch = (q & 1) * 8;   // dy: (pixel, channel) blocks
    const int b_pix = r + (q & 1) * 8, b_ch = (q >> 1) * 8;   // x:  (pixel, channel) blocks
    const uint32_t ones = 0x3F803F80u;                         // two BF16 1.0

    const int tiles_x = (W + kCvTW - 1) / kCvTW, tiles_y = (H + kCvTH - 1) / kCvTH;
    const int ntiles = nimg * tiles_x * tiles_y;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int n = tile / (tiles_x * tiles_y);
        const int rem = tile - n * tiles_x * tiles_y;
        const int r0 = (rem / tiles_x) * kCvTH, c0 = (rem % tiles_x) * kCvTW;
        __syncthreads();                 // previous tile's fragment loads are done
        constexpr int XV = CIN / 8;
        for (int idx = tid; idx < kCvHP * kCvWP * XV; idx += 288) {
            const int pp = idx / XV, v = idx - pp * XV;
            const int ty = pp / kCvWP, tx = pp - ty * kCvWP;
            const int gy = r0 - 1 + ty, gx = c0 - 1 + tx;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (gy >= 0 && gy < H && gx >= 0 && gx < W)
                val = __ldg(reinterpret_cast<const uint4 *>(x + ((size_t)(n * H + gy) * W + gx) * xs + xo + v * 8));
            *reinterpret_cast<uint4 *>(sx + pp * XS + v * 8) = val;
        }
        constexpr int DV = COUT / 8;
        for (int idx = tid; idx < kCvTH * kCvTW * DV; idx += 288) {
            const int pp = idx / DV, v = idx - pp * DV;
            const int ty = pp / kCvTW, tx = pp - ty * kCvTW;
            const int gy = r0 + ty, gx = c0 + tx;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (gy < H && gx < W)
                val = __ldg(reinterpret_cast<const uint4 *>(dy + ((size_t)(n * H + gy) * W + gx) * dys + dyo + v * 8));
            *reinterpret_cast<uint4 *>(sd + pp * DS + v * 8) = val;
        }
        __syncthreads();
#pragma unroll 1
        for (int row = 0; row < kCvTH; ++row) {
            uint32_t a[MT][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
                ldsm_x4_trans(a[mt][0], a[mt][1], a[mt][2], a[mt][3],
                              sd + (row * kCvTW + a_pix) * DS + (m0 + mt) * 16 + a_ch);
            const bf16 *xrow = sx + ((row + ky) * kCvWP + kx + b_pix) * XS + b_ch;
#pragma unroll
            for (int np = 0; np < NT / 2; ++np) {
                uint32_t b0, b1, b2, b3;
                ldsm_x4_trans(b0, b1, b2, b3, xrow + np * 16);
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    mma_bf16_16816(acc[mt][2 * np], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
                    mma_bf16_16816(acc[mt][2 * np + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b2, b3);
                }
            }
            if (bias_warp) {
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
                    mma_bf16_16816(accb[mt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], ones, ones);
            }
        }
    }
    // D fragment: c0, c1 at (row g, columns 2t, 2t+1), c2, c3 at row g + 8
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const int ci = nt * 8 + 2 * t;
            float *p0 = dw + ((size_t)((m0 + mt) * 16 + g) * 9 + tap) * CIN + ci;
            float *p1 = dw + ((size_t)((m0 + mt) * 16 + g + 8) * 9 + tap) * CIN + ci;
            atomicAdd(p0, acc[mt][nt][0]);
            atomicAdd(p0 + 1, acc[mt][nt][1]);
            atomicAdd(p1, acc[mt][nt][2]);
            atomicAdd(p1 + 1, acc[mt][nt][3]);
        }
        if (bias_warp && t == 0) {
            atomicAdd(db + (m0 + mt) * 16 + g, accb[mt][0]);
            atomicAdd(db + (m0 + mt) * 16 + g + 8, accb[mt][2]);
        }
    }
}

// Master FP32 weights [cout][9][cin] -> BF16 forward layout and BF16 data-gradient layout
// wb[ci][tap'][co] = w[co][8 - tap'][ci] (taps flipped, channels swapped).
__global__ void k_weights_to_bf16(const float *__restrict__ w, int cout, int cin,
                                  bf16 *__restrict__ wf, bf16 *__restrict__ wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cout * 9 * cin) return;
    const int co = i / (9 * cin), rem = i - co * 9 * cin, tap = rem / cin, ci = rem - tap * cin;
    const bf16 v = __float2bfloat16_rn(w[i]);
    if (wf) wf[i] = v;
    if (wb) wb[((size_t)ci * 9 + (8 - tap)) * cout + co] = v;
}

__global__ void k_maxpool2(const bf16 *__restrict__ x, int nimg, int H, int W, int xs, int xo, int C,
                           bf16 *__restrict__ y, int ys, int yo) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int Ho = H / 2, Wo = W / 2;
    if (i >= (long long)nimg * Ho * Wo * C) return;
    const int c = (int)(i % C);
    const long long p = i / C;
    const int n = (int)(p / (Ho * Wo)), rr = (int)(p % (Ho * Wo)), r = rr / Wo, q = rr % Wo;
    const bf16 *b = x + ((size_t)(n * H + 2 * r) * W + 2 * q) * xs + xo + c;
    float m = __bfloat162float(b[0]);
    m = fmaxf(m, __bfloat162float(b[xs]));
    m = fmaxf(m, __bfloat162float(b[(size_t)W * xs]));
    m = fmaxf(m, __bfloat162float(b[(size_t)W * xs + xs]));
    y[((size_t)(n * Ho + r) * Wo + q) * ys + yo + c] = __float2bfloat16_rn(m);
}

// dx (+)= gradient routed to the first maximum of each 2x2 window (row-major order)
__global__ void k_maxpool2_bwd(const bf16 *__restrict__ x, int nimg, int H, int W, int xs, int xo,
                               int C, const bf16 *__restrict__ dy, int dys, int dyo,
                               bf16 *__restrict__ dx, int dxs, int dxo, int accumulate) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int Ho = H / 2, Wo = W / 2;
    if (i >= (long long)nimg * Ho * Wo * C) return;
    const int c = (int)(i % C);
    const long long p = i / C;
    const int n = (int)(p / (Ho * Wo)), rr = (int)(p % (Ho * Wo)), r = rr / Wo, q = rr % Wo;
    float v[4];
    size_t off[4];
    for (int k = 0; k < 4; ++k) {
        const int yy = 2 * r + k / 2, xx = 2 * q + k % 2;
        v[k] = __bfloat162float(x[((size_t)(n * H + yy) * W + xx) * xs + xo + c]);
        off[k] = ((size_t)(n * H + yy) * W + xx) * dxs + dxo + c;
    }
    int best = 0;
    for (int k = 1; k < 4; ++k) if (v[k] > v[best]) best = k;
    const float g = __bfloat162float(dy[((size_t)(n * Ho + r) * Wo + q) * dys + dyo + c]);
    for (int k = 0; k < 4; ++k) {
        const float add = (k == best) ? g : 0.0f;
        const float base = accumulate ? __bfloat162float(dx[off[k]]) : 0.0f;
        dx[off[k]] = __float2bfloat16_rn(base + add);
    }
}

__global__ void k_upsample2(const bf16 *__restrict__ x, int nimg, int H, int W, int xs, int xo, int C,
                            bf16 *__restrict__ y, int ys, int yo) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int Ho = 2 * H, Wo = 2 * W;
    if (i >= (long long)nimg * Ho * Wo * C) return;
    const int c = (int)(i % C);
    const long long p = i / C;
    const int n = (int)(p / (Ho * Wo)), rr = (int)(p % (Ho * Wo)), r = rr / Wo, q = rr % Wo;
    y[((size_t)(n * Ho + r) * Wo + q) * ys + yo + c] = x[((size_t)(n * H + r / 2) * W + q / 2) * xs + xo + c];
}

__global__ void k_upsample2_bwd(const bf16 *__restrict__ dy, int nimg, int H, int W, int dys, int dyo,
                                int C, bf16 *__restrict__ dx, int dxs, int dxo) {
    // H, W: the upsampled (input of this backward) size
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int Ho = H / 2, Wo = W / 2;
    if (i >= (long long)nimg * Ho * Wo * C) return;
    const int c = (int)(i % C);
    const long long p = i / C;
    const int n = (int)(p / (Ho * Wo)), rr = (int)(p % (Ho * Wo)), r = rr / Wo, q = rr % Wo;
    float s = 0.0f;
    for (int k = 0; k < 4; ++k)
        s += __bfloat162float(dy[((size_t)(n * H + 2 * r + k / 2) * W + 2 * q + k % 2) * dys + dyo + c]);
    dx[((size_t)(n * Ho + r) * Wo + q) * dxs + dxo + c] = __float2bfloat16_rn(s);
}

// dz = dy where the ReLU output a > 0, else 0 (in place allowed)
__global__ void k_relu_bwd(const bf16 *__restrict__ a, int as, int ao, const bf16 *dy, int dys, int dyo,
                           bf16 *dz, int dzs, int dzo, long long npix, int C) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npix * C) return;
    const long long p = i / C;
    const int c = (int)(i % C);
    const float av = __bfloat162float(a[p * as + ao + c]);
    const bf16 g = dy[p * dys + dyo + c];
    dz[p * dzs + dzo + c] = (av > 0.0f) ? g : __float2bfloat16_rn(0.0f);
}

// 1x1 head (16 -> 2): f0 = o0, w = sigmoid(o1).  With targets: loss += mean((f0-ft)^2 +
// (w-wt)^2) terms, dx = hW^T do, dhW += do x^T, dhb += do (do = dL/do, L averaged over the
// pixels of all images).
// Network input: x[p][0] = a[p] sa, x[p][1] = b[p] sb (0 without b), channels 2..15 = 0,
// BF16 rows of 16 channels (two 16-byte stores per pixel).
__global__ void __launch_bounds__(256)
k_pack_input(const float *__restrict__ a, float sa, const float *__restrict__ b, float sb,
             long long npix, bf16 *__restrict__ x) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const __nv_bfloat162 v01 = __floats2bfloat162_rn(a[p] * sa, b ? b[p] * sb : 0.0f);
    uint4 lo = make_uint4(0u, 0u, 0u, 0u);
    lo.x = *reinterpret_cast<const uint32_t *>(&v01);
    uint4 *dst = reinterpret_cast<uint4 *>(x + p * 16);
    dst[0] = lo;
    dst[1] = make_uint4(0u, 0u, 0u, 0u);
}

__global__ void __launch_bounds__(256)
k_head(const bf16 *__restrict__ x, int xs, int xo, long long npix, const float *__restrict__ hw,
       const float *__restrict__ hb, float *__restrict__ f0, float *__restrict__ w,
       const float *__restrict__ base, float f_scale,
       const float *__restrict__ ft, const float *__restrict__ wt, bf16 *__restrict__ dx, int dxs,
       int dxo, float *__restrict__ dhw, float *__restrict__ dhb, double *__restrict__ loss,
       float inv_n) {
    __shared__ float s_hw[32], s_hb[2];
    __shared__ float red[8][35];
    if (threadIdx.x < 32) s_hw[threadIdx.x] = hw[threadIdx.x];
    if (threadIdx.x < 2) s_hb[threadIdx.x] = hb[threadIdx.x];
    __syncthreads();
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float part[35];
#pragma unroll
    for (int k = 0; k < 35; ++k) part[k] = 0.0f;
    if (p < npix) {
        float xv[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) xv[c] = __bfloat162float(x[p * xs + xo + c]);
        float o0 = s_hb[0], o1 = s_hb[1];
#pragma unroll
        for (int c = 0; c < 16; ++c) { o0 = fmaf(s_hw[c], xv[c], o0); o1 = fmaf(s_hw[16 + c], xv[c], o1); }
        const float sg = 1.0f / (1.0f + __expf(-o1));
        if (f0) f0[p] = base ? fmaxf(fmaf(f_scale, o0, base[p]), 0.0f) : o0;
        if (w) w[p] = sg;
        if (ft) {
            const float e0 = o0 - ft[p], e1 = sg - wt[p];
            const float d0 = 2.0f * e0 * inv_n, d1 = 2.0f * e1 * inv_n * sg * (1.0f - sg);
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                part[c] = d0 * xv[c];
                part[16 + c] = d1 * xv[c];
                dx[p * dxs + dxo + c] = __float2bfloat16_rn(s_hw[c] * d0 + s_hw[16 + c] * d1);
            }
            part[32] = d0;
            part[33] = d1;
            part[34] = (e0 * e0 + e1 * e1) * inv_n;
        }
    }
    if (!ft) return;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 35; ++k) {
        float v = warp_sum(part[k]);
        if (lane == 0) red[wp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 35) {
        float s = 0.0f;
        for (int i = 0; i < 8; ++i) s += red[i][threadIdx.x];
        if (threadIdx.x < 32) atomicAdd(dhw + threadIdx.x, s);
        else if (threadIdx.x < 34) atomicAdd(dhb + threadIdx.x - 32, s);
        else atomicAdd(loss, (double)s);
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, long long n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// ------------------------------------------------------------------- host launchers

template <int CIN, int COUT>
static cudaError_t launch_conv_t(const bf16 *x, int n, int H, int W, int xs, int xo, const bf16 *wt,
                                 const float *b, bf16 *y, int ys, int yo, int relu, cudaStream_t st) {
    constexpr int smem = conv_smem_bytes<CIN, COUT>();
    static bool attr_set = false;        // per process; same value on every device
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_conv3x3_mma<CIN, COUT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int ntiles = n * ((W + kCvTW - 1) / kCvTW) * ((H + kCvTH - 1) / kCvTH);
    const int blocks_per_sm = smem > 110 * 1024 ? 1 : 2;
    const int grid = std::min(ntiles, 148 * blocks_per_sm * 2);
    ++g_launch_count;
    k_conv3x3_mma<CIN, COUT><<<grid, 128, smem, st>>>(x, n, H, W, xs, xo, wt, b, y, ys, yo, relu);
    return cudaGetLastError();
}

// 0: the tcgen05 / tensor-memory kernel for the shapes where it is not slower (else
// mma.sync); 1: mma.sync always; 2: the tensor-memory kernel wherever it tiles the image
static std::atomic<int> g_conv_path{0};

cudaError_t unet_conv3x3(const void *x, int n, int H, int W, int cin, int xs, int xo, const void *wt,
                         const float *b, int cout, void *y, int ys, int yo, int relu, cudaStream_t st) {
    const int path = g_conv_path.load(std::memory_order_relaxed);
    if (path != 1) {
        const cudaError_t e = unet_conv3x3_tc(x, n, H, W, cin, xs, xo, wt, b, cout, y, ys, yo, relu, st, path == 2);
        if (e != cudaErrorNotSupported) return e;
    }
    const bf16 *X = static_cast<const bf16 *>(x);
    const bf16 *Wt = static_cast<const bf16 *>(wt);
    bf16 *Y = static_cast<bf16 *>(y);
#define CONV_CASE(CI, CO) \
    if (cin == CI && cout == CO) return launch_conv_t<CI, CO>(X, n, H, W, xs, xo, Wt, b, Y, ys, yo, relu, st);
    CONV_CASE(16, 16) CONV_CASE(16, 32) CONV_CASE(32, 32) CONV_CASE(32, 64) CONV_CASE(64, 64)
    CONV_CASE(96, 32) CONV_CASE(48, 16) CONV_CASE(32, 16) CONV_CASE(64, 32) CONV_CASE(32, 96)
    CONV_CASE(16, 48) CONV_CASE(64, 96)
#undef CONV_CASE
    return cudaErrorInvalidValue;
}

bool unet_conv_supported(int cin, int cout) {
    const int pairs[][2] = {{16, 16}, {16, 32}, {32, 32}, {32, 64}, {64, 64}, {96, 32}, {48, 16},
                            {32, 16}, {64, 32}, {32, 96}, {16, 48}, {64, 96}};
    for (auto &p : pairs) if (p[0] == cin && p[1] == cout) return true;
    return false;
}

template <int CIN, int COUT>
static cudaError_t launch_wgrad_t(const bf16 *x, int n, int H, int W, int xs, int xo, const bf16 *dy,
                                  int dys, int dyo, float *dw, float *db, cudaStream_t st) {
    constexpr int smem = wgrad_smem_bytes<CIN, COUT>();
    static bool attr_set = false;        // per process; same value on every device
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_conv3x3_wgrad_mma<CIN, COUT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int ntiles = n * ((W + kCvTW - 1) / kCvTW) * ((H + kCvTH - 1) / kCvTH);
    // about two blocks per SM in all; each block adds its partial sums to dW once
    constexpr int groups = (COUT / 16) / wgrad_mgroups<CIN, COUT>();
    const dim3 grid(std::min(ntiles, std::max(1, 296 / groups)), groups);
    ++g_launch_count;
    k_conv3x3_wgrad_mma<CIN, COUT><<<grid, 288, smem, st>>>(x, n, H, W, xs, xo, dy, dys, dyo, dw, db);
    return cudaGetLastError();
}

cudaError_t unet_conv3x3_wgrad(const void *x, int n, int H, int W, int cin, int xs, int xo,
                               const void *dy, int dys, int dyo, int cout, float *dw, float *db,
                               cudaStream_t st) {
    const bf16 *X = static_cast<const bf16 *>(x);
    const bf16 *D = static_cast<const bf16 *>(dy);
#define WGRAD_CASE(CI, CO) \
    if (cin == CI && cout == CO) return launch_wgrad_t<CI, CO>(X, n, H, W, xs, xo, D, dys, dyo, dw, db, st);
    WGRAD_CASE(16, 16) WGRAD_CASE(16, 32) WGRAD_CASE(32, 32) WGRAD_CASE(32, 64) WGRAD_CASE(64, 64)
    WGRAD_CASE(96, 32) WGRAD_CASE(48, 16) WGRAD_CASE(32, 16) WGRAD_CASE(64, 32) WGRAD_CASE(32, 96)
    WGRAD_CASE(16, 48) WGRAD_CASE(64, 96)
#undef WGRAD_CASE
    return cudaErrorInvalidValue;
}

cudaError_t unet_weights_to_bf16(const float *w, int cout, int cin, void *wf, void *wb, cudaStream_t st) {
    const int n = cout * 9 * cin;
    ++g_launch_count;
    k_weights_to_bf16<<<(n + 255) / 256, 256, 0, st>>>(w, cout, cin, static_cast<bf16 *>(wf),
                                                       static_cast<bf16 *>(wb));
    return cudaGetLastError();
}

static unsigned nblk(long long n) { return (unsigned)((n + 255) / 256); }

cudaError_t unet_maxpool2(const void *x, int n, int H, int W, int xs, int xo, int C, void *y, int ys,
                          int yo, cudaStream_t st) {
    ++g_launch_count;
    k_maxpool2<<<nblk((long long)n * (H / 2) * (W / 2) * C), 256, 0, st>>>(
        static_cast<const bf16 *>(x), n, H, W, xs, xo, C, static_cast<bf16 *>(y), ys, yo);
    return cudaGetLastError();
}

cudaError_t unet_maxpool2_bwd(const void *x, int n, int H, int W, int xs, int xo, int C, const void *dy,
                              int dys, int dyo, void *dx, int dxs, int dxo, int acc, cudaStream_t st) {
    ++g_launch_count;
    k_maxpool2_bwd<<<nblk((long long)n * (H / 2) * (W / 2) * C), 256, 0, st>>>(
        static_cast<const bf16 *>(x), n, H, W, xs, xo, C, static_cast<const bf16 *>(dy), dys, dyo,
        static_cast<bf16 *>(dx), dxs, dxo, acc);
    return cudaGetLastError();
}

cudaError_t unet_upsample2(const void *x, int n, int H, int W, int xs, int xo, int C, void *y, int ys,
                           int yo, cudaStream_t st) {
    ++g_launch_count;
    k_upsample2<<<nblk((long long)n * 4 * H * W * C), 256, 0, st>>>(
        static_cast<const bf16 *>(x), n, H, W, xs, xo, C, static_cast<bf16 *>(y), ys, yo);
    return cudaGetLastError();
}

cudaError_t unet_upsample2_bwd(const void *dy, int n, int H, int W, int dys, int dyo, int C, void *dx,
                               int dxs, int dxo, cudaStream_t st) {
    ++g_launch_count;
    k_upsample2_bwd<<<nblk((long long)n * (H / 2) * (W / 2) * C), 256, 0, st>>>(
        static_cast<const bf16 *>(dy), n, H, W, dys, dyo, C, static_cast<bf16 *>(dx), dxs, dxo);
    return cudaGetLastError();
}

cudaError_t unet_relu_bwd(const void *a, int as, int ao, const void *dy, int dys, int dyo, void *dz,
                          int dzs, int dzo, long long npix, int C, cudaStream_t st) {
    ++g_launch_count;
    k_relu_bwd<<<nblk(npix * C), 256, 0, st>>>(static_cast<const bf16 *>(a), as, ao,
                                              static_cast<const bf16 *>(dy), dys, dyo,
                                              static_cast<bf16 *>(dz), dzs, dzo, npix, C);
    return cudaGetLastError();
}

cudaError_t unet_head(const void *x, int xs, int xo, long long npix, const float *hw, const float *hb,
                      float *f0, float *w, const float *base, float f_scale, const float *ft,
                      const float *wt, void *dx, int dxs, int dxo, float *dhw, float *dhb, double *loss,
                      cudaStream_t st) {
    ++g_launch_count;
    k_head<<<nblk(npix), 256, 0, st>>>(static_cast<const bf16 *>(x), xs, xo, npix, hw, hb, f0, w, base,
                                       f_scale, ft, wt,
                                       static_cast<bf16 *>(dx), dxs, dxo, dhw, dhb, loss,
                                       (float)(1.0 / (double)npix));
    return cudaGetLastError();
}

cudaError_t unet_pack_input(const float *a, float sa, const float *b, float sb, long long npix, void *x,
                            cudaStream_t st) {
    ++g_launch_count;
    k_pack_input<<<nblk(npix), 256, 0, st>>>(a, sa, b, sb, npix, static_cast<bf16 *>(x));
    return cudaGetLastError();
}

cudaError_t unet_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1,
                      float b2, float eps, int step, cudaStream_t st) {
    const float bc1 = 1.0f - powf(b1, (float)step), bc2 = 1.0f - powf(b2, (float)step);
    ++g_launch_count;
    k_adam<<<nblk(n), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
    return cudaGetLastError();
}

}  // namespace eptv

namespace eptv {
int report_error(int code, const char *msg);   // host.cu
}

using namespace eptv;

static int unet_rc(cudaError_t e) {
    if (e == cudaSuccess) return 0;
    return report_error(EPTV_ERR_CUDA, cudaGetErrorString(e));
}

static bool al16(const void *p) { return (((uintptr_t)p) & 15) == 0; }

extern "C" {

int eptv_unet_conv3x3(const void *d_x, int n, int h, int w, int cin, int x_stride, int x_off,
                      const void *d_wt, const float *d_bias, int cout, void *d_y, int y_stride,
                      int y_off, int relu, void *stream) {
    if (!d_x || !d_wt || !d_y) return report_error(EPTV_ERR_ARG, "NULL argument");
    if (n < 1 || h < 1 || w < 1) return report_error(EPTV_ERR_ARG, "bad tensor size");
    if (!unet_conv_supported(cin, cout)) return report_error(EPTV_ERR_ARG, "unsupported channel pair");
    if (x_stride < x_off + cin || y_stride < y_off + cout || (x_stride % 8) || (x_off % 8) ||
        (y_stride % 2) || (y_off % 2))
        return report_error(EPTV_ERR_ARG, "bad channel stride/offset (input: multiples of 8)");
    if (!al16(d_x) || !al16(d_wt) || (((uintptr_t)d_y) & 3))
        return report_error(EPTV_ERR_ARG, "input and weights must be 16-byte aligned");
    return unet_rc(unet_conv3x3(d_x, n, h, w, cin, x_stride, x_off, d_wt, d_bias, cout, d_y, y_stride,
                                y_off, relu, (cudaStream_t)stream));
}

int eptv_unet_conv3x3_wgrad(const void *d_x, int n, int h, int w, int cin, int x_stride, int x_off,
                            const void *d_dy, int dy_stride, int dy_off, int cout, float *d_dw,
                            float *d_db, void *stream) {
    if (!d_x || !d_dy || !d_dw) return report_error(EPTV_ERR_ARG, "NULL argument");
    if (n < 1 || h < 1 || w < 1) return report_error(EPTV_ERR_ARG, "bad tensor size");
    if (!unet_conv_supported(cin, cout)) return report_error(EPTV_ERR_ARG, "unsupported channel pair");
    if (x_stride < x_off + cin || dy_stride < dy_off + cout || (x_stride % 8) || (x_off % 8) ||
        (dy_stride % 8) || (dy_off % 8))
        return report_error(EPTV_ERR_ARG, "bad channel stride/offset (multiples of 8)");
    if (!al16(d_x) || !al16(d_dy)) return report_error(EPTV_ERR_ARG, "x and dy must be 16-byte aligned");
    return unet_rc(unet_conv3x3_wgrad(d_x, n, h, w, cin, x_stride, x_off, d_dy, dy_stride, dy_off,
                                      cout, d_dw, d_db, (cudaStream_t)stream));
}

int eptv_unet_set_conv_kernel(int mode) {
    if (mode != EPTV_CONV_TENSOR_MEMORY && mode != EPTV_CONV_MMA_SYNC && mode != EPTV_CONV_TENSOR_MEMORY_ALL)
        return report_error(EPTV_ERR_ARG, "bad conv kernel mode");
    g_conv_path.store(mode);
    return 0;
}

int eptv_unet_tc_status(void) {
    int flag = 0;
    const cudaError_t e = unet_tc_status(&flag);
    if (e != cudaSuccess) return report_error(EPTV_ERR_CUDA, cudaGetErrorString(e));
    if (flag) return report_error(EPTV_ERR_TIMEOUT, "a bounded wait of the tensor-core conv ran out");
    return 0;
}

int eptv_unet_weights_to_bf16(const float *d_w, int cout, int cin, void *d_wf, void *d_wb, void *stream) {
    if (!d_w || (!d_wf && !d_wb) || cout < 1 || cin < 1) return report_error(EPTV_ERR_ARG, "bad arguments");
    return unet_rc(unet_weights_to_bf16(d_w, cout, cin, d_wf, d_wb, (cudaStream_t)stream));
}

int eptv_unet_maxpool2(const void *d_x, int n, int h, int w, int x_stride, int x_off, int c, void *d_y,
                       int y_stride, int y_off, void *stream) {
    if (!d_x || !d_y || (h % 2) || (w % 2) || c < 1) return report_error(EPTV_ERR_ARG, "bad arguments");
    return unet_rc(unet_maxpool2(d_x, n, h, w, x_stride, x_off, c, d_y, y_stride, y_off, (cudaStream_t)stream));
}

int eptv_unet_maxpool2_bwd(const void *d_x, int n, int h, int w, int x_stride, int x_off, int c,
                           const void *d_dy, int dy_stride, int dy_off, void *d_dx, int dx_stride,
                           int dx_off, int accumulate, void *stream) {
    if (!d_x || !d_dy || !d_dx || (h % 2) || (w % 2)) return report_error(EPTV_ERR_ARG, "bad arguments");
    return unet_rc(unet_maxpool2_bwd(d_x, n, h, w, x_stride, x_off, c, d_dy, dy_stride, dy_off, d_dx,
                                     dx_stride, dx_off, accumulate, (cudaStream_t)stream));
}

int eptv_unet_upsample2(const void *d_x, int n, int h, int w, int x_stride, int x_off, int c, void *d_y,
                        int y_stride, int y_off, void *stream) {
    if (!d_x || !d_y || c < 1) return report_error(EPTV_ERR_ARG, "bad arguments");
    return unet_rc(unet_upsample2(d_x, n, h, w, x_stride, x_off, c, d_y, y_stride, y_off, (cudaStream_t)stream));
}

int eptv_unet_upsample2_bwd(const void *d_dy, int n, int h, int w, int dy_stride, int dy_off, int c,
                            void *d_dx, int dx_stride, int dx_off, void *stream) {
    if (!d_dy || !d_dx || (h % 2) || (w % 2)) return report_error(EPTV_ERR_ARG, "bad arguments");
    return unet_rc(unet_upsample2_bwd(d_dy, n, h, w, dy_stride, dy_off, c, d_dx, dx_stride, dx_off,
                                      (cudaStream_t)stream));
}

int eptv_unet_relu_bwd(const void *d_a, int a_stride, int a_off, const void *d_dy, int dy_stride,
                       int dy_off, void *d_dz, int dz_stride, int dz_off, long long npix, int c,
                       void *stream) {
    if (!d_a || !d_dy || !d_dz || npix < 1 || c < 1) return report_error(EPTV_ERR_ARG, "bad arguments");
    return unet_rc(unet_relu_bwd(d_a, a_stride, a_off, d_dy, dy_stride, dy_off, d_dz, dz_stride, dz_off,
                                 npix, c, (cudaStream_t)stream));
}

int eptv_unet_head(const void *d_x, int x_stride, int x_off, long long npix, const float *d_hw,
                   const float *d_hb, float *d_f0, float *d_w, const float *d_base, float f_scale,
                   const float *d_ft, const float *d_wt, void *d_dx, int dx_stride, int dx_off,
                   float *d_dhw, float *d_dhb, double *d_loss, void *stream) {
    if (!d_x || !d_hw || !d_hb || npix < 1) return report_error(EPTV_ERR_ARG, "bad arguments");
    if (x_stride < x_off + 16) return report_error(EPTV_ERR_ARG, "bad channel stride/offset");
    if (d_ft && (!d_wt || !d_dx || !d_dhw || !d_dhb || !d_loss || dx_stride < dx_off + 16))
        return report_error(EPTV_ERR_ARG, "training mode needs targets and gradient buffers");
    return unet_rc(unet_head(d_x, x_stride, x_off, npix, d_hw, d_hb, d_f0, d_w, d_base, f_scale, d_ft,
                             d_wt, d_dx, dx_stride, dx_off, d_dhw, d_dhb, d_loss, (cudaStream_t)stream));
}

int eptv_unet_pack_input(const float *d_a, float scale_a, const float *d_b, float scale_b,
                         long long npix, void *d_x, void *stream) {
    if (!d_a || !d_x || npix < 1) return report_error(EPTV_ERR_ARG, "bad arguments");
    if (!al16(d_x)) return report_error(EPTV_ERR_ARG, "x must be 16-byte aligned");
    return unet_rc(unet_pack_input(d_a, scale_a, d_b, scale_b, npix, d_x, (cudaStream_t)stream));
}

int eptv_unet_adam(float *d_p, const float *d_g, float *d_m, float *d_v, long long n, float lr,
                   float beta1, float beta2, float eps, int step, void *stream) {
    if (!d_p || !d_g || !d_m || !d_v || n < 1 || step < 1) return report_error(EPTV_ERR_ARG, "bad arguments");
    return unet_rc(unet_adam(d_p, d_g, d_m, d_v, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream));
}

}  // extern "C"
