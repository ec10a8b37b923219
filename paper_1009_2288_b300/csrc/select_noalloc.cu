// Order-statistic selection that allocates nothing: a variant of the radix-select
// kernel (k5_radix_pass) whose working memory -- a 4096-bucket histogram, the
// finishing-block ticket and the prefix/rank state -- lives in one file-scope device
// array instead of a geometry handle's workspace.
//
// Who needs it: code that may not call cudaMalloc -- for example a host function that
// runs while another library owns the device allocator, a memory-capped service
// process that has reserved all of its device memory up front, or a callback that must
// not take the allocator's locks.  Such a caller passes its input and output buffers
// and nothing else.
//
// Every GPU that loads this library keeps the array (16.5 KB) until the process exits.
// All calls on one device share it and it keeps the last call's contents, so each call
// first clears the histogram and the ticket; calls that overlap on the GPU (different
// streams, or host threads racing) corrupt each other's results.
#include <mutex>

#include "eptv_internal.cuh"
#include "kernels.cuh"

namespace eptv {

constexpr int kNaBins = kHistBins;                // 12-bit buckets (pass 2 uses 256)
constexpr int kNaTicket = kNaBins;                // finishing-block ticket
constexpr int kNaPrefix = kNaBins + 1;            // selected bit prefix so far
constexpr int kNaRankLo = kNaBins + 2;            // remaining 1-based rank (64-bit)
constexpr int kNaRankHi = kNaBins + 3;
constexpr int kNaWords = kNaBins + 64;            // 16.6 KB, 256-byte multiple
constexpr long kNaMaxN = 2147483647L;             // bucket counts are 32-bit

static __device__ __align__(256) unsigned int g_noalloc_scratch[kNaWords];

__global__ void na_clear(unsigned int *scr) {
    for (int i = threadIdx.x; i < kNaWords; i += blockDim.x) scr[i] = 0u;
}

// One pass over n values: pass 0 buckets the top 12 bits, pass 1 the next 12 bits of
// keys sharing the pass-0 prefix, pass 2 the low 8 bits of keys sharing the 24-bit
// prefix.  The last block to finish narrows the prefix and, after pass 2, writes the
// selected value.
__global__ void __launch_bounds__(256)
na_radix_pass(const float *__restrict__ vals, long long n, long long k, int pass,
              unsigned int *scr, float *out)
{
    __shared__ unsigned int sh[kNaBins];
    __shared__ unsigned int s_cnt[256];
    __shared__ int s_last;
    const int nbins = (pass == 2) ? 256 : kNaBins;
    for (int b = threadIdx.x; b < nbins; b += 256) sh[b] = 0u;
    __syncthreads();
    const unsigned int prefix = (pass == 0) ? 0u : __ldcg(scr + kNaPrefix);
    const long long e0 = (long long)blockIdx.x * 2048;
    for (int q = 0; q < 8; ++q) {
        const long long e = e0 + q * 256 + threadIdx.x;
        if (e < n) sel_hist_add(sh, sel_key(__ldg(vals + e)), pass, prefix);   // as the handle-based selection
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += 256) {
        const unsigned int c = sh[b];
        if (c) atomicAdd(scr + b, c);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int ticket = atomicAdd(scr + kNaTicket, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last block: find the bucket that holds the remaining rank
    const int per = nbins / 256;
    unsigned int local = 0;
    for (int q = 0; q < per; ++q) local += __ldcg(scr + threadIdx.x * per + q);
    s_cnt[threadIdx.x] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long rank = (pass == 0)
            ? (unsigned long long)k
            : ((unsigned long long)__ldcg(scr + kNaRankHi) << 32) | __ldcg(scr + kNaRankLo);
        unsigned long long cum = 0;
        int tb = 0;
        for (; tb < 255; ++tb) { if (cum + s_cnt[tb] >= rank) break; cum += s_cnt[tb]; }
        int b = tb * per;
        for (int q = 0; q < per; ++q, ++b) {
            const unsigned int c = __ldcg(scr + b);
            if (cum + c >= rank || q == per - 1) break;
            cum += c;
        }
        rank -= cum;
        unsigned int pre = prefix;
        if (pass == 0) pre = (unsigned int)b;
        else if (pass == 1) pre = (pre << 12) | (unsigned int)b;
        else pre = (pre << 8) | (unsigned int)b;
        scr[kNaPrefix] = pre;
        scr[kNaRankLo] = (unsigned int)(rank & 0xFFFFFFFFull);
        scr[kNaRankHi] = (unsigned int)(rank >> 32);
        scr[kNaTicket] = 0u;                       // re-arm for the next pass
        if (pass == 2) *out = __uint_as_float(pre);
    }
    __syncthreads();
    for (int q = 0; q < per; ++q) scr[threadIdx.x * per + q] = 0u;   // clear for the next pass
}

// Device address of the scratch array, looked up once per device.
static std::mutex g_na_mutex;
static unsigned int *g_na_ptr[64] = {};

static int na_scratch_for_current_device(unsigned int **ptr, const char **err) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        *err = "no current CUDA device (or device ordinal >= 64)";
        return EPTV_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            *err = cudaGetErrorString(e);
            return EPTV_ERR_CUDA;
        }
        g_na_ptr[dev] = static_cast<unsigned int *>(p);
    }
    *ptr = g_na_ptr[dev];
    return 0;
}

int select_kth_noalloc(const float *d_vals, long n, long k, float *d_out, cudaStream_t st,
                       const char **err) {
    if (!d_vals || !d_out) { *err = "NULL argument"; return EPTV_ERR_ARG; }
    if (n < 1 || n > kNaMaxN) { *err = "n must be in [1, 2^31 - 1]"; return EPTV_ERR_ARG; }
    if (k < 1 || k > n) { *err = "k must be in [1, n]"; return EPTV_ERR_ARG; }
    // an error left by earlier work on this thread is reported as such and left pending
    const cudaError_t e0 = cudaPeekAtLastError();
    if (e0 != cudaSuccess) { *err = "a CUDA error from earlier work is pending on this thread"; return EPTV_ERR_CUDA; }
    unsigned int *scr = nullptr;
    int rc = na_scratch_for_current_device(&scr, err);
    if (rc) return rc;
    // both buffers must live on the current device (the scratch array is this device's)
    int dev = 0;
    cudaGetDevice(&dev);
    for (const void *ptr : {(const void *)d_vals, (const void *)d_out}) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
            cudaGetLastError();
            *err = "cudaPointerGetAttributes failed on an argument";
            return EPTV_ERR_ARG;
        }
        if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) {
            *err = "vals and out must be device memory";
            return EPTV_ERR_ARG;
        }
        if (at.type == cudaMemoryTypeDevice && at.device != dev) {
            *err = "vals and out must be on the current device";
            return EPTV_ERR_ARG;
        }
    }
    const int nblk = (int)((n + 2047) / 2048);
    na_clear<<<1, 256, 0, st>>>(scr);
    for (int pass = 0; pass <= 2; ++pass)
        na_radix_pass<<<nblk, 256, 0, st>>>(d_vals, (long long)n, (long long)k, pass, scr, d_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { *err = cudaGetErrorString(e); return EPTV_ERR_CUDA; }
    return 0;
}

int report_error(int code, const char *msg);   // host.cu: sets eptv_last_error()

}  // namespace eptv

extern "C" int eptv_select_kth_noalloc(const float *d_vals, long n, long k, float *d_out,
                                       void *stream) {
    const char *err = "";
    const int rc = eptv::select_kth_noalloc(d_vals, n, k, d_out, (cudaStream_t)stream, &err);
    if (rc) return eptv::report_error(rc, err);
    return 0;
}
