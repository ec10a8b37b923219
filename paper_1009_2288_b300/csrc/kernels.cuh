// Kernel-family declarations, launch arguments and the batch container shared by the
// host orchestration (host.cu) and the kernel files.
#pragma once

#include <vector>

#include "eptv_internal.cuh"

namespace eptv {

// Kernel families: each has its own blocks-per-slice map.
enum Family {
    FAM_K1 = 0,   // projector: n_views * ceil(n_bins / 32) blocks
    FAM_K2,       // back projector / TV stencils: ceil(nx / 32) * ceil(ny / 16) blocks
    FAM_IMG,      // image elementwise with transpose: ceil(nx / 32) * ceil(ny / 32) blocks
    FAM_SINO,     // sinogram elementwise: ceil(n_rays / 1024) blocks
    FAM_EDGE,     // half-edge arrays: ceil(n_edges / 2048) blocks
    FAM_TV,       // fused TV descent: ceil(nx / 32) * ceil(ny / kGdTileRows) blocks
    FAM_SPMV_P,   // stored P: ceil(n_rays / 32) blocks (8 warps per 32-ray slice)
    FAM_SPMV_PT,  // stored P^T: ceil(ny / 8) * ceil(nx / 32) blocks (32 x 8 pixel tiles)
    FAM_COUNT
};

constexpr int kTileW = 32, kTileH = 8;
constexpr int kGdTileRows = 8;
constexpr int kHistBins = 4096;    // radix-select histogram (12 bits per pass)

// Radix selection over FP32 bit patterns (the sigma order statistic and the generic
// selections): the key of a value (-0 counts as +0; the selections take non-negative or
// same-sign inputs, whose keys order like the values), and one pass's histogram update:
// pass 0 buckets the top 12 bits, pass 1 the next 12 bits of keys with the pass-0 prefix,
// pass 2 the low 8 bits of keys with the 24-bit prefix.
__device__ __forceinline__ unsigned int sel_key(float x) {
    unsigned int b = __float_as_uint(x);
    return (b == 0x80000000u) ? 0u : b;     // -0 -> +0
}

__device__ __forceinline__ void sel_hist_add(unsigned int *sh, unsigned int key, int pass,
                                             unsigned int prefix) {
    if (pass == 0) atomicAdd(&sh[key >> 20], 1u);
    else if (pass == 1) { if ((key >> 20) == prefix) atomicAdd(&sh[(key >> 8) & 0xFFFu], 1u); }
    else { if ((key >> 8) == prefix) atomicAdd(&sh[key & 0xFFu], 1u); }
}

// Finalisers run by the last block of a reduction.
enum Fin {
    FIN_NONE = 0,
    FIN_NORM,        // sc[SC_NORM] = sum0, sc[SC_NORM2] = sum1
    FIN_QQ_TO_A,     // qq = sum0; a = gamma / qq
    FIN_GAMMA0,      // gamma = sum0
    FIN_B,           // b = sum0 / gamma; gamma = sum0
};

enum ImgSel { IMG_U = 0, IMG_S = 1 };
enum SinoSel { SINO_R = 0, SINO_Q = 1 };

struct ProjArgs {
    int img;                    // ImgSel
    int out;                    // SinoSel
    int resid;                  // out = y - P img
    int fin;                    // Fin
    const float *img_override;  // single-slice calls with caller buffers
    const float *imgT_override;
    float *out_override;
    const float *y_override;    // data for resid mode (default: S.y)
    int no_T;                   // ignore the slice's transposed copy
};

struct BackArgs {
    int out;                    // 0: s (+ sT), 1: t, 2: u
    int write_T;                // also write the transposed image
    int fin;
    const float *in_override;   // sinogram input (default: r)
    float *out_override;
    int eq11;                   // the interpolating back projector of Eq. (11) for this call
};

// Launch plan of K4p for a batch: region shape (tiles), trial template, block size, grid.
struct P2Plan {
    int ok = 0;
    int rtx = 0, rty = 0, kt = 0, nt = 0, blocks = 0;
    size_t smem = 0;
};

struct Batch {
    int n = 0;
    SliceDev *d_sd = nullptr;
    std::vector<SliceDev> h_sd;
    int *d_start = nullptr;         // [FAM_COUNT][n + 1]
    std::vector<int> h_start;
    unsigned int *d_counters = nullptr;   // [n][counter stride]: reduction tickets (SliceDev::ctr)
    unsigned long long *d_acc = nullptr;  // [n][kPartialStride][kAccCopies][kAccStride]: exact sums
    double *d_partials = nullptr;         // [max blocks][kPartialStride]
    unsigned int *d_hist = nullptr;       // [n][kHistBins]
    ParamsDev *d_params = nullptr;
    int k1_seg = 8;        // projector: warps (row segments) per 32-ray block (4, 8, 16)
    int k2_vg = 4;         // back projector: view groups per 4-pixel strip (1, 2, 4, 8)
    int stored = 0;        // 1: P and P^T are applied from the stored matrices (stored.cu)
    int stored_pt = 0;     // 1: only P^T is applied from the stored matrix (P on the fly)
    int bp_eq11 = 0;       // 1: P^T is the interpolating back projector of Eq. (11)
    // persistent (P2) kernel K4p (tv_p2.cu): region starts of the current plan, the grid
    // barrier counter, the accumulator sets, and the plan the starts were uploaded for
    int *d_p2start = nullptr;             // [n + 1]
    unsigned int *d_p2bar = nullptr;      // [2]: arrival count, its value at the next launch
    unsigned long long *d_p2acc = nullptr;  // [n][3][kPartialStride][kAccCopies][kAccStride]
    unsigned int *d_p2hist = nullptr;     // [n][kP2HistWords]
    int p2_rtx = 0, p2_rty = 0;           // shape whose starts are in d_p2start (0: none)
    std::vector<int> h_p2start;
    int p2_disabled = 0;                  // 1: cooperative capture failed: per-iteration K4
    int p2_forbid = 0;                    // 1: the caller asked for per-iteration K4
    int p2_bar_extra = 0;                 // test hook: phantom blocks the barrier waits for
    long long p2_wait_cycles = 2000000000ll;  // bound of one barrier wait (~1 s at 2 GHz)
    P2Plan p2;                            // plan of the next (P2) solves (ok = 0: K4)
    TileMap map(int fam) const { return TileMap{d_start + fam * (n + 1), n}; }
    int blocks(int fam) const { return h_start[fam * (n + 1) + n]; }
};

// The scalar a finalisation mode divides by (SC_GAMMA), read by the caller at kernel start
// so that the finishing block's tail waits on no global load (only that block writes it).
__device__ __forceinline__ double fin_gamma(const double *sc, int fin) {
    return (fin == FIN_QQ_TO_A || fin == FIN_B) ? sc[SC_GAMMA] : 0.0;
}

__device__ __forceinline__ void finalize(double *sc, int fin, double s0, double s1, double gamma) {
    if (!isfinite(s0) || !isfinite(s1)) sc[SC_NONFINITE] = 1.0;
    switch (fin) {
    case FIN_NORM: sc[SC_NORM] = s0; sc[SC_NORM2] = s1; break;
    case FIN_QQ_TO_A: sc[SC_QQ] = s0; sc[SC_A] = (s0 > 0.0) ? gamma / s0 : 0.0; break;
    case FIN_GAMMA0: sc[SC_GAMMA] = s0; break;
    case FIN_B:
        sc[SC_B] = (gamma > 0.0) ? s0 / gamma : 0.0;
        sc[SC_GAMMA] = s0;
        break;
    default: break;
    }
}

struct GdArgs {
    int first;               // 1: the iterate is v itself (no previous step to apply)
    int last;                // 1: write the final edge weights (if S.wout is set)
    int n_trials;            // Armijo trial steps evaluated (1 for fixed steps, 0: gradient only)
    int energy_only_fin;     // store the energy in SC_E_FIRST, take no step decision
    const float *fprev;      // previous iterate (null: slice ping-pong / v)
    const float *gprev;      // previous gradient (null: slice ping-pong)
    const float *v;          // (P2) input (null: S.u)
    float *fout, *gout;      // outputs (null: slice ping-pong)
    int write_f;             // store the iterate
};

// Arguments of the persistent (P2) kernel K4p (its barrier words, accumulator sets and
// selection histograms are SliceDev::p2bar / p2acc / p2hist: kP2Sets sets of kP2SetWords
// words and kP2HistWords histogram words per slice).
constexpr int kP2Sets = 3;
constexpr size_t kP2SetWords = (size_t)kPartialStride * kAccCopies * kAccStride;
constexpr int kP2HistWords = 2 * kHistBins + 256;     // passes 0, 1 (12 bits), 2 (8 bits)
struct P2Args {
    const float *v;               // (P2) input (null: S.u)
    float *out;                   // result max(f, 0) (null: S.u and S.uT)
    int n_gd, n_trials;
    int bar_extra;                // blocks the barrier waits for beyond the grid (tests: > 0)
    long long wait_cycles;        // bound of one barrier wait in SM cycles
    int fold;                     // v = u + a s: the CGLS's last update (u += a s), applied on load
};

int p2_plan(Batch &B, int n_trials, int n_gd, P2Plan *plan);
void p2_region_starts(const Batch &B, int rtx, int rty, std::vector<int> &starts);
cudaError_t launch_p2(const Batch &B, const P2Plan &plan, const P2Args &pa, cudaStream_t st);

// Stored-matrix operator (stored.cu): device CSR matrices of P (rows = rays) and P^T
// (rows = pixels), rows padded to multiples of 4 entries.
struct StoredMatrices {
    int *p_ptr = nullptr, *p_col = nullptr;
    float *p_val = nullptr;
    long long nnz_p = 0;
    int *pt_ptr = nullptr, *pt_col = nullptr;
    float *pt_val = nullptr;
    long long nnz_pt = 0;
    // SELL-32 copies read by the SpMV kernels: slice offsets, row length per slice, entries
    int *p_sptr = nullptr, *p_slen = nullptr, *p_scol = nullptr;
    float *p_sval = nullptr;
    long long sell_p = 0;
    int *pt_sptr = nullptr, *pt_slen = nullptr, *pt_scol = nullptr;
    float *pt_sval = nullptr;
    long long sell_pt = 0;
    int pt_keep = 0;             // leading P^T slices kept in L2 (see SliceDev::pt_keep)
};
typedef cudaError_t (*StoredAlloc)(void *ctx, void **p, size_t bytes);
cudaError_t build_stored(const SliceDev &S, const SliceDev *d_sd, StoredAlloc alloc, void *ctx,
                         StoredMatrices *m, cudaStream_t st);
void launch_spmv_p(const Batch &B, const ProjArgs &a, cudaStream_t st);
// parameter checks and the device copy of a parameter record (host.cu)
void fill_params(const eptv_params *p, ParamsDev *d);
int check_params(const eptv_params *p);
int report_error(int code, const char *msg);
int select_kth_noalloc(const float *d_vals, long n, long k, float *d_out, cudaStream_t st,
                       const char **err);

void launch_quality(const Batch &B, const float *f, const float *r, int rx0, int ry0, int rw, int rh,
                    double scale2, unsigned char *bf, unsigned char *br, cudaStream_t st);
void launch_spmv_pt(const Batch &B, const BackArgs &a, cudaStream_t st);

// Kernel launches issued by this thread (graph captures included); read by the host
// code to report how many kernels a call ran.
extern thread_local long long g_launch_count;

// Launchers (stream-ordered, no host synchronisation).
void launch_project(const Batch &B, const ProjArgs &a, cudaStream_t st);
void launch_backproject(const Batch &B, const BackArgs &a, cudaStream_t st);
void launch_cgls_update_r(const Batch &B, cudaStream_t st);                 // r -= a q
void launch_cgls_update_us(const Batch &B, int update_s, cudaStream_t st);  // u += a s; s = t + b s
void launch_sigma(const Batch &B, const float *v_override, cudaStream_t st);
void launch_gd_iter(const Batch &B, const GdArgs &ga, int iter, cudaStream_t st);
void launch_gd_finish(const Batch &B, int n_gd, const float *f0_override, float *out_override,
                      cudaStream_t st);
void launch_select_generic(const Batch &B, const TileMap &m, int nblk, const float *vals,
                           long long n, long long k, float *out, cudaStream_t st);
void launch_set_scalar(const Batch &B, int which, double value, cudaStream_t st);
void launch_transpose(const Batch &B, const float *src, float *dst, cudaStream_t st);

}  // namespace eptv
