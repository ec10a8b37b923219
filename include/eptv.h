/*
 * eptv.h -- C ABI of the B300 (sm_103a) EPTV reconstruction library (libeptv.so).
 *
 * Method: Tian, Jia, Yuan, Pan, Jiang, "GPU-based low dose CT reconstruction via
 * edge-preserving total variation regularization".  The library computes
 *   E(f) = mu/2 |P f - y|^2 + J(f),  f >= 0                              (Eq. 2)
 *   J(f) = sum_e w_e T_e(f),  w_e = exp(-(T_e / sigma)^2)            (Eqs. 4, 5)
 * with P the fan-beam system matrix whose element p_ij is the length of ray i inside
 * pixel j (Eq. 1, Sec. 2.1), T_e the half-point magnitude of Eq. (A3), and the
 * two-step iteration of Sec. 2.2: (P1) CGLS on |P f - y|^2 (App. I), (P2) gradient
 * descent with Armijo line search on lambda/2 |f - v|^2 + J(f) with the weights
 * recomputed every descent iteration (Eqs. 8, 9, A2), then the positivity clamp.
 *
 * Conventions
 *   image   float32, row-major [ny][nx] (x fastest); pixel (i, j) covers
 *           [x0 + i dx, x0 + (i+1) dx] x [y0 + j dy, y0 + (j+1) dy] mm with
 *           x0 = -nx dx / 2, y0 = -ny dy / 2; values in 1/mm.
 *   sinogram float32, [n_views][n_bins] (bins fastest); values are line integrals.
 *   view v  angle theta_v = angles[v] (radians) or 2 pi v / n_views; source at
 *           sid (cos theta_v, sin theta_v) mm; central ray towards the isocentre.
 *   bin k   fan angle beta_k = k' dbeta (arc detector) or atan(k' dbeta) (flat),
 *           k' = k - (n_bins - 1)/2 + bin_offset, measured counter-clockwise from the
 *           central ray.
 *
 * Memory and streams
 *   Every d_* pointer is device memory owned by the caller (e.g. a torch tensor), 4-byte
 *   aligned at least, and must stay valid until the stream has run the call.  Pointers
 *   named h_* are host memory.  `stream` is a cudaStream_t (NULL = legacy default
 *   stream).  Calls are asynchronous on `stream` unless they return host results
 *   (documented per call), in which case they synchronise that stream before returning.
 *   A geometry handle owns device workspace (ray tables, solver vectors, reduction
 *   partials); calls that use the same handle must be issued on one stream or otherwise
 *   serialised.  The library never falls back to the CPU.
 *
 * Errors
 *   Every int-returning call returns 0 (EPTV_OK) or a negative code; the message of the
 *   last failure on the calling thread is available from eptv_last_error().  Argument
 *   errors are detected before any work is queued.
 */
#ifndef EPTV_H
#define EPTV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EPTV_OK               0
#define EPTV_ERR_ARG         -1   /* invalid argument (null pointer, bad size, ...)      */
#define EPTV_ERR_CUDA        -2   /* a CUDA runtime call failed                          */
#define EPTV_ERR_NONFINITE   -3   /* a reduction met a NaN or infinity                   */
#define EPTV_ERR_TIMEOUT     -4   /* a bounded device wait ran out                       */
#define EPTV_ERR_NOMEM       -5   /* device allocation failed                            */
#define EPTV_WARN_LINESEARCH  1   /* reported in stats: some Armijo searches found no step */

#define EPTV_DETECTOR_ARC   0
#define EPTV_DETECTOR_FLAT  1

#define EPTV_WEIGHTS_EPTV   0     /* w = exp(-(T/sigma)^2), Eq. (5)                        */
#define EPTV_WEIGHTS_ONE    1     /* w = 1: plain TV, the special case of Sec. 4           */
#define EPTV_WEIGHTS_PRIOR  2     /* w from a per-pixel prior map for the first prior_iters */

#define EPTV_STEP_ARMIJO    0
#define EPTV_STEP_FIXED     1

#define EPTV_OPERATOR_ON_THE_FLY 0   /* P, P^T recomputed by the kernels at each use (default) */
#define EPTV_OPERATOR_STORED     1   /* P, P^T stored as CSR matrices in device memory         */
#define EPTV_OPERATOR_EQ11       2   /* P on the fly, P^T = the interpolating back projector of
                                        Eq. (11) (an approximation of the transpose)           */
#define EPTV_OPERATOR_STORED_PT  3   /* P on the fly, P^T from the stored matrix (the same
                                        canonical entries: still the exact transpose)          */

/* Scan geometry (Sec. 3: fan beam, arc detector). */
typedef struct {
    int nx, ny;              /* image size in pixels, 1..8192 each                     */
    double dx, dy;           /* pixel pitch, mm                                        */
    int n_views;             /* number of projection angles, >= 1                      */
    const double *angles;    /* host, n_views radians, or NULL for 2 pi v / n_views    */
    int n_bins;              /* detector bins per view, >= 1                           */
    double dbeta;            /* arc: angular pitch (rad); flat: pitch / sdd             */
    double bin_offset;       /* detector offset in bins (0.25 keeps rays off the grid)  */
    double sid, sdd;         /* source-isocentre and source-detector distances, mm     */
    int detector;            /* EPTV_DETECTOR_ARC or EPTV_DETECTOR_FLAT                */
} eptv_geometry_desc;

/* Solver parameters.  The paper fixes none of these numerically except the sigma
 * percentile (90-95%, Sec. 2.1); eptv_default_params() gives this library's defaults. */
typedef struct {
    int n_outer;             /* outer iterations NI (Sec. 2.2)                          */
    int cgls_iters;          /* M, CGLS iterations per (P1), App. I                     */
    int n_gd;                /* gradient-descent iterations per (P2)                    */
    double lambda;           /* lambda of (P2), Eq. (8)                                 */
    double mu;               /* mu of Eq. (2); used only by the reported energy         */
    double sigma_q;          /* sigma = ceil(q n)-th smallest half-edge magnitude of v  */
    double sigma_floor;      /* lower bound on sigma                                    */
    double eps;              /* smoothing inside the A3 magnitude, 1/mm                 */
    int step_rule;           /* EPTV_STEP_ARMIJO or EPTV_STEP_FIXED                     */
    double t_fixed;          /* step of EPTV_STEP_FIXED                                 */
    double armijo_c;         /* sufficient-decrease constant                            */
    double armijo_shrink;    /* trial step ratio, in (0, 1)                             */
    double armijo_grow;      /* first trial = min(grow * previous step, t_max)          */
    int max_trials;          /* trial steps evaluated per GD iteration, 1..16           */
    double t_max;            /* <= 0: 1/lambda                                          */
    double t_init;           /* first "previous step"; <= 0: 1/lambda                   */
    int weights_mode;        /* EPTV_WEIGHTS_*                                          */
    int prior_iters;         /* outer iterations that use the prior map (PRIOR mode)    */
} eptv_params;

/* Result of one (P2) solve. */
typedef struct {
    double sigma;            /* sigma used (Sec. 2.1)                                   */
    double energy_first;     /* lambda/2|f-v|^2 + J(f) at the first GD iterate          */
    double energy_last;      /* same, frozen weights, after the last accepted step      */
    double t_prev;           /* last accepted step (carried to the next solve)          */
    int n_accepted;          /* GD iterations with a step > 0                           */
    int n_fail;              /* GD iterations whose Armijo search found no step         */
    int status;              /* EPTV_OK or EPTV_WARN_LINESEARCH                         */
} eptv_stats;

/* Result of a reconstruction. */
typedef struct {
    int n_outer;             /* iterations run                                          */
    double sigma_last;       /* sigma of the last (P2) solve                            */
    double t_prev;           /* last accepted Armijo step                               */
    int n_fail;              /* Armijo searches without a step, all iterations          */
    int status;              /* EPTV_OK or EPTV_WARN_LINESEARCH                         */
    long long n_launches;    /* kernels the call ran (graph replays counted per node)    */
} eptv_report;

typedef struct eptv_geometry eptv_geometry;

/* Fills *p with the library defaults.  Never fails. */
void eptv_default_params(eptv_params *p);

/* Builds the ray tables of a scan (host FP64, stored FP32 on the current device) and
 * allocates the solver workspace on the current device.  Sec. 3 geometry.
 * Returns EPTV_ERR_ARG for a bad descriptor, EPTV_ERR_NOMEM / EPTV_ERR_CUDA on device
 * failures.  *out receives the handle; release it with eptv_destroy_geometry. */
int eptv_create_geometry(const eptv_geometry_desc *desc, eptv_geometry **out);

/* Frees the handle and its device memory (synchronises the device first).  NULL is a
 * no-op. */
void eptv_destroy_geometry(eptv_geometry *g);

/* y = P f  (Eq. 1).  d_f: image [ny][nx]; d_y: sinogram [n_views][n_bins], overwritten.
 * p_ij is the exact Siddon intersection length (Sec. 2.1), evaluated on the fly by a
 * ray-driven gather kernel. */
int eptv_project(const eptv_geometry *g, const float *d_f, float *d_y, void *stream);

/* y = P f with a caller-supplied transposed copy d_fT ([nx][ny], may be NULL) of the
 * image: rays that cross columns faster than rows march over d_fT, which keeps the 32
 * lanes of a warp on one cache line.  Launches exactly one kernel (eptv_project adds a
 * transpose into the handle's scratch first). */
int eptv_project_t(const eptv_geometry *g, const float *d_f, const float *d_fT, float *d_y,
                   void *stream);

/* d_fT[i][j] = d_f[j][i] for the handle's image size (d_fT is [nx][ny]). */
int eptv_transpose(const eptv_geometry *g, const float *d_f, float *d_fT, void *stream);

/* f = P^T y, the exact transpose of eptv_project (adjoint identity <Px, y> = <x, P^T y>,
 * Eq. A3 of App. III), evaluated by a scatter-free pixel-driven gather that recomputes
 * each p_ij with the same arithmetic as the projector.  d_f is overwritten. */
int eptv_backproject(const eptv_geometry *g, const float *d_y, float *d_f, void *stream);

/* The paper's pixel-driven back projector, Eq. (11) (Sec. 2.3, App. III), whatever the
 * handle's operator mode:
 *   d_f[iy nx + ix] = (dx dy / dbeta) sum_v y_v(beta*) / l,
 * beta* = fan angle (from the central ray) of the line from the source of view v through
 * the pixel centre, l = its length, y_v(beta*) = linear interpolation of d_y[v nb + k]
 * between the two bins around beta* (bins off the detector read 0).  Flat detector (bins
 * uniform in t = tan beta): weight (dx dy / dbeta) (1 + t*^2) / l.  It approximates P^T
 * (the adjoint identity holds to about 1e-5 for smooth inputs, 1e-4 for noise).  The
 * operator mode EPTV_OPERATOR_EQ11 uses it for every P^T of the handle. */
int eptv_backproject_eq11(const eptv_geometry *g, const float *d_y, float *d_f, void *stream);

/* M CGLS iterations (App. I) for min |P u - y|^2 started at the content of d_u, which
 * is overwritten with u^(M).  d_y: sinogram.  Uses the handle's workspace. */
int eptv_cgls(const eptv_geometry *g, int M, const float *d_y, float *d_u, void *stream);

/* sigma of (P2) (Sec. 2.1): the ceil(q n)-th smallest of the n = (nx+1) ny + nx (ny+1)
 * half-edge magnitudes T of Eq. (A3) of d_v (zero outside the image), floored at
 * p->sigma_floor.  Synchronises `stream`; *h_sigma receives the value. */
int eptv_sigma(const eptv_geometry *g, const eptv_params *p, const float *d_v,
               double *h_sigma, void *stream);

/* One fused evaluation of the (P2) gradient (Eq. 9 with Eq. A2) at f:
 *   d_g = lambda (f - v) + dJ/df,  weights w_e from Eq. (5) with the given sigma (or 1,
 * per p->weights_mode; PRIOR mode is not accepted here).  If h_energy is not NULL the
 * call synchronises and returns lambda/2 |f - v|^2 + J(f) there (FP64 reduction). */
int eptv_tv_gradient(const eptv_geometry *g, const eptv_params *p, double sigma,
                     const float *d_f, const float *d_v, float *d_g, double *h_energy,
                     void *stream);

/* One (P2) solve (Sec. 2.2, step 2): sigma from d_v, then p->n_gd gradient-descent
 * iterations from f = v with Armijo steps (or fixed steps), weights recomputed every
 * iteration, followed by the positivity clamp of step 3.  d_f receives the result.
 * *t_prev_io (host, may be NULL = p->t_init) is the previous accepted step; it is updated.
 * d_weights_opt (may be NULL): receives the final half-edge weights, [2][ny+1][nx+1]
 * (plane 0: x half-edge between pixels (i-1, j) and (i, j) at [0][j][i]; plane 1: y
 * half-edge between (i, j-1) and (i, j) at [1][j][i]).  If out_opt is not NULL the call
 * synchronises and fills it. */
int eptv_tv_step(const eptv_geometry *g, const eptv_params *p, const float *d_v, float *d_f,
                 double *t_prev_io, float *d_weights_opt, eptv_stats *out_opt, void *stream);

/* The EPTV algorithm (Sec. 2.2): d_f holds the start image (zero for f^(0) = 0, or a
 * warm start, clamped to >= 0) and receives f^(n_outer).  d_y: sinogram.
 * d_wprior_opt (may be NULL): per-pixel weight map [ny][nx] used as edge weights
 * (mean of the two pixels beside each half-edge) for the first p->prior_iters
 * iterations when p->weights_mode == EPTV_WEIGHTS_PRIOR.  One outer iteration is
 * captured once into a CUDA graph (cached in the handle) and replayed.  If rep_opt is
 * not NULL the call synchronises and fills it. */
int eptv_reconstruct(const eptv_geometry *g, const eptv_params *p, const float *d_y,
                     float *d_f, const float *d_wprior_opt, eptv_report *rep_opt,
                     void *stream);

/* Reported energy E(f) = mu/2 |P f - y|^2 + J(f; w(f; sigma_ref)) (Eq. 2).
 * Synchronises; *h_energy receives the value. */
int eptv_report_energy(const eptv_geometry *g, const eptv_params *p, double sigma_ref,
                       const float *d_f, const float *d_y, double *h_energy, void *stream);

/* Per-iteration log of the last eptv_reconstruct on this handle: the step taken by every
 * GD iteration (0 where the Armijo search found none), laid out [n_outer][n_gd], and the
 * sigma of every (P2) solve.  Copies min(count, cap) values into each non-NULL host array
 * and the layout into *n_outer / *n_gd (either may be NULL).  Synchronises the device. */
int eptv_get_log(const eptv_geometry *g, double *h_steps, int steps_cap, double *h_sigmas,
                 int sigmas_cap, int *n_outer, int *n_gd);

/* Exact k-th smallest (1-based) of n non-negative finite floats by radix selection on
 * their bit patterns (the order statistic behind sigma).  d_vals: n floats; d_out: one
 * float.  Uses a small workspace of the handle g.  k must be in [1, n]. */
int eptv_select_kth(const eptv_geometry *g, const float *d_vals, long n, long k,
                    float *d_out, void *stream);

/* The same selection as eptv_select_kth, for callers that cannot allocate device memory
 * (a process whose device memory is reserved by another allocator, a memory-capped
 * service, a callback that must not enter the allocator): it needs no geometry handle
 * and allocates nothing.  The paper has no counterpart; this is a library convenience.
 * Its working memory is one 16.5 KB array compiled into the library, kept by every GPU
 * that loads it until the process exits.  n must be in [1, 2^31 - 1] (the histogram
 * counts are 32-bit) and k in [1, n]; otherwise EPTV_ERR_ARG.  d_vals: n non-negative
 * finite floats; d_out: one float; both in device memory of the current device
 * (EPTV_ERR_ARG otherwise).  The first call on a device looks up the array's device
 * address and caches it (make that first call before any stream capture); a
 * cudaDeviceReset of that device invalidates the cached address, so do not call this
 * again in a process after resetting the device.  A CUDA error left pending by earlier
 * work on the calling thread is reported (EPTV_ERR_CUDA) and left pending, not cleared.
 * All calls on a device share the array: each call clears it before use, and calls
 * that overlap on the GPU (other streams or threads) race and give wrong results. */
int eptv_select_kth_noalloc(const float *d_vals, long n, long k, float *d_out, void *stream);

/* ------------------------------------------------------------------ 3-D cone beam
 * The paper is 2-D; this is the same method for a circular cone-beam scan with a flat
 * detector.  Conventions: volume [nz][ny][nx] (x fastest), voxel (ix, iy, iz) covers
 * [x0 + ix dx, x0 + (ix+1) dx] x ... with x0 = -nx dx / 2 (likewise y0, z0); view k at
 * angle theta_k (angles[k], else 2 pi k / n_views), source at sid (cos, sin, 0); flat
 * detector perpendicular to c = -(cos, sin, 0) at distance sdd from the source, pixel
 * (iu, iv) centred at source + sdd c + u e_u + w e_z, e_u = (-sin, cos, 0),
 * u = (iu - (nu-1)/2 + u_off) du, w = (iv - (nv-1)/2 + v_off) dv; projections
 * [n_views][nv][nu] (ray index (k nv + iv) nu + iu).
 * P: p_ij = length of ray i inside voxel j (Eq. 1 in 3-D); P^T its exact transpose.
 * (P2): half-faces (App. II's half-edges extended), magnitude T^2 = eps^2 + D^2 +
 * 1/2 (c+^2 + c-^2) over each transverse direction (A3 extended), weights Eq. (5),
 * variation A2 extended (lagged), GD with Armijo as in 2-D; PRIOR weights are 2-D only.
 * The cone must be narrow enough that no ray crosses z planes faster than x and y planes
 * (EPTV_ERR_ARG otherwise).  All buffers are device FP32, caller-owned. */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;               /* voxel size (mm) */
    int n_views;
    const double *angles;            /* [n_views] radians, or NULL */
    int nu, nv;                      /* detector columns, rows */
    double du, dv;                   /* detector pixel pitch (mm) */
    double u_off, v_off;             /* detector offsets (pixels) */
    double sid, sdd;                 /* source-isocentre, source-detector (mm) */
} eptv3_geometry_desc;

typedef struct eptv3_geometry eptv3_geometry;

/* Builds the ray tables (host FP64, stored FP32: 16 bytes per view and detector column,
 * 8 per detector row, 4 per detector pixel; rays are parametrised by their depth along the
 * central ray, so that P = diag(F) L' with F = |a| per detector pixel) and the solver
 * workspace (about 9 volumes of faces, 6 volumes, 4 projections).  EPTV_ERR_ARG for a bad
 * descriptor: sizes or pitches not positive, sid not above the volume's half-diagonal in
 * x-y or sdd not above sid, 2^31 or more voxels, rays or faces, more than 65535 views or
 * 131070 slices, a cone too wide for the narrow-cone march, or a detector row band of one
 * z slab too tall for the back projector's shared-memory table; EPTV_ERR_NOMEM,
 * EPTV_ERR_CUDA. */
int eptv3_create_geometry(const eptv3_geometry_desc *desc, eptv3_geometry **out);
void eptv3_destroy_geometry(eptv3_geometry *g);
/* Warps per 32-ray block of the 3-D projector (2, 4, 8 or 16). */
int eptv3_set_tuning(eptv3_geometry *g, int seg);
/* Voxels stacked in z per thread of the 3-D back projector (2 or 4; default 4).  The
 * result does not depend on it: every voxel sums the same terms in the same order. */
int eptv3_set_backprojector_stack(eptv3_geometry *g, int zp);
/* d_y [n_rays] = P d_f [n_vox]; d_f = P^T d_y. */
int eptv3_project(const eptv3_geometry *g, const float *d_f, float *d_y, void *stream);
int eptv3_backproject(const eptv3_geometry *g, const float *d_y, float *d_f, void *stream);
/* M CGLS iterations (App. I) from the content of d_u, overwritten with u^(M). */
int eptv3_cgls(const eptv3_geometry *g, int M, const float *d_y, float *d_u, void *stream);
/* One (P2) solve from f = v (sigma from v, n_gd GD iterations with Armijo or fixed steps,
 * then f = max(f, 0)); *t_prev_io (may be NULL) is the previous accepted step, updated.
 * Synchronises `stream`. */
int eptv3_tv_step(const eptv3_geometry *g, const eptv_params *p, const float *d_v, float *d_f,
                  double *t_prev_io, eptv_stats *out_opt, void *stream);
/* p->n_outer outer iterations from the content of d_f (clamped at 0), result in d_f. */
int eptv3_reconstruct(const eptv3_geometry *g, const eptv_params *p, const float *d_y, float *d_f,
                      eptv_report *rep_opt, void *stream);
/* Eq. (2) in 3-D: mu/2 |P f - y|^2 + J(f; w(f; sigma_ref)).  Synchronises `stream`. */
int eptv3_report_energy(const eptv3_geometry *g, const eptv_params *p, double sigma_ref,
                        const float *d_f, const float *d_y, double *h_energy, void *stream);

/* Image-quality metrics of Sec. 3 for an image d_f of g's grid (FP32 [ny][nx]) against a
 * reference d_ref_opt (the ground truth; may be NULL):
 *   rel_error  Eq. (12): |f - f_ref|^2 / |f_ref|^2                           (NaN if no ref)
 *   ecc        Eq. (13): correlation coefficient of the binary edge maps of f and f_ref
 *              (NaN if no ref or if a map is constant); an edge is an interior pixel whose
 *              squared 3x3 Sobel magnitude exceeds edge_scale^2 times its mean over the
 *              interior (the paper names a standard Sobel detector without a threshold;
 *              edge_scale = 2 is the usual choice), evaluated in FP64; border pixels are
 *              never edges
 *   edges, edges_ref, edges_both: the edge counts behind ecc
 *   snr_db     Eq. (14): 10 log10(E(P)^2 / E([P - E(P)]^2)) over the rectangle
 *              h_roi_opt = {x0, y0, w, h} (columns x0 .. x0 + w - 1, rows y0 .. y0 + h - 1)
 *              of d_f; NaN if h_roi_opt is NULL.
 * d_edges_opt / d_edges_ref_opt (may be NULL) receive the byte edge maps [ny][nx].
 * Synchronises `stream`.  Errors: EPTV_ERR_ARG (ROI outside the image, edge_scale <= 0). */
typedef struct {
    double rel_error;
    double ecc;
    long long edges, edges_ref, edges_both;
    double snr_db;
} eptv_quality;

int eptv_quality_metrics(const eptv_geometry *g, const float *d_f, const float *d_ref_opt,
                         const int *h_roi_opt, double edge_scale, unsigned char *d_edges_opt,
                         unsigned char *d_edges_ref_opt, eptv_quality *out, void *stream);

/* Stored-matrix operator (Sec. 2.3: the sparse-matrix strategy for small problems).
 * mode EPTV_OPERATOR_STORED makes every later P / P^T of this handle -- eptv_project(_t),
 * eptv_backproject, eptv_cgls, eptv_reconstruct, eptv_reconstruct_batched (all members
 * of a batch must use the same mode), eptv_report_energy -- a sparse matrix-vector
 * product with device CSR matrices of P (rows = rays v nb + k) and P^T (rows = pixels
 * iy nx + ix).  Their entries are the canonical p_ij that the on-the-fly kernels compute
 * (only p_ij > 0 stored; columns increasing in each row; rows padded with zero entries
 * to multiples of 4), and the two matrices are exact transposes of each other.  The first
 * switch to STORED builds them (synchronous; owned by the handle; about 32 bytes per
 * nonzero of P for both matrices in both forms: CSR for export, SELL-32 for the SpMV);
 * EPTV_OPERATOR_ON_THE_FLY switches back and keeps them.
 * *h_nnz_opt (may be NULL) receives the stored entries of P, padding included.
 * EPTV_OPERATOR_STORED_PT builds the same matrices but applies only P^T from them (P stays
 * on the fly): each operator from whichever form is faster on this hardware for small
 * problems -- the entries are identical, so the pair is still an exact transpose pair.
 * EPTV_OPERATOR_EQ11 keeps P on the fly and makes every P^T the back projector of
 * Eq. (11) (eptv_backproject_eq11); the solver then iterates with an approximate adjoint,
 * as the paper's GPU code did.
 * Errors: EPTV_ERR_ARG (unknown mode; a row of P longer than 4096 entries; 2^31 or more
 * entries), EPTV_ERR_NOMEM, EPTV_ERR_CUDA. */
int eptv_set_operator(eptv_geometry *g, int mode, long long *h_nnz_opt);

/* Chooses the form of P^T for handle g by measurement (the choice Sec. 2.3 leaves to the
 * problem size): when the stored matrices can take at most max_matrix_bytes of device
 * memory (bounded before anything is built by 32 bytes x n_rays x (nx + ny)), it builds
 * them, times P^T from the kernel (at the shape eptv_autotune chose) and from the stored
 * matrix in interleaved rounds of 20 launches on the handle's workspace (overwritten), and
 * keeps the faster: EPTV_OPERATOR_STORED_PT or EPTV_OPERATOR_ON_THE_FLY (whose stored
 * matrices are then freed).  P stays on the fly either way.  *mode_out (may be NULL)
 * receives the choice.  The two forms have identical entries, so results differ only in
 * summation order.  EPTV_ERR_ARG if g is in another operator mode; a matrix that cannot be
 * built (too large, no memory) leaves the handle on the fly; EPTV_ERR_CUDA. */
int eptv_autotune_operator(eptv_geometry *g, long long max_matrix_bytes, int *mode_out);

/* Rows and stored entries (padding included) of the built matrix `which` (0: P, 1: P^T)
 * in the exported CSR form; *h_sell_opt (may be NULL) receives the entries of the SELL-32
 * copy the SpMV kernels stream (rows in slices of 32, each slice padded to its longest
 * row).  EPTV_ERR_ARG if the matrices have not been built. */
int eptv_matrix_info(const eptv_geometry *g, int which, long long *h_rows, long long *h_nnz,
                     long long *h_sell_opt);

/* Copies the built matrix `which` (0: P, 1: P^T) into caller device buffers:
 * d_ptr [rows + 1] int32 row offsets, d_col [nnz] int32 columns, d_val [nnz] FP32 values
 * (sizes from eptv_matrix_info).  Asynchronous on `stream`. */
int eptv_copy_matrix(const eptv_geometry *g, int which, int *d_ptr, int *d_col, float *d_val,
                     void *stream);

/* Batched reconstruction of n independent slices (any mix of sizes) with one set of
 * parameters: every kernel of one outer iteration covers all slices in a single launch,
 * and one outer iteration of the whole batch is captured into one CUDA graph.
 * d_y[i], d_f[i] as in eptv_reconstruct for slice i (handle geoms[i]).  The batch
 * workspace is owned by geoms[0].  reps (host, may be NULL) receives n reports. */
int eptv_reconstruct_batched(int n, eptv_geometry *const *geoms, const eptv_params *p,
                             const float *const *d_y, float *const *d_f,
                             eptv_report *reps, void *stream);

/* Launch shapes of the projector and back projector used by calls on handle g: k1_seg =
 * warps marching each block of 32 adjacent rays (4, 8 or 16; the rows of a ray are split
 * among them), k2_vg = threads sharing the views of each 4 x 2 pixel block (1, 2, 4, 8 or 16).
 * Defaults 8 and 4.  EPTV_ERR_ARG for other values. */
int eptv_set_tuning(eptv_geometry *g, int k1_seg, int k2_vg);

/* (P2) descent kernel used by (P2) solves of handle g (eptv_tv_step, eptv_reconstruct, and
 * batches whose first member is g); Sec. 2.2, Eqs. 5, 9, A2, A3.
 *   EPTV_TV_AUTO (default): when every region of the slices fits on the GPU at once, one
 *     cooperative launch runs the sigma selection (three grid-wide barriers), all n_gd GD
 *     iterations of a (P2) solve (one grid-wide barrier per iteration) and the clamp
 *     (bounded waits: EPTV_ERR_TIMEOUT, reported by the calls that read their scalars, if
 *     one runs out); otherwise, or for more than 8 Armijo trials, three sigma launches
 *     and one launch per GD iteration;
 *   EPTV_TV_PER_ITERATION: always three sigma launches, one launch per GD iteration and
 *     one for the clamp.
 * Both give bit-identical results.  EPTV_ERR_ARG for other values. */
#define EPTV_TV_AUTO           0
#define EPTV_TV_PER_ITERATION  1
int eptv_set_tv_kernel(eptv_geometry *g, int mode);

/* Test hook of the persistent (P2) kernel's bounded waits (no counterpart in the paper):
 * its grid barrier waits for extra_blocks blocks beyond the launch (0: none, the default)
 * and gives up after wait_cycles SM cycles (default 2e9, about one second), after which
 * the kernel stops and the call that reads the scalars returns EPTV_ERR_TIMEOUT; the next
 * call re-arms the barrier.  extra_blocks > 0 makes every wait run out without
 * faulting or hanging the GPU.  EPTV_ERR_ARG outside [0, 1024] x [1e3, 4e9]. */
int eptv_debug_set_p2_wait(eptv_geometry *g, int extra_blocks, long long wait_cycles);

/* Autotuner: times every launch shape of the projector and the back projector on the
 * handle's own geometry (zero images in its workspace, which it overwrites) and keeps
 * the fastest for later calls on g.  *k1_seg / *k2_vg (may be NULL) receive the choice.
 * Synchronises the device. */
int eptv_autotune(eptv_geometry *g, int *k1_seg, int *k2_vg);

/* The same for the batch {geoms[0..n)} used by eptv_reconstruct_batched (the choice is
 * kept with that batch, cached in geoms[0], also when the members change operator mode
 * together). */
int eptv_autotune_batched(int n, eptv_geometry *const *geoms, int *k1_seg, int *k2_vg);

/* ---------------------------------------------------------------------------------
 * Layer kernels of the learned warm-start network (not in the paper: a small U-Net that
 * predicts a warm-start image and a per-pixel edge-weight map from the back projection
 * of the noisy sinogram; plain EPTV finishes the solve, see EPTV_WEIGHTS_PRIOR).
 * Activations are BF16 (uint16 storage) in NHWC layout [n][h][w][stride]; a call reads
 * or writes the channel slice [off, off + c) of such a tensor.  Master weights are FP32.
 * All calls are asynchronous on `stream`, allocate nothing and return EPTV_ERR_ARG for
 * bad shapes before queueing work.
 * --------------------------------------------------------------------------------- */

/* y[.., y_off + o] = act(b[o] + sum_{c, tap} wt[o][tap][c] x[pixel + tap][x_off + c]),
 * 3x3, zero padding, act = ReLU if relu else identity.  BF16 tensor cores (mma.sync
 * m16n8k16, FP32 accumulation).  (cin, cout) in {(16,16), (16,32), (32,32), (32,64),
 * (64,64), (96,32), (48,16), (32,16), (64,32), (32,96), (16,48), (64,96)}; x_stride, x_off
 * multiples of 8; x and wt 16-byte aligned; bias may be NULL.  wt: [cout][9][cin] BF16. */
int eptv_unet_conv3x3(const void *d_x, int n, int h, int w, int cin, int x_stride, int x_off,
                      const void *d_wt, const float *d_bias, int cout, void *d_y, int y_stride,
                      int y_off, int relu, void *stream);

/* Kernel of eptv_unet_conv3x3 (process-wide; not part of the paper):
 *   EPTV_CONV_TENSOR_MEMORY (default): tcgen05.mma with the FP32 accumulator in tensor
 *     memory and TMA-loaded input halos, M = 128 pixels of one tile, N = cout, K = 9 cin,
 *     for the shapes where it is not slower than the mma.sync kernel on B300 (image width
 *     a multiple of 128 with cin >= 32 or cout >= 48); the mma.sync kernel for the others;
 *   EPTV_CONV_MMA_SYNC: always the warp-level mma.sync kernel;
 *   EPTV_CONV_TENSOR_MEMORY_ALL: the tensor-memory kernel wherever it tiles the image
 *     (width a multiple of 128, or 64 with an even height; input channel stride and
 *     offset multiples of 8, input 16-byte aligned).
 * All sum the same BF16 products in FP32 (different order).  EPTV_ERR_ARG otherwise. */
#define EPTV_CONV_TENSOR_MEMORY     0
#define EPTV_CONV_MMA_SYNC          1
#define EPTV_CONV_TENSOR_MEMORY_ALL 2
int eptv_unet_set_conv_kernel(int mode);

/* Synchronises with the device and reports (then clears) the tensor-memory conv's error
 * flag: EPTV_ERR_TIMEOUT if one of its bounded waits for the MMAs ran out since the last
 * call (that launch stopped early and its outputs are incomplete), else EPTV_OK. */
int eptv_unet_tc_status(void);

/* Weight (and bias, if d_db) gradient of eptv_unet_conv3x3, accumulated into FP32 buffers:
 * dw[o][tap][c] += sum_p dy[p][o] x[p + tap][c], db[o] += sum_p dy[p][o].  Same channel
 * pairs as eptv_unet_conv3x3; strides and offsets of x and dy multiples of 8 channels,
 * d_x and d_dy 16-byte aligned.  Sums are FP32 and their order is not fixed (atomic adds). */
int eptv_unet_conv3x3_wgrad(const void *d_x, int n, int h, int w, int cin, int x_stride, int x_off,
                            const void *d_dy, int dy_stride, int dy_off, int cout, float *d_dw,
                            float *d_db, void *stream);

/* FP32 master weights [cout][9][cin] -> BF16 forward weights (d_wf, [cout][9][cin]) and the
 * BF16 weights of the data gradient (d_wb, [cin][9][cout], taps mirrored), either may be
 * NULL.  The data gradient of a conv is eptv_unet_conv3x3 with d_wb and cin/cout swapped. */
int eptv_unet_weights_to_bf16(const float *d_w, int cout, int cin, void *d_wf, void *d_wb,
                              void *stream);

/* 2x2 max pooling (h, w even) and its gradient (to the first maximum of each window in
 * row-major order; accumulate != 0 adds to d_dx instead of overwriting). */
int eptv_unet_maxpool2(const void *d_x, int n, int h, int w, int x_stride, int x_off, int c,
                       void *d_y, int y_stride, int y_off, void *stream);
int eptv_unet_maxpool2_bwd(const void *d_x, int n, int h, int w, int x_stride, int x_off, int c,
                           const void *d_dy, int dy_stride, int dy_off, void *d_dx, int dx_stride,
                           int dx_off, int accumulate, void *stream);

/* Nearest-neighbour 2x upsampling of an h x w input, and its gradient (h, w: the size of
 * the upsampled gradient, even; each input pixel receives the sum of its 4 copies). */
int eptv_unet_upsample2(const void *d_x, int n, int h, int w, int x_stride, int x_off, int c,
                        void *d_y, int y_stride, int y_off, void *stream);
int eptv_unet_upsample2_bwd(const void *d_dy, int n, int h, int w, int dy_stride, int dy_off, int c,
                            void *d_dx, int dx_stride, int dx_off, void *stream);

/* ReLU gradient: dz = dy where the ReLU output a > 0, else 0 (in place allowed). */
int eptv_unet_relu_bwd(const void *d_a, int a_stride, int a_off, const void *d_dy, int dy_stride,
                       int dy_off, void *d_dz, int dz_stride, int dz_off, long long npix, int c,
                       void *stream);

/* 1x1 head (16 -> 2 channels): o = hb + hw x; w = sigmoid(o1); f0 = o0, or, with d_base,
 * f0 = max(base + f_scale o0, 0) (a warm-start image composed on a base image).  Outputs are
 * FP32 [npix]; d_f0, d_w may be NULL.  x: BF16, channels [x_off, x_off + 16) of rows of
 * x_stride channels.  Training mode (d_ft != NULL, f0 = o0 in network units):
 * *d_loss += mean((o0-ft)^2) + mean((w-wt)^2) over the npix pixels, d_dx (BF16, 16 channels
 * at dx_off) = dL/dx, d_dhw [2][16], d_dhb [2] += parameter gradients. */
int eptv_unet_head(const void *d_x, int x_stride, int x_off, long long npix, const float *d_hw,
                   const float *d_hb, float *d_f0, float *d_w, const float *d_base, float f_scale,
                   const float *d_ft, const float *d_wt, void *d_dx, int dx_stride, int dx_off,
                   float *d_dhw, float *d_dhb, double *d_loss, void *stream);

/* Network input rows: x[p][0] = a[p] scale_a, x[p][1] = b[p] scale_b (0 if d_b is NULL),
 * x[p][2..15] = 0, rounded to BF16; d_x: BF16 [npix][16], 16-byte aligned. */
int eptv_unet_pack_input(const float *d_a, float scale_a, const float *d_b, float scale_b,
                         long long npix, void *d_x, void *stream);

/* Adam step (bias-corrected with step >= 1) on n FP32 parameters. */
int eptv_unet_adam(float *d_p, const float *d_g, float *d_m, float *d_v, long long n, float lr,
                   float beta1, float beta2, float eps, int step, void *stream);

/* Message of the last failed call on this thread ("" if none). */
const char *eptv_last_error(void);

/* Library version string. */
const char *eptv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EPTV_H */
