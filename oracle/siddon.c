/*
 * FP64 CPU oracle: Siddon ray tracing for the fan-beam system matrix P (Eq. 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This file shares no code, header or constant with the
 * CUDA path; only the test suite, the smoke check and the benchmark's CPU baseline
 * load it.
 *
 * p_ij is the length of the intersection of ray i with pixel j (Sec. 2.1), computed by
 * Siddon's method: the ray's parametric crossings with the x grid lines and with the y
 * grid lines form two monotone lists; merging them gives consecutive crossings, and
 * each pair bounds one segment whose pixel is found from its midpoint.
 *
 * P^T is the exact transpose: the same traversal scatters p_ij * y_i into pixel j
 * (the ray-driven back projection of Sec. 2.3 -- slow, but exact by construction).
 *
 * Ray i: source point (sx, sy), unit direction (ux, uy); only t >= 0 (in front of the
 * source) counts.  Image: nx x ny pixels of dx x dy mm, row-major [ny][nx], centred
 * on the origin, so pixel (i, j) covers [x0 + i dx, x0 + (i+1) dx] x [y0 + j dy, ...]
 * with x0 = -nx dx / 2, y0 = -ny dy / 2.  A ray with ux == 0 has no x crossings
 * (likewise uy == 0).
 */
#include <math.h>
#include <stdlib.h>

/* Crossing parameters t of one family of grid lines, ascending, restricted to the open
 * interval (tlo, thi).  Returns the number written. */
static int crossings(double s, double u, double origin, double pitch, int n,
                     double tlo, double thi, double *out)
{
    int m = 0;
    if (u == 0.0) return 0;
    if (u > 0.0) {
        for (int k = 0; k <= n; ++k) {
            double t = (origin + k * pitch - s) / u;
            if (t > tlo && t < thi) out[m++] = t;
        }
    } else {
        for (int k = n; k >= 0; --k) {
            double t = (origin + k * pitch - s) / u;
            if (t > tlo && t < thi) out[m++] = t;
        }
    }
    return m;
}

/* Entry/exit parameters of the ray in the slab origin <= s + t u <= origin + n pitch. */
static int slab(double s, double u, double origin, double pitch, int n,
                double *tmin, double *tmax)
{
    double lo = origin, hi = origin + n * pitch;
    if (u == 0.0) {
        if (s > lo && s < hi) { *tmin = -INFINITY; *tmax = INFINITY; return 1; }
        return 0;
    }
    double a = (lo - s) / u, b = (hi - s) / u;
    *tmin = a < b ? a : b;
    *tmax = a < b ? b : a;
    return 1;
}

/* Trace one ray; writes (pixel index, length) pairs, returns their count. */
static int trace(int nx, int ny, double dx, double dy,
                 double sx, double sy, double ux, double uy,
                 double *ta, double *tb, double *tm, long *pix, double *len)
{
    double x0 = -0.5 * nx * dx, y0 = -0.5 * ny * dy;
    double txmin, txmax, tymin, tymax;
    if (!slab(sx, ux, x0, dx, nx, &txmin, &txmax)) return 0;
    if (!slab(sy, uy, y0, dy, ny, &tymin, &tymax)) return 0;
    double tmin = txmin > tymin ? txmin : tymin;
    double tmax = txmax < tymax ? txmax : tymax;
    if (tmin < 0.0) tmin = 0.0;
    if (!(tmin < tmax)) return 0;

    int na = crossings(sx, ux, x0, dx, nx, tmin, tmax, ta);
    int nb = crossings(sy, uy, y0, dy, ny, tmin, tmax, tb);

    /* merge tmin, the two ascending lists, tmax */
    int m = 0, ia = 0, ib = 0;
    tm[m++] = tmin;
    while (ia < na || ib < nb) {
        if (ib >= nb || (ia < na && ta[ia] <= tb[ib])) tm[m++] = ta[ia++];
        else tm[m++] = tb[ib++];
    }
    tm[m++] = tmax;

    int cnt = 0;
    for (int k = 0; k + 1 < m; ++k) {
        double l = tm[k + 1] - tm[k];
        if (!(l > 0.0)) continue;
        double mid = 0.5 * (tm[k] + tm[k + 1]);
        long i = (long)floor((sx + mid * ux - x0) / dx);
        long j = (long)floor((sy + mid * uy - y0) / dy);
        if (i < 0) i = 0;
        if (i >= nx) i = nx - 1;
        if (j < 0) j = 0;
        if (j >= ny) j = ny - 1;
        pix[cnt] = j * nx + i;
        len[cnt] = l;
        ++cnt;
    }
    return cnt;
}

typedef struct { double *ta, *tb, *tm, *len; long *pix; } scratch_t;

static int scratch_alloc(scratch_t *s, int nx, int ny)
{
    int n = nx + ny + 4;
    s->ta = malloc(sizeof(double) * (nx + 1));
    s->tb = malloc(sizeof(double) * (ny + 1));
    s->tm = malloc(sizeof(double) * n);
    s->len = malloc(sizeof(double) * n);
    s->pix = malloc(sizeof(long) * n);
    return s->ta && s->tb && s->tm && s->len && s->pix;
}

static void scratch_free(scratch_t *s)
{
    free(s->ta); free(s->tb); free(s->tm); free(s->len); free(s->pix);
}

/* y = P f  (y overwritten) */
int og_project(int nx, int ny, double dx, double dy, long n_rays,
               const double *sx, const double *sy, const double *ux, const double *uy,
               const double *f, double *y)
{
    scratch_t s;
    if (!scratch_alloc(&s, nx, ny)) { scratch_free(&s); return -1; }
    for (long r = 0; r < n_rays; ++r) {
        int c = trace(nx, ny, dx, dy, sx[r], sy[r], ux[r], uy[r], s.ta, s.tb, s.tm, s.pix, s.len);
        double acc = 0.0;
        for (int k = 0; k < c; ++k) acc += s.len[k] * f[s.pix[k]];
        y[r] = acc;
    }
    scratch_free(&s);
    return 0;
}

/* f = P^T y  (f overwritten) */
int og_backproject(int nx, int ny, double dx, double dy, long n_rays,
                   const double *sx, const double *sy, const double *ux, const double *uy,
                   const double *y, double *f)
{
    scratch_t s;
    if (!scratch_alloc(&s, nx, ny)) { scratch_free(&s); return -1; }
    for (long p = 0; p < (long)nx * ny; ++p) f[p] = 0.0;
    for (long r = 0; r < n_rays; ++r) {
        int c = trace(nx, ny, dx, dy, sx[r], sy[r], ux[r], uy[r], s.ta, s.tb, s.tm, s.pix, s.len);
        for (int k = 0; k < c; ++k) f[s.pix[k]] += s.len[k] * y[r];
    }
    scratch_free(&s);
    return 0;
}

/* Sparse listing of ray r's row of P: returns the count, fills pix/len (capacity nx+ny+4). */
int og_ray_row(int nx, int ny, double dx, double dy,
               double sx, double sy, double ux, double uy, long *pix, double *len)
{
    scratch_t s;
    if (!scratch_alloc(&s, nx, ny)) { scratch_free(&s); return -1; }
    int c = trace(nx, ny, dx, dy, sx, sy, ux, uy, s.ta, s.tb, s.tm, s.pix, s.len);
    for (int k = 0; k < c; ++k) { pix[k] = s.pix[k]; len[k] = s.len[k]; }
    scratch_free(&s);
    return c;
}
