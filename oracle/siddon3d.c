/*
 * FP64 CPU oracle: Siddon ray tracing through a voxel volume (3-D cone-beam system
 * matrix, the 3-D extension of Eq. 1: p_ij = length of ray i inside voxel j).
 *
 * TEST INFRASTRUCTURE ONLY.  This file shares no code, header or constant with the
 * CUDA path; only the test suite and the benchmark's CPU baseline load it.
 *
 * Siddon's method in three dimensions: the ray's parametric crossings with the x, y and
 * z grid planes inside the volume, together with its entry and exit, are pooled and
 * sorted; each pair of consecutive crossings bounds one segment, whose voxel is the one
 * containing the segment's midpoint.  P^T is the exact transpose: the same traversal
 * scatters p_ij * y_i into voxel j.
 *
 * Ray i: source point s, unit direction u; only t >= 0 counts.  Volume: nx x ny x nz
 * voxels of dx x dy x dz mm, [nz][ny][nx], centred on the origin: voxel (ix, iy, iz)
 * covers [x0 + ix dx, x0 + (ix+1) dx] x ... with x0 = -nx dx / 2 (likewise y0, z0).
 */
#include <math.h>
#include <stdlib.h>

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Entry / exit of the ray in one slab; 0 if the ray misses it (parallel and outside). */
static int slab3(double s, double u, double lo, double hi, double *tmin, double *tmax)
{
    if (u == 0.0) {
        if (s > lo && s < hi) { *tmin = -INFINITY; *tmax = INFINITY; return 1; }
        return 0;
    }
    double a = (lo - s) / u, b = (hi - s) / u;
    *tmin = a < b ? a : b;
    *tmax = a < b ? b : a;
    return 1;
}

/* Crossings of one family of planes strictly inside (tlo, thi), appended to out. */
static int planes(double s, double u, double origin, double pitch, int n, double tlo, double thi,
                  double *out)
{
    int m = 0;
    if (u == 0.0) return 0;
    for (int k = 0; k <= n; ++k) {
        double t = (origin + k * pitch - s) / u;
        if (t > tlo && t < thi) out[m++] = t;
    }
    return m;
}

/* Segments of one ray: voxel indices and lengths; returns the count (buffers hold at
 * least nx + ny + nz + 4 entries). */
static int trace3(int nx, int ny, int nz, double dx, double dy, double dz, double sx, double sy,
                  double sz, double ux, double uy, double uz, double *tb, long *vox, double *len)
{
    const double x0 = -0.5 * nx * dx, y0 = -0.5 * ny * dy, z0 = -0.5 * nz * dz;
    double a0, a1, b0, b1, c0, c1;
    if (!slab3(sx, ux, x0, x0 + nx * dx, &a0, &a1)) return 0;
    if (!slab3(sy, uy, y0, y0 + ny * dy, &b0, &b1)) return 0;
    if (!slab3(sz, uz, z0, z0 + nz * dz, &c0, &c1)) return 0;
    double tmin = fmax(fmax(fmax(a0, b0), c0), 0.0);
    double tmax = fmin(fmin(a1, b1), c1);
    if (!(tmax > tmin)) return 0;
    int m = 0;
    tb[m++] = tmin;
    m += planes(sx, ux, x0, dx, nx, tmin, tmax, tb + m);
    m += planes(sy, uy, y0, dy, ny, tmin, tmax, tb + m);
    m += planes(sz, uz, z0, dz, nz, tmin, tmax, tb + m);
    tb[m++] = tmax;
    qsort(tb, (size_t)m, sizeof(double), cmp_double);
    int c = 0;
    for (int k = 0; k + 1 < m; ++k) {
        double l = tb[k + 1] - tb[k];
        if (!(l > 0.0)) continue;
        double tm = 0.5 * (tb[k] + tb[k + 1]);
        int ix = (int)floor((sx + tm * ux - x0) / dx);
        int iy = (int)floor((sy + tm * uy - y0) / dy);
        int iz = (int)floor((sz + tm * uz - z0) / dz);
        if (ix < 0) ix = 0;
        if (ix >= nx) ix = nx - 1;
        if (iy < 0) iy = 0;
        if (iy >= ny) iy = ny - 1;
        if (iz < 0) iz = 0;
        if (iz >= nz) iz = nz - 1;
        vox[c] = ((long)iz * ny + iy) * nx + ix;
        len[c] = l;
        ++c;
    }
    return c;
}

typedef struct { double *tb; long *vox; double *len; } scratch3_t;

static int scratch3_alloc(scratch3_t *s, int nx, int ny, int nz)
{
    size_t cap = (size_t)nx + ny + nz + 8;
    s->tb = (double *)malloc(cap * sizeof(double));
    s->vox = (long *)malloc(cap * sizeof(long));
    s->len = (double *)malloc(cap * sizeof(double));
    return s->tb && s->vox && s->len;
}

static void scratch3_free(scratch3_t *s)
{
    free(s->tb);
    free(s->vox);
    free(s->len);
}

/* y_i = sum_j p_ij f_j for n rays. */
int og3_project(int nx, int ny, int nz, double dx, double dy, double dz, long n, const double *sx,
                const double *sy, const double *sz, const double *ux, const double *uy, const double *uz,
                const double *f, double *y)
{
    scratch3_t s;
    if (!scratch3_alloc(&s, nx, ny, nz)) { scratch3_free(&s); return -1; }
    for (long i = 0; i < n; ++i) {
        int c = trace3(nx, ny, nz, dx, dy, dz, sx[i], sy[i], sz[i], ux[i], uy[i], uz[i], s.tb, s.vox, s.len);
        double acc = 0.0;
        for (int k = 0; k < c; ++k) acc += s.len[k] * f[s.vox[k]];
        y[i] = acc;
    }
    scratch3_free(&s);
    return 0;
}

/* f_j = sum_i p_ij y_i (exact transpose, ray-driven scatter). */
int og3_backproject(int nx, int ny, int nz, double dx, double dy, double dz, long n, const double *sx,
                    const double *sy, const double *sz, const double *ux, const double *uy,
                    const double *uz, const double *y, double *f)
{
    scratch3_t s;
    if (!scratch3_alloc(&s, nx, ny, nz)) { scratch3_free(&s); return -1; }
    for (long j = 0; j < (long)nx * ny * nz; ++j) f[j] = 0.0;
    for (long i = 0; i < n; ++i) {
        int c = trace3(nx, ny, nz, dx, dy, dz, sx[i], sy[i], sz[i], ux[i], uy[i], uz[i], s.tb, s.vox, s.len);
        for (int k = 0; k < c; ++k) f[s.vox[k]] += s.len[k] * y[i];
    }
    scratch3_free(&s);
    return 0;
}

/* Nonzeros of one ray's row of P; returns the count or -1. */
int og3_ray_row(int nx, int ny, int nz, double dx, double dy, double dz, double sx, double sy,
                double sz, double ux, double uy, double uz, long *vox, double *len)
{
    scratch3_t s;
    if (!scratch3_alloc(&s, nx, ny, nz)) { scratch3_free(&s); return -1; }
    int c = trace3(nx, ny, nz, dx, dy, dz, sx, sy, sz, ux, uy, uz, s.tb, s.vox, s.len);
    for (int k = 0; k < c; ++k) { vox[k] = s.vox[k]; len[k] = s.len[k]; }
    scratch3_free(&s);
    return c;
}
