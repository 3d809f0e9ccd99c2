/*
 * FP64 oracle for the Joseph projector K and its transpose K^T (parallel beam, and
 * per ray for the fan beam).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this file.  It shares no code with the
 * CUDA library.
 *
 * Geometry (the paper's Radon transform, Sec. 2, eq. (radon-def)): a ray is
 * the line u cos(theta) + v sin(theta) = s.  Pixel (row j, column i) of an
 * N x N image sits at u = i - (N-1)/2, v = (N-1)/2 - j (pixel units).
 * Bin t of angle a has s_t = (t - (n_det-1)/2)*spacing + offset.
 *
 * K (Joseph's method; the paper itself used MATLAB's radon): when the ray is
 * closer to vertical (|cos| >= |sin|, flagged by row_branch[a]) it is stepped
 * over image rows v_j: at each row the ray crosses u = (s - v_j sin)/cos, the
 * image is interpolated linearly between the two neighbouring columns, and the
 * sum is scaled by the path length per row, 1/|cos|.  Otherwise it is stepped
 * over columns u_i with v = (s - u_i cos)/sin, interpolated between the two
 * neighbouring rows and scaled by 1/|sin|.  Pixels outside the image are zero.
 *
 * K^T is written as the literal transpose: the same ray loops, scattering
 * instead of gathering.  Row-branch rays are processed per image row and
 * column-branch rays per image column, so OpenMP threads never share a pixel.
 */
#include <math.h>
#include <string.h>

static double pix(const double* x, int N, int j, int i)
{
    if (j < 0 || j >= N || i < 0 || i >= N) return 0.0;
    return x[(long)j * N + i];
}

static void add_pix(double* x, int N, int j, int i, double val)
{
    if (j < 0 || j >= N || i < 0 || i >= N) return;
    x[(long)j * N + i] += val;
}

/* Position of ray (a, t) on image row j, as a fractional column index. */
static double row_cross(int N, double c, double s, double st, int j)
{
    double cN = 0.5 * (N - 1);
    double v = cN - j;
    double u = (st - v * s) / c;
    return u + cN;
}

/* Position of ray (a, t) on image column i, as a fractional row index. */
static double col_cross(int N, double c, double s, double st, int i)
{
    double cN = 0.5 * (N - 1);
    double u = i - cN;
    double v = (st - u * c) / s;
    return cN - v;
}

/* Below this many (line, ray) steps a call runs on one thread: the thread start-up
 * would cost more than the work.  Each output entry is summed by one thread in the
 * same order either way, so the results do not depend on the thread count. */
#define OMP_MIN_WORK 2000000L

void oracle_joseph_forward(int N, int n_ang, int n_det,
                           const double* cos_t, const double* sin_t, const int* row_branch,
                           double spacing, double offset,
                           const double* x, double* y)
{
    double cd = 0.5 * (n_det - 1);
#pragma omp parallel for schedule(dynamic) if ((long)N * n_ang * n_det > OMP_MIN_WORK)
    for (int a = 0; a < n_ang; ++a) {
        double c = cos_t[a], s = sin_t[a];
        for (int t = 0; t < n_det; ++t) {
            double st = (t - cd) * spacing + offset;
            double acc = 0.0;
            if (row_branch[a]) {
                for (int j = 0; j < N; ++j) {
                    double fi = row_cross(N, c, s, st, j);
                    double f0 = floor(fi);
                    int i0 = (int)f0;
                    double w = fi - f0;
                    acc += (1.0 - w) * pix(x, N, j, i0) + w * pix(x, N, j, i0 + 1);
                }
                acc /= fabs(c);
            } else {
                for (int i = 0; i < N; ++i) {
                    double fj = col_cross(N, c, s, st, i);
                    double f0 = floor(fj);
                    int j0 = (int)f0;
                    double w = fj - f0;
                    acc += (1.0 - w) * pix(x, N, j0, i) + w * pix(x, N, j0 + 1, i);
                }
                acc /= fabs(s);
            }
            y[(long)a * n_det + t] = acc;
        }
    }
}

void oracle_joseph_transpose(int N, int n_ang, int n_det,
                             const double* cos_t, const double* sin_t, const int* row_branch,
                             double spacing, double offset,
                             const double* y, double* x)
{
    double cd = 0.5 * (n_det - 1);
    memset(x, 0, sizeof(double) * (size_t)N * N);
    /* rays stepped over rows: each thread owns one image row */
#pragma omp parallel for schedule(static) if ((long)N * n_ang * n_det > OMP_MIN_WORK)
    for (int j = 0; j < N; ++j) {
        for (int a = 0; a < n_ang; ++a) {
            if (!row_branch[a]) continue;
            double c = cos_t[a], s = sin_t[a];
            for (int t = 0; t < n_det; ++t) {
                double st = (t - cd) * spacing + offset;
                double val = y[(long)a * n_det + t] / fabs(c);
                double fi = row_cross(N, c, s, st, j);
                double f0 = floor(fi);
                int i0 = (int)f0;
                double w = fi - f0;
                add_pix(x, N, j, i0, (1.0 - w) * val);
                add_pix(x, N, j, i0 + 1, w * val);
            }
        }
    }
    /* rays stepped over columns: each thread owns one image column */
#pragma omp parallel for schedule(static) if ((long)N * n_ang * n_det > OMP_MIN_WORK)
    for (int i = 0; i < N; ++i) {
        for (int a = 0; a < n_ang; ++a) {
            if (row_branch[a]) continue;
            double c = cos_t[a], s = sin_t[a];
            for (int t = 0; t < n_det; ++t) {
                double st = (t - cd) * spacing + offset;
                double val = y[(long)a * n_det + t] / fabs(s);
                double fj = col_cross(N, c, s, st, i);
                double f0 = floor(fj);
                int j0 = (int)f0;
                double w = fj - f0;
                add_pix(x, N, j0, i, (1.0 - w) * val);
                add_pix(x, N, j0 + 1, i, w * val);
            }
        }
    }
}

/*
 * Per-ray form of the same projector, for geometries whose rays do not come in
 * parallel families (the fan beam of the Sec. 4 "fan beam and cone beam geometry"
 * remark).  Ray r is the line u cos_r[r] + v sin_r[r] = s_r[r], stepped over rows
 * when row_branch[r] is 1 and over columns otherwise, with exactly the crossing,
 * interpolation and path-length weight of the functions above.
 */
void oracle_joseph_forward_rays(int N, long n_rays, const double* cos_r, const double* sin_r,
                                const double* s_r, const int* row_branch, const double* x, double* y)
{
#pragma omp parallel for schedule(dynamic, 64) if ((long)N * n_rays > OMP_MIN_WORK)
    for (long r = 0; r < n_rays; ++r) {
        double c = cos_r[r], s = sin_r[r], st = s_r[r];
        double acc = 0.0;
        if (row_branch[r]) {
            for (int j = 0; j < N; ++j) {
                double fi = row_cross(N, c, s, st, j);
                double f0 = floor(fi);
                int i0 = (int)f0;
                double w = fi - f0;
                acc += (1.0 - w) * pix(x, N, j, i0) + w * pix(x, N, j, i0 + 1);
            }
            acc /= fabs(c);
        } else {
            for (int i = 0; i < N; ++i) {
                double fj = col_cross(N, c, s, st, i);
                double f0 = floor(fj);
                int j0 = (int)f0;
                double w = fj - f0;
                acc += (1.0 - w) * pix(x, N, j0, i) + w * pix(x, N, j0 + 1, i);
            }
            acc /= fabs(s);
        }
        y[r] = acc;
    }
}

void oracle_joseph_transpose_rays(int N, long n_rays, const double* cos_r, const double* sin_r,
                                  const double* s_r, const int* row_branch, const double* y, double* x)
{
    memset(x, 0, sizeof(double) * (size_t)N * N);
#pragma omp parallel for schedule(static) if ((long)N * n_rays > OMP_MIN_WORK)
    for (int j = 0; j < N; ++j) {
        for (long r = 0; r < n_rays; ++r) {
            if (!row_branch[r]) continue;
            double c = cos_r[r];
            double val = y[r] / fabs(c);
            double fi = row_cross(N, c, sin_r[r], s_r[r], j);
            double f0 = floor(fi);
            int i0 = (int)f0;
            double w = fi - f0;
            add_pix(x, N, j, i0, (1.0 - w) * val);
            add_pix(x, N, j, i0 + 1, w * val);
        }
    }
#pragma omp parallel for schedule(static) if ((long)N * n_rays > OMP_MIN_WORK)
    for (int i = 0; i < N; ++i) {
        for (long r = 0; r < n_rays; ++r) {
            if (row_branch[r]) continue;
            double s = sin_r[r];
            double val = y[r] / fabs(s);
            double fj = col_cross(N, cos_r[r], s, s_r[r], i);
            double f0 = floor(fj);
            int j0 = (int)f0;
            double w = fj - f0;
            add_pix(x, N, j0, i, (1.0 - w) * val);
            add_pix(x, N, j0 + 1, i, w * val);
        }
    }
}

/*
 * Cone beam on a circular orbit (Sec. 4, "fan beam and cone beam geometry": the 3-D
 * divergent-beam transform).  Volume x[k][j][i], Nz slices of N x N, voxel centre
 * (u, v, w) = (i - cN, cN - j, k - cZ).  Ray r is given by its in-plane line
 * u cos_r + v sin_r = s_r (a fan-beam ray), its source (su_r, sv_r) in the plane w = 0, and
 * its slope sig_r: along the in-plane direction d = (sin_r, -cos_r), which points from the
 * source into the volume, the ray rises by sig_r per unit of in-plane distance.  It is stepped
 * over the in-plane lines like the in-plane ray (rows when row_branch, else columns).  On each
 * line the in-plane crossing gives the fractional index along the other in-plane axis, and the
 * in-plane distance h = (P - S) . d of the crossing point P gives the fractional slice index
 * sig_r h + cZ; the volume is interpolated bilinearly in those two indices and the sum is
 * scaled by the path length per step, sqrt(1 + sig_r^2) / |cos| (or / |sin|).  Voxels outside
 * the volume are zero.  The transpose is the literal scatter, threads owning one row (row
 * branch) or one column (column branch) of every slice.
 */
static double vox(const double* x, int N, int Nz, int k, int j, int i)
{
    if (k < 0 || k >= Nz || j < 0 || j >= N || i < 0 || i >= N) return 0.0;
    return x[((long)k * N + j) * N + i];
}

static void add_vox(double* x, int N, int Nz, int k, int j, int i, double val)
{
    if (k < 0 || k >= Nz || j < 0 || j >= N || i < 0 || i >= N) return;
    x[((long)k * N + j) * N + i] += val;
}

/* Crossing of cone ray r with in-plane line q: index f along the interpolation axis, slice
 * index g. */
static void cone_cross(int N, int Nz, int row, double c, double s, double st, double su, double sv,
                       double sg, int q, double* f, double* g)
{
    double cN = 0.5 * (N - 1), cZ = 0.5 * (Nz - 1), u, v;
    if (row) {
        v = cN - q;
        u = (st - v * s) / c;
        *f = u + cN;
    } else {
        u = q - cN;
        v = (st - u * c) / s;
        *f = cN - v;
    }
    *g = sg * ((u - su) * s - (v - sv) * c) + cZ;
}

void oracle_cone_forward(int N, int Nz, long n_rays, const double* cos_r, const double* sin_r, const double* s_r,
                         const double* su_r, const double* sv_r, const double* sig_r, const int* row_branch,
                         const double* x, double* y)
{
#pragma omp parallel for schedule(dynamic, 64) if ((long)N * n_rays > OMP_MIN_WORK)
    for (long r = 0; r < n_rays; ++r) {
        double c = cos_r[r], s = sin_r[r], acc = 0.0;
        int row = row_branch[r];
        for (int q = 0; q < N; ++q) {
            double f, g;
            cone_cross(N, Nz, row, c, s, s_r[r], su_r[r], sv_r[r], sig_r[r], q, &f, &g);
            double f0 = floor(f), g0 = floor(g);
            int p0 = (int)f0, k0 = (int)g0;
            double w = f - f0, wz = g - g0;
            double a0, a1;
            if (row) {
                a0 = (1.0 - w) * vox(x, N, Nz, k0, q, p0) + w * vox(x, N, Nz, k0, q, p0 + 1);
                a1 = (1.0 - w) * vox(x, N, Nz, k0 + 1, q, p0) + w * vox(x, N, Nz, k0 + 1, q, p0 + 1);
            } else {
                a0 = (1.0 - w) * vox(x, N, Nz, k0, p0, q) + w * vox(x, N, Nz, k0, p0 + 1, q);
                a1 = (1.0 - w) * vox(x, N, Nz, k0 + 1, p0, q) + w * vox(x, N, Nz, k0 + 1, p0 + 1, q);
            }
            acc += (1.0 - wz) * a0 + wz * a1;
        }
        y[r] = acc * sqrt(1.0 + sig_r[r] * sig_r[r]) / fabs(row ? c : s);
    }
}

void oracle_cone_transpose(int N, int Nz, long n_rays, const double* cos_r, const double* sin_r, const double* s_r,
                           const double* su_r, const double* sv_r, const double* sig_r, const int* row_branch,
                           const double* y, double* x)
{
    memset(x, 0, sizeof(double) * (size_t)N * N * Nz);
    for (int pass = 1; pass >= 0; --pass) {        /* rays stepped over rows, then over columns */
#pragma omp parallel for schedule(static) if ((long)N * n_rays > OMP_MIN_WORK)
        for (int q = 0; q < N; ++q) {
            for (long r = 0; r < n_rays; ++r) {
                if (row_branch[r] != pass) continue;
                double c = cos_r[r], s = sin_r[r];
                double val = y[r] * sqrt(1.0 + sig_r[r] * sig_r[r]) / fabs(pass ? c : s);
                double f, g;
                cone_cross(N, Nz, pass, c, s, s_r[r], su_r[r], sv_r[r], sig_r[r], q, &f, &g);
                double f0 = floor(f), g0 = floor(g);
                int p0 = (int)f0, k0 = (int)g0;
                double w = f - f0, wz = g - g0;
                double v00 = (1.0 - wz) * (1.0 - w) * val, v01 = (1.0 - wz) * w * val;
                double v10 = wz * (1.0 - w) * val, v11 = wz * w * val;
                if (pass) {
                    add_vox(x, N, Nz, k0, q, p0, v00);
                    add_vox(x, N, Nz, k0, q, p0 + 1, v01);
                    add_vox(x, N, Nz, k0 + 1, q, p0, v10);
                    add_vox(x, N, Nz, k0 + 1, q, p0 + 1, v11);
                } else {
                    add_vox(x, N, Nz, k0, p0, q, v00);
                    add_vox(x, N, Nz, k0, p0 + 1, q, v01);
                    add_vox(x, N, Nz, k0 + 1, p0, q, v10);
                    add_vox(x, N, Nz, k0 + 1, p0 + 1, q, v11);
                }
            }
        }
    }
}
