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
