/*
 * FP64 CPU oracle kernels for the semi-Lagrangian (SL) transport path of
 * "CLAIRE at scale" (arXiv 2209.08189).  TEST INFRASTRUCTURE ONLY: nothing
 * in the product path may call, link or load this file.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Everything here is the plain definition written out as loops, in double
 * precision, with no blocking or fusion:
 *
 *   - interpolation of a periodic grid function at off-grid points
 *     (Sec. 3: "IP kernel", linear and cubic Lagrange), written as the
 *     tensor product of 1-D Lagrange cardinal polynomials;
 *   - the exact transpose (scatter) of that interpolation, used for the
 *     discretise-then-optimise (DTO) adjoint pins;
 *   - the second-order Runge-Kutta (Heun) backtrace of characteristic
 *     points for a stationary velocity (Sec. 2.2 "Discretization");
 *   - 8th-order central finite differences for the gradient and the
 *     divergence (Sec. 2.2 / Sec. 3 "FD kernel").
 *
 * Conventions: grid n[0] x n[1] x n[2] on [0, 2*pi)^3, C order (x3 fastest),
 * spacing h_c = 2*pi / n_c.  A vector field is stored component-major
 * [3][n0][n1][n2].  Displacements are in grid units: the off-grid point of
 * grid node (i,j,k) is (i + d0, j + d1, k + d2).
 */
#include <math.h>
#include <stddef.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TWO_PI 6.283185307179586476925286766559

static long orc_wrap(long i, long n)
{
    long r = i % n;
    return r < 0 ? r + n : r;
}

/*
 * 1-D basis at fractional offset t in [0,1) from the cell's left node.
 * order 3: cubic Lagrange cardinal functions on the four nodes -1,0,1,2
 *          (l_a(t) = prod_{b != a} (t - s_b) / (s_a - s_b)).
 * order 4: the uniform cubic B-spline beta(x) (x = t - s_a), beta(x) =
 *          (4 - 6x^2 + 3|x|^3)/6 for |x| <= 1, (2 - |x|)^3/6 for 1 < |x| < 2,
 *          on the same four nodes (applied to prefiltered coefficients).
 * order 1: linear hat functions on nodes 0,1.
 * Returns the number of nodes and fills node offsets and weights.
 */
static double orc_bspline(double x)
{
    double a = fabs(x);
    if (a <= 1.0) return (4.0 - 6.0 * a * a + 3.0 * a * a * a) / 6.0;
    if (a < 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
    return 0.0;
}

/* derivative of beta */
static double orc_bspline_d(double x)
{
    double a = fabs(x), sg = x < 0 ? -1.0 : 1.0;
    if (a <= 1.0) return sg * (-12.0 * a + 9.0 * a * a) / 6.0;
    if (a < 2.0) return -sg * (2.0 - a) * (2.0 - a) / 2.0;
    return 0.0;
}

static int orc_basis(int order, double t, long off[4], double w[4])
{
    if (order == 4) {
        for (int a = 0; a < 4; ++a) {
            off[a] = a - 1;
            w[a] = orc_bspline(t - (double)(a - 1));
        }
        return 4;
    }
    if (order == 3) {
        const double s[4] = {-1.0, 0.0, 1.0, 2.0};
        for (int a = 0; a < 4; ++a) {
            double num = 1.0, den = 1.0;
            for (int b = 0; b < 4; ++b) {
                if (b == a) continue;
                num *= (t - s[b]);
                den *= (s[a] - s[b]);
            }
            w[a] = num / den;
            off[a] = (long)s[a];
        }
        return 4;
    }
    w[0] = 1.0 - t; off[0] = 0;
    w[1] = t;       off[1] = 1;
    return 2;
}

/* Derivative of the 1-D basis with respect to t: d/dt of each cardinal
 * polynomial, prod rule over its factors; linear: -1, 1. */
static void orc_basis_deriv(int order, double t, double dw[4])
{
    if (order == 4) {
        for (int a = 0; a < 4; ++a) dw[a] = orc_bspline_d(t - (double)(a - 1));
        return;
    }
    if (order == 3) {
        const double s[4] = {-1.0, 0.0, 1.0, 2.0};
        for (int a = 0; a < 4; ++a) {
            double den = 1.0;
            for (int b = 0; b < 4; ++b)
                if (b != a) den *= (s[a] - s[b]);
            double sum = 0.0;
            for (int skip = 0; skip < 4; ++skip) {
                if (skip == a) continue;
                double prod = 1.0;
                for (int b = 0; b < 4; ++b)
                    if (b != a && b != skip) prod *= (t - s[b]);
                sum += prod;
            }
            dw[a] = sum / den;
        }
        return;
    }
    dw[0] = -1.0;
    dw[1] = 1.0;
}

/* Stencil of the interpolant at grid-unit position y: wrapped node indices
 * and tensor-product weights.  Returns the node count per axis. */
static int orc_stencil(const long n[3], const double y[3], int order,
                       long idx[3][4], double w[3][4])
{
    int m = 0;
    for (int c = 0; c < 3; ++c) {
        double fl = floor(y[c]);
        long off[4];
        m = orc_basis(order, y[c] - fl, off, w[c]);
        for (int a = 0; a < m; ++a) idx[c][a] = orc_wrap((long)fl + off[a], n[c]);
    }
    return m;
}

static double orc_interp_at(const long n[3], const double *f, const double y[3], int order)
{
    long idx[3][4];
    double w[3][4];
    int m = orc_stencil(n, y, order, idx, w);
    double s = 0.0;
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b)
            for (int c = 0; c < m; ++c)
                s += w[0][a] * w[1][b] * w[2][c] *
                     f[(idx[0][a] * n[1] + idx[1][b]) * n[2] + idx[2][c]];
    return s;
}

/* Gradient (grid units, per axis) of the interpolant of f at x_p + d_p for
 * every node p: out[c][p] = d/dy_c I[f](y) at y = x_p + d_p. */
void orc_interp_grad(const long n[3], const double *f, const double *d, int order, double *out)
{
    const long N = n[0] * n[1] * n[2];
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; ++p) {
        long i = p / (n[1] * n[2]), j = (p / n[2]) % n[1], k = p % n[2];
        double y[3] = {i + d[p], j + d[N + p], k + d[2 * N + p]};
        long idx[3][4];
        double w[3][4], dw[3][4];
        int m = orc_stencil(n, y, order, idx, w);
        for (int c = 0; c < 3; ++c) orc_basis_deriv(order, y[c] - floor(y[c]), dw[c]);
        double g0 = 0.0, g1 = 0.0, g2 = 0.0;
        for (int a = 0; a < m; ++a)
            for (int b = 0; b < m; ++b)
                for (int c = 0; c < m; ++c) {
                    double fv = f[(idx[0][a] * n[1] + idx[1][b]) * n[2] + idx[2][c]];
                    g0 += dw[0][a] * w[1][b] * w[2][c] * fv;
                    g1 += w[0][a] * dw[1][b] * w[2][c] * fv;
                    g2 += w[0][a] * w[1][b] * dw[2][c] * fv;
                }
        out[p] = g0;
        out[N + p] = g1;
        out[2 * N + p] = g2;
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* out[p] = f(x_p + d_p) for every grid node p. */
void orc_interp(const long n[3], const double *f, const double *d, int order, double *out)
{
    const long N = n[0] * n[1] * n[2];
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; ++p) {
        long i = p / (n[1] * n[2]), j = (p / n[2]) % n[1], k = p % n[2];
        double y[3] = {i + d[p], j + d[N + p], k + d[2 * N + p]};
        out[p] = orc_interp_at(n, f, y, order);
    }
}

/* Interpolate at explicit grid-unit points y[3][M] (used for sampled checks). */
void orc_interp_points(const long n[3], const double *f, const double *y, long M, int order,
                       double *out)
{
#pragma omp parallel for schedule(static)
    for (long q = 0; q < M; ++q) {
        double yy[3] = {y[q], y[M + q], y[2 * M + q]};
        out[q] = orc_interp_at(n, f, yy, order);
    }
}

/* Exact transpose of orc_interp: out = W^T yv, i.e. every node receives the
 * weighted sum of the point values whose stencil touches it (serial scatter). */
void orc_interp_transpose(const long n[3], const double *yv, const double *d, int order,
                          double *out)
{
    const long N = n[0] * n[1] * n[2];
    memset(out, 0, sizeof(double) * (size_t)N);
    for (long p = 0; p < N; ++p) {
        long i = p / (n[1] * n[2]), j = (p / n[2]) % n[1], k = p % n[2];
        double y[3] = {i + d[p], j + d[N + p], k + d[2 * N + p]};
        long idx[3][4];
        double w[3][4];
        int m = orc_stencil(n, y, order, idx, w);
        for (int a = 0; a < m; ++a)
            for (int b = 0; b < m; ++b)
                for (int c = 0; c < m; ++c)
                    out[(idx[0][a] * n[1] + idx[1][b]) * n[2] + idx[2][c]] +=
                        w[0][a] * w[1][b] * w[2][c] * yv[p];
    }
}

/*
 * Heun (RK2) characteristic of a stationary velocity v (physical units).
 *   sign = +1: X  = x - dt/2 [v(x) + v(x - dt v(x))]   (state / incremental state)
 *   sign = -1: X+ = x + dt/2 [v(x) + v(x + dt v(x))]   (adjoint solves)
 * The velocity at the predictor point is interpolated with the same scheme as
 * the transported fields, from vc (v itself, or its B-spline coefficients for
 * order 4).  Output: d = (X - x) / h per axis, grid units.
 */
void orc_backtrace(const long n[3], const double *v, const double *vc, double dt, int sign, int order, double *d)
{
    const long N = n[0] * n[1] * n[2];
    double h[3];
    for (int c = 0; c < 3; ++c) h[c] = ORC_TWO_PI / (double)n[c];
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; ++p) {
        long i = p / (n[1] * n[2]), j = (p / n[2]) % n[1], k = p % n[2];
        double x[3] = {(double)i, (double)j, (double)k};
        double u0[3], ys[3];
        for (int c = 0; c < 3; ++c) {
            u0[c] = v[c * N + p] / h[c];
            ys[c] = x[c] - sign * dt * u0[c];
        }
        for (int c = 0; c < 3; ++c) {
            double us = orc_interp_at(n, vc + c * N, ys, order) / h[c];
            d[c * N + p] = -sign * 0.5 * dt * (u0[c] + us);
        }
    }
}

/* Standard 8th-order central first-derivative weights for offsets s = 1..4. */
static const double orc_fd8[4] = {4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0};

static double orc_fd8_axis(const long n[3], const double *f, long i, long j, long k, int axis)
{
    double s = 0.0;
    for (int q = 1; q <= 4; ++q) {
        long ip = i, jp = j, kp = k, im = i, jm = j, km = k;
        if (axis == 0) { ip = orc_wrap(i + q, n[0]); im = orc_wrap(i - q, n[0]); }
        if (axis == 1) { jp = orc_wrap(j + q, n[1]); jm = orc_wrap(j - q, n[1]); }
        if (axis == 2) { kp = orc_wrap(k + q, n[2]); km = orc_wrap(k - q, n[2]); }
        s += orc_fd8[q - 1] * (f[(ip * n[1] + jp) * n[2] + kp] - f[(im * n[1] + jm) * n[2] + km]);
    }
    return s * (double)n[axis] / ORC_TWO_PI;
}

/* g[c] = d f / d x_c, c = 0,1,2. */
void orc_fd8_grad(const long n[3], const double *f, double *g)
{
    const long N = n[0] * n[1] * n[2];
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; ++p) {
        long i = p / (n[1] * n[2]), j = (p / n[2]) % n[1], k = p % n[2];
        for (int c = 0; c < 3; ++c) g[c * N + p] = orc_fd8_axis(n, f, i, j, k, c);
    }
}

/* dv = sum_c d v_c / d x_c. */
void orc_fd8_div(const long n[3], const double *v, double *dv)
{
    const long N = n[0] * n[1] * n[2];
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; ++p) {
        long i = p / (n[1] * n[2]), j = (p / n[2]) % n[1], k = p % n[2];
        double s = 0.0;
        for (int c = 0; c < 3; ++c) s += orc_fd8_axis(n, v + c * N, i, j, k, c);
        dv[p] = s;
    }
}
