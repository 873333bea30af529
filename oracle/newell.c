/*
 * Oracle: demagnetisation tensor of a uniform grid of rectangular cells.
 *
 * TEST INFRASTRUCTURE ONLY.  This file belongs to the plain CPU oracle that
 * the parity tests and the benchmark's CPU baseline compare the CUDA path
 * against.  Nothing in the product library links, includes or calls it.
 *
 * What it computes (paper Sec. II-B, demag equation of Sec. II-A, and the
 * FFT-convolution method of Nakatani et al. / Hayashi et al. it cites):
 *   N_ij(R) = cell-averaged field tensor between two cells whose centres are
 *   R apart, defined so that H_i(target) = -sum_j N_ij(R) M_j(source).  By
 *   definition
 *       N_ij(R) = -1/(4 pi V) * Int_{[-d,d]^3} L(u) d_i d_j (1/|R+u|) du,
 *   L(u) = prod_k (d_k - |u_k|)  (the overlap volume of two boxes).
 *
 * Two evaluations of that definition:
 *   near offsets: the closed form of Newell, Williams & Dunlop (J. Geophys.
 *     Res. 98, 9551, 1993): auxiliary functions f (diagonal) and g
 *     (off-diagonal) combined with the 27-point weights (-1, 2, -1)^3.
 *     The combination cancels catastrophically as |R| grows (relative error
 *     about eps * (|R|/d)^6), so it is used only up to a switch distance.
 *   far offsets: Gauss-Legendre quadrature of the definition above, with
 *     every axis split at u_k = 0 where L(u) has its kink; the integrand is
 *     smooth there because the singular point u = -R lies outside the box.
 *
 * A third, extended-precision evaluation of Newell's closed form (binary128:
 * __float128 with libquadmath on x86-64, long double on AArch64) exists for
 * the pins only: it does not suffer the cancellation at the distances used.
 *
 * Component order everywhere: xx, yy, zz, xy, xz, yz.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#if defined(__x86_64__) && defined(MXO_HAVE_QUADMATH)
#include <quadmath.h>
typedef __float128 qreal;
#define Q_SQRT sqrtq
#define Q_ASINH asinhq
#define Q_ATAN atanq
#define MXO_HAS_QUAD 1
#elif defined(__aarch64__)
typedef long double qreal; /* IEEE binary128 on AArch64 Linux */
#define Q_SQRT sqrtl
#define Q_ASINH asinhl
#define Q_ATAN atanl
#define MXO_HAS_QUAD 1
#else
#define MXO_HAS_QUAD 0
#endif

#define MXO_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------ */
/* Newell's auxiliary functions in double precision.                   */
/* Every term whose polynomial prefactor vanishes is taken as zero: its */
/* transcendental factor may be singular there but the product tends   */
/* to zero.                                                            */
/* ------------------------------------------------------------------ */
static double newell_f(double x, double y, double z)
{
    double x2 = x * x, y2 = y * y, z2 = z * z;
    double R = sqrt(x2 + y2 + z2);
    if (R == 0.0) return 0.0;
    double s = 0.0;
    double p;
    p = 0.5 * y * (z2 - x2);
    if (p != 0.0) s += p * asinh(y / sqrt(x2 + z2));
    p = 0.5 * z * (y2 - x2);
    if (p != 0.0) s += p * asinh(z / sqrt(x2 + y2));
    p = x * y * z;
    if (p != 0.0) s -= p * atan(y * z / (x * R));
    s += (2.0 * x2 - y2 - z2) * R / 6.0;
    return s;
}

static double newell_g(double x, double y, double z)
{
    double x2 = x * x, y2 = y * y, z2 = z * z;
    double R = sqrt(x2 + y2 + z2);
    if (R == 0.0) return 0.0;
    double s = 0.0;
    double p;
    p = x * y * z;
    if (p != 0.0) s += p * asinh(z / sqrt(x2 + y2));
    p = y * (3.0 * z2 - y2) / 6.0;
    if (p != 0.0) s += p * asinh(x / sqrt(y2 + z2));
    p = x * (3.0 * z2 - x2) / 6.0;
    if (p != 0.0) s += p * asinh(y / sqrt(x2 + z2));
    p = z * z2 / 6.0;
    if (p != 0.0) s -= p * atan(x * y / (z * R));
    p = 0.5 * z * y2;
    if (p != 0.0) s -= p * atan(x * z / (y * R));
    p = 0.5 * z * x2;
    if (p != 0.0) s -= p * atan(y * z / (x * R));
    s -= x * y * R / 3.0;
    return s;
}

typedef double (*aux_fn)(double, double, double);

/* Sum over a, b, c in {-1,0,1} of w_a w_b w_c F(X + a hx, Y + b hy, Z + c hz)
   with w_0 = 2, w_{+-1} = -1, divided by 4 pi hx hy hz.                    */
static double newell_combo(aux_fn F, double X, double Y, double Z,
                           double hx, double hy, double hz)
{
    static const double w[3] = {-1.0, 2.0, -1.0};
    double s = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c)
                s += w[a] * w[b] * w[c] *
                     F(X + (a - 1) * hx, Y + (b - 1) * hy, Z + (c - 1) * hz);
    return s / (4.0 * MXO_PI * hx * hy * hz);
}

/* All six components from the closed form.  The diagonal ones use f with
   the component's own axis first; the off-diagonal ones use g with the two
   coupled axes first and the third axis last.                            */
static void newell_all(double X, double Y, double Z, double dx, double dy,
                       double dz, double out[6])
{
    out[0] = newell_combo(newell_f, X, Y, Z, dx, dy, dz);
    out[1] = newell_combo(newell_f, Y, X, Z, dy, dx, dz);
    out[2] = newell_combo(newell_f, Z, Y, X, dz, dy, dx);
    out[3] = newell_combo(newell_g, X, Y, Z, dx, dy, dz);
    out[4] = newell_combo(newell_g, X, Z, Y, dx, dz, dy);
    out[5] = newell_combo(newell_g, Y, Z, X, dy, dz, dx);
}

/* ------------------------------------------------------------------ */
/* Gauss-Legendre nodes/weights on [-1,1] by Newton's method on the     */
/* three-term Legendre recurrence (textbook construction).             */
/* ------------------------------------------------------------------ */
#define MXO_MAX_GL 16
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double t = cos(MXO_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = t; p0 = 1.0; }
            /* p1 = P_n(t), p0 = P_{n-1}(t) */
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        x[i] = -t;
        x[n - 1 - i] = t;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

/* Quadrature of the defining integral with n Gauss points on each half of
   every axis ((2n)^3 evaluations).                                        */
static void quad_all(double X, double Y, double Z, double dx, double dy,
                     double dz, int n, double out[6])
{
    double gx[MXO_MAX_GL], gw[MXO_MAX_GL];
    if (n > MXO_MAX_GL) n = MXO_MAX_GL;
    gauss_legendre(n, gx, gw);
    /* one-dimensional node lists: u in [-d,0] and [0,d], weight times the
       factor (d - |u|) of L(u). */
    double ux[2 * MXO_MAX_GL], wx[2 * MXO_MAX_GL];
    double uy[2 * MXO_MAX_GL], wy[2 * MXO_MAX_GL];
    double uz[2 * MXO_MAX_GL], wz[2 * MXO_MAX_GL];
    const double d3[3] = {dx, dy, dz};
    double *U[3] = {ux, uy, uz}, *W[3] = {wx, wy, wz};
    for (int k = 0; k < 3; ++k) {
        double h = d3[k];
        for (int i = 0; i < n; ++i) {
            double u = 0.5 * h * (1.0 + gx[i]); /* in [0,h] */
            double wt = 0.5 * h * gw[i] * (h - u);
            U[k][i] = u;
            W[k][i] = wt;
            U[k][n + i] = -u;
            W[k][n + i] = wt;
        }
    }
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int a = 0; a < 2 * n; ++a) {
        double rx = X + ux[a];
        for (int b = 0; b < 2 * n; ++b) {
            double ry = Y + uy[b];
            double wab = wx[a] * wy[b];
            for (int c = 0; c < 2 * n; ++c) {
                double rz = Z + uz[c];
                double r2 = rx * rx + ry * ry + rz * rz;
                double ir = 1.0 / sqrt(r2);
                double ir5 = ir * ir * ir * ir * ir;
                double wt = wab * wz[c] * ir5;
                /* d_i d_j (1/r) = (3 r_i r_j - delta_ij r^2) / r^5 */
                s[0] += wt * (3.0 * rx * rx - r2);
                s[1] += wt * (3.0 * ry * ry - r2);
                s[2] += wt * (3.0 * rz * rz - r2);
                s[3] += wt * (3.0 * rx * ry);
                s[4] += wt * (3.0 * rx * rz);
                s[5] += wt * (3.0 * ry * rz);
            }
        }
    }
    double V = dx * dy * dz;
    for (int k = 0; k < 6; ++k) out[k] = -s[k] / (4.0 * MXO_PI * V);
}

/* Distance from the singular point u = -R to the box [-d,d]^3, in units of
   the largest cell edge. */
static double sep_cells(double X, double Y, double Z, double dx, double dy,
                        double dz)
{
    double ex = fabs(X) - dx, ey = fabs(Y) - dy, ez = fabs(Z) - dz;
    ex = ex > 0 ? ex : 0;
    ey = ey > 0 ? ey : 0;
    ez = ez > 0 ? ez : 0;
    double h = dx > dy ? dx : dy;
    h = h > dz ? h : dz;
    return sqrt(ex * ex + ey * ey + ez * ez) / h;
}

/* Number of Gauss points per half-axis for a separation s (in cells);
   chosen so the quadrature error stays near 1e-13 relative (checked
   against the binary128 closed form by the oracle's tests). */
static int quad_points(double s)
{
    if (s >= 80.0) return 3;
    if (s >= 30.0) return 4;
    if (s >= 12.0) return 6;
    if (s >= 4.0) return 8;
    if (s >= 2.0) return 12;
    return 16;
}

/* Closed form while |R| <= switch * V^(1/3): there the cancellation costs
   at most eps * switch^6.  The quadrature needs the box to stay clear of
   the singular point, so the closed form is also kept for separations
   below one cell edge whatever |R| is (elongated cells only). */
static double g_switch_cells = 5.0;

void mxo_set_switch(double cells) { g_switch_cells = cells; }
double mxo_get_switch(void) { return g_switch_cells; }

static int use_closed_form(double X, double Y, double Z, double dx, double dy,
                           double dz)
{
    double R = sqrt(X * X + Y * Y + Z * Z);
    double h = cbrt(dx * dy * dz);
    return R <= g_switch_cells * h || sep_cells(X, Y, Z, dx, dy, dz) < 1.0;
}

/* ------------------------------------------------------------------ */
/* Exported entry points (called through ctypes).                      */
/* ------------------------------------------------------------------ */

/* Closed form in double precision at one offset. */
void mxo_newell_f64(double X, double Y, double Z, double dx, double dy,
                    double dz, double *out6)
{
    newell_all(X, Y, Z, dx, dy, dz, out6);
}

/* Quadrature with n points per half-axis at one offset. */
void mxo_quad_f64(double X, double Y, double Z, double dx, double dy, double dz,
                  int n, double *out6)
{
    quad_all(X, Y, Z, dx, dy, dz, n, out6);
}

/* The oracle's tensor at one offset: closed form near, quadrature far. */
void mxo_tensor_at(double X, double Y, double Z, double dx, double dy,
                   double dz, double *out6)
{
    if (use_closed_form(X, Y, Z, dx, dy, dz))
        newell_all(X, Y, Z, dx, dy, dz, out6);
    else
        quad_all(X, Y, Z, dx, dy, dz,
                 quad_points(sep_cells(X, Y, Z, dx, dy, dz)), out6);
}

/* Tensor on the non-negative offsets X = i dx, Y = j dy, Z = k dz with
   0 <= i < nx, 0 <= j < ny, 0 <= k < nz.  Output layout:
   out[c][k][j][i], c = 0..5 (xx, yy, zz, xy, xz, yz). */
void mxo_tensor_octant(int nx, int ny, int nz, double dx, double dy, double dz,
                       double *out)
{
    long plane = (long)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 16) collapse(2)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double t[6];
                mxo_tensor_at(i * dx, j * dy, k * dz, dx, dy, dz, t);
                long o = ((long)k * ny + j) * nx + i;
                for (int c = 0; c < 6; ++c) out[c * plane + o] = t[c];
            }
}

int mxo_has_quad(void) { return MXO_HAS_QUAD; }

#if MXO_HAS_QUAD
static qreal q_f(qreal x, qreal y, qreal z)
{
    qreal x2 = x * x, y2 = y * y, z2 = z * z;
    qreal R = Q_SQRT(x2 + y2 + z2);
    if (R == 0) return 0;
    qreal s = 0, p;
    p = (qreal)0.5 * y * (z2 - x2);
    if (p != 0) s += p * Q_ASINH(y / Q_SQRT(x2 + z2));
    p = (qreal)0.5 * z * (y2 - x2);
    if (p != 0) s += p * Q_ASINH(z / Q_SQRT(x2 + y2));
    p = x * y * z;
    if (p != 0) s -= p * Q_ATAN(y * z / (x * R));
    s += (2 * x2 - y2 - z2) * R / 6;
    return s;
}

static qreal q_g(qreal x, qreal y, qreal z)
{
    qreal x2 = x * x, y2 = y * y, z2 = z * z;
    qreal R = Q_SQRT(x2 + y2 + z2);
    if (R == 0) return 0;
    qreal s = 0, p;
    p = x * y * z;
    if (p != 0) s += p * Q_ASINH(z / Q_SQRT(x2 + y2));
    p = y * (3 * z2 - y2) / 6;
    if (p != 0) s += p * Q_ASINH(x / Q_SQRT(y2 + z2));
    p = x * (3 * z2 - x2) / 6;
    if (p != 0) s += p * Q_ASINH(y / Q_SQRT(x2 + z2));
    p = z * z2 / 6;
    if (p != 0) s -= p * Q_ATAN(x * y / (z * R));
    p = z * y2 / 2;
    if (p != 0) s -= p * Q_ATAN(x * z / (y * R));
    p = z * x2 / 2;
    if (p != 0) s -= p * Q_ATAN(y * z / (x * R));
    s -= x * y * R / 3;
    return s;
}

typedef qreal (*q_aux_fn)(qreal, qreal, qreal);

static double q_combo(q_aux_fn F, double X, double Y, double Z, double hx,
                      double hy, double hz)
{
    static const int w[3] = {-1, 2, -1};
    qreal s = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 3; ++c)
                s += (qreal)(w[a] * w[b] * w[c]) *
                     F((qreal)X + (a - 1) * (qreal)hx,
                       (qreal)Y + (b - 1) * (qreal)hy,
                       (qreal)Z + (c - 1) * (qreal)hz);
    qreal pi = (qreal)4 * Q_ATAN((qreal)1);
    return (double)(s / (4 * pi * (qreal)hx * (qreal)hy * (qreal)hz));
}
#endif

/* Closed form in binary128 at one offset (pins only).  Returns 0 if this
   platform has no binary128 arithmetic available. */
int mxo_newell_q(double X, double Y, double Z, double dx, double dy, double dz,
                 double *out6)
{
#if MXO_HAS_QUAD
    out6[0] = q_combo(q_f, X, Y, Z, dx, dy, dz);
    out6[1] = q_combo(q_f, Y, X, Z, dy, dx, dz);
    out6[2] = q_combo(q_f, Z, Y, X, dz, dy, dx);
    out6[3] = q_combo(q_g, X, Y, Z, dx, dy, dz);
    out6[4] = q_combo(q_g, X, Z, Y, dx, dz, dy);
    out6[5] = q_combo(q_g, Y, Z, X, dy, dz, dx);
    return 1;
#else
    (void)X; (void)Y; (void)Z; (void)dx; (void)dy; (void)dz;
    memset(out6, 0, 6 * sizeof(double));
    return 0;
#endif
}
