/*
 * Oracle (test infrastructure only; never linked into the product library):
 * the cell-averaged demagnetisation tensor of a regular cuboid grid, evaluated
 * in quadruple precision.
 *
 * The paper (Section 3) computes the demagnetisation field "with an FFT
 * accelerated convolution" on a regular cuboid grid and names no tensor.  The
 * kernel used here is the cell-pair-averaged tensor of Newell, Williams and
 * Dunlop, J. Geophys. Res. 98 (1993) 9551: two auxiliary functions f (diagonal
 * entries) and g (off-diagonal entries) combined by a 27-point second
 * difference over the neighbouring lattice offsets,
 *
 *   N_xx(X,Y,Z) = 1/(4 pi dx dy dz) * sum_{e in {-1,0,1}^3} c(e) f(X+e1 dx, Y+e2 dy, Z+e3 dz)
 *   c(e) = 8, -4, 2, -1 for 0, 1, 2, 3 non-zero entries of e,
 *
 * with N_yy, N_zz by permuting coordinates (and cell sizes) and N_xy, N_xz,
 * N_yz likewise from g.  With this sign, H_demag = -Ms * sum_j N(r_i - r_j) m_j.
 *
 * The second difference cancels ~R^6 (R in cells) of the magnitude of f, so
 * the far field is evaluated in a 113-bit-mantissa type: __float128 with
 * libquadmath on x86-64, IEEE binary128 long double on aarch64.  Results are
 * rounded to double once, at the end.
 */
#include <math.h>
#include <float.h>
#include <stdint.h>
#include <stdlib.h>

#if defined(__x86_64__) || defined(__i386__)
#include <quadmath.h>
typedef __float128 qreal;
#define Q_ASINH asinhq
#define Q_ATAN atanq
#define Q_SQRT sqrtq
#define Q_FABS fabsq
#define Q_MANT FLT128_MANT_DIG
#elif defined(__aarch64__)
typedef long double qreal;
#define Q_ASINH asinhl
#define Q_ATAN atanl
#define Q_SQRT sqrtl
#define Q_FABS fabsl
#define Q_MANT LDBL_MANT_DIG
#else
#error "oracle needs a binary128 type: __float128 (x86-64) or long double (aarch64)"
#endif

#if Q_MANT < 113
#error "oracle quad type must carry a 113-bit mantissa"
#endif

/* f of Newell et al. (1993), used for the diagonal entries.  Even in x, y, z.
 * Every term is dropped when its polynomial prefactor vanishes; this is the
 * limit of the term and avoids 0/0 inside the inverse functions. */
static qreal newell_f(qreal x, qreal y, qreal z)
{
    x = Q_FABS(x); y = Q_FABS(y); z = Q_FABS(z);
    const qreal x2 = x * x, y2 = y * y, z2 = z * z;
    const qreal R = Q_SQRT(x2 + y2 + z2);
    qreal acc = 0;
    if (y > 0 && z2 != x2)
        acc += (y / 2) * (z2 - x2) * Q_ASINH(y / Q_SQRT(x2 + z2));
    if (z > 0 && y2 != x2)
        acc += (z / 2) * (y2 - x2) * Q_ASINH(z / Q_SQRT(x2 + y2));
    if (x > 0 && y > 0 && z > 0)
        acc -= x * y * z * Q_ATAN(y * z / (x * R));
    acc += (2 * x2 - y2 - z2) * R / 6;
    return acc;
}

/* g of Newell et al. (1993), used for the off-diagonal entries.  Odd in x and
 * in y, even in z; evaluated on |x|,|y|,|z| and signed afterwards. */
static qreal newell_g(qreal x, qreal y, qreal z)
{
    int sgn = 1;
    if (x < 0) { sgn = -sgn; x = -x; }
    if (y < 0) { sgn = -sgn; y = -y; }
    z = Q_FABS(z);
    const qreal x2 = x * x, y2 = y * y, z2 = z * z;
    const qreal R = Q_SQRT(x2 + y2 + z2);
    qreal acc = 0;
    if (x > 0 && y > 0 && z > 0)
        acc += x * y * z * Q_ASINH(z / Q_SQRT(x2 + y2));
    if (y > 0 && 3 * z2 != y2 && x > 0)
        acc += (y / 6) * (3 * z2 - y2) * Q_ASINH(x / Q_SQRT(y2 + z2));
    if (x > 0 && 3 * z2 != x2 && y > 0)
        acc += (x / 6) * (3 * z2 - x2) * Q_ASINH(y / Q_SQRT(x2 + z2));
    if (z > 0 && x > 0 && y > 0)
        acc -= (z2 * z / 6) * Q_ATAN(x * y / (z * R));
    if (z > 0 && y > 0 && x > 0)
        acc -= (z * y2 / 2) * Q_ATAN(x * z / (y * R));
    if (z > 0 && x > 0 && y > 0)
        acc -= (z * x2 / 2) * Q_ATAN(y * z / (x * R));
    acc -= x * y * R / 3;
    return sgn > 0 ? acc : -acc;
}

/* Weight of a stencil offset with nnz non-zero entries. */
static const int STENCIL_W[4] = {8, -4, 2, -1};

static qreal q_pi(void) { return 4 * Q_ATAN((qreal)1); }

/* One tensor entry set at a signed lattice offset (i,j,k), all six
 * components, directly from 27 evaluations of f and g each. */
static void entry_q(long i, long j, long k, qreal hx, qreal hy, qreal hz, qreal out[6])
{
    qreal s[6] = {0, 0, 0, 0, 0, 0};
    for (int e1 = -1; e1 <= 1; ++e1)
        for (int e2 = -1; e2 <= 1; ++e2)
            for (int e3 = -1; e3 <= 1; ++e3) {
                const int w = STENCIL_W[(e1 != 0) + (e2 != 0) + (e3 != 0)];
                const qreal X = (qreal)(i + e1) * hx, Y = (qreal)(j + e2) * hy, Z = (qreal)(k + e3) * hz;
                s[0] += w * newell_f(X, Y, Z);
                s[1] += w * newell_f(Y, X, Z);
                s[2] += w * newell_f(Z, Y, X);
                s[3] += w * newell_g(X, Y, Z);
                s[4] += w * newell_g(X, Z, Y);
                s[5] += w * newell_g(Y, Z, X);
            }
    const qreal norm = 1 / (4 * q_pi() * hx * hy * hz);
    for (int c = 0; c < 6; ++c) out[c] = s[c] * norm;
}

/* Scale the cell so its largest edge is 1 (the tensor is scale-free). */
static int scaled_cell(double dx, double dy, double dz, qreal *hx, qreal *hy, qreal *hz)
{
    if (!(dx > 0) || !(dy > 0) || !(dz > 0)) return -1;
    double h = dx;
    if (dy > h) h = dy;
    if (dz > h) h = dz;
    *hx = (qreal)dx / (qreal)h; *hy = (qreal)dy / (qreal)h; *hz = (qreal)dz / (qreal)h;
    return 0;
}

/* Newell f / g at one point, rounded to double (for the oracle's own pins). */
double oracle_newell_f(double x, double y, double z) { return (double)newell_f(x, y, z); }
double oracle_newell_g(double x, double y, double z) { return (double)newell_g(x, y, z); }

/* All six components at one signed lattice offset; out[6] = xx,yy,zz,xy,xz,yz. */
int oracle_newell_entry(long i, long j, long k, double dx, double dy, double dz, double out[6])
{
    qreal hx, hy, hz, q[6];
    if (scaled_cell(dx, dy, dz, &hx, &hy, &hz)) return -1;
    entry_q(i, j, k, hx, hy, hz, q);
    for (int c = 0; c < 6; ++c) out[c] = (double)q[c];
    return 0;
}

/*
 * The first octant of offsets, 0 <= i < nx, 0 <= j < ny, 0 <= k < nz, for all
 * six components: out[c][k][j][i] (x fastest), c = xx,yy,zz,xy,xz,yz.  The
 * other octants follow from N_aa even in every coordinate and N_ab odd in
 * coordinates a and b.  f and g are tabulated once on the (nx+1)(ny+1)(nz+1)
 * non-negative lattice and the 27-point stencil reads them with |index|
 * (and the sign rule of g).  Returns 0, or -1 on bad arguments / no memory.
 */
int oracle_newell_octant(int nx, int ny, int nz, double dx, double dy, double dz, double *out)
{
    qreal hx, hy, hz;
    if (nx < 1 || ny < 1 || nz < 1 || !out) return -1;
    if (scaled_cell(dx, dy, dz, &hx, &hy, &hz)) return -1;
    const long ax = nx + 1, ay = ny + 1, az = nz + 1, na = ax * ay * az;
    qreal *T = (qreal *)malloc(sizeof(qreal) * 6 * (size_t)na);
    if (!T) return -1;
    /* T[c][c3][b][a]: lattice point (a,b,c3) in units of cells. */
#pragma omp parallel for schedule(dynamic, 64)
    for (long p = 0; p < na; ++p) {
        const long a = p % ax, b = (p / ax) % ay, c3 = p / (ax * ay);
        const qreal X = a * hx, Y = b * hy, Z = c3 * hz;
        T[0 * na + p] = newell_f(X, Y, Z);
        T[1 * na + p] = newell_f(Y, X, Z);
        T[2 * na + p] = newell_f(Z, Y, X);
        T[3 * na + p] = newell_g(X, Y, Z);
        T[4 * na + p] = newell_g(X, Z, Y);
        T[5 * na + p] = newell_g(Y, Z, X);
    }
    const qreal norm = 1 / (4 * q_pi() * hx * hy * hz);
    const long nn = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (long p = 0; p < nn; ++p) {
        const long i = p % nx, j = (p / nx) % ny, k = p / ((long)nx * ny);
        qreal s[6] = {0, 0, 0, 0, 0, 0};
        for (int e1 = -1; e1 <= 1; ++e1)
            for (int e2 = -1; e2 <= 1; ++e2)
                for (int e3 = -1; e3 <= 1; ++e3) {
                    const int w = STENCIL_W[(e1 != 0) + (e2 != 0) + (e3 != 0)];
                    const long a = i + e1, b = j + e2, c3 = k + e3;
                    const long q = (labs(c3) * ay + labs(b)) * ax + labs(a);
                    const int sa = a < 0 ? -1 : 1, sb = b < 0 ? -1 : 1, sc = c3 < 0 ? -1 : 1;
                    s[0] += w * T[0 * na + q];
                    s[1] += w * T[1 * na + q];
                    s[2] += w * T[2 * na + q];
                    s[3] += (w * sa * sb) * T[3 * na + q]; /* g(x,y,z): odd in x, y */
                    s[4] += (w * sa * sc) * T[4 * na + q]; /* g(x,z,y): odd in x, z */
                    s[5] += (w * sb * sc) * T[5 * na + q]; /* g(y,z,x): odd in y, z */
                }
        for (int c = 0; c < 6; ++c) out[(size_t)c * nn + p] = (double)(s[c] * norm);
    }
    free(T);
    return 0;
}

/* Number of mantissa bits of the quad type this oracle was built with. */
int oracle_quad_mant_dig(void) { return Q_MANT; }
