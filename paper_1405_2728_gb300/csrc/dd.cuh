// Double-double ("dd") arithmetic and the Newell auxiliary functions f, g.
//
// A dd value is an unevaluated sum hi + lo of two doubles with |lo| <= ulp(hi)/2,
// about 106 significant bits.  The error-free transformations are Knuth's
// TwoSum, Dekker's Fast2Sum and the FMA product (Dekker 1971; Knuth, TAOCP
// vol. 2, 4.2.2); the arithmetic on pairs follows the construction of
// Hida, Li and Bailey, "Algorithms for quad-double precision floating point
// arithmetic" (ARITH-15, 2001).  The elementary functions are written here from
// their mathematics: exp by ln 2 reduction, a scaled Taylor polynomial and
// repeated squaring; log by one Newton step on exp; atan by argument halving
// (atan t = 2 atan(t / (1 + sqrt(1 + t^2)))) and the alternating series; asinh
// through log.  The only library calls are double-precision first guesses.
//
// The Newell tensor needs this: its 27-point second difference cancels about
// R^6 (R in cells) of the magnitude of f and g, which leaves nothing of a
// double result beyond R ~ 500 cells.
//
// Compiled for the device (Newell setup kernels) and, through the same
// header, for the host in a unit test against multiprecision values.
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define DD_HD __host__ __device__ __forceinline__
#else
#define DD_HD static inline
#endif

struct dd_t {
    double hi, lo;
};

DD_HD dd_t dd_make(double h, double l) { dd_t r; r.hi = h; r.lo = l; return r; }
DD_HD dd_t dd_from(double h) { return dd_make(h, 0.0); }

// s + e == a + b exactly (Knuth TwoSum)
DD_HD dd_t dd_two_sum(double a, double b)
{
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return dd_make(s, e);
}

// s + e == a + b exactly when |a| >= |b| or a == 0 (Fast2Sum)
DD_HD dd_t dd_fast_two_sum(double a, double b)
{
    double s = a + b;
    double e = b - (s - a);
    return dd_make(s, e);
}

// p + e == a * b exactly (one FMA)
DD_HD dd_t dd_two_prod(double a, double b)
{
    double p = a * b;
    double e = fma(a, b, -p);
    return dd_make(p, e);
}

DD_HD dd_t dd_neg(dd_t a) { return dd_make(-a.hi, -a.lo); }

DD_HD dd_t dd_add(dd_t a, dd_t b)
{
    dd_t s = dd_two_sum(a.hi, b.hi);
    dd_t t = dd_two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = dd_fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return dd_fast_two_sum(s.hi, s.lo);
}

DD_HD dd_t dd_sub(dd_t a, dd_t b) { return dd_add(a, dd_neg(b)); }

DD_HD dd_t dd_add_d(dd_t a, double b)
{
    dd_t s = dd_two_sum(a.hi, b);
    s.lo += a.lo;
    return dd_fast_two_sum(s.hi, s.lo);
}

DD_HD dd_t dd_mul(dd_t a, dd_t b)
{
    dd_t p = dd_two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return dd_fast_two_sum(p.hi, p.lo);
}

DD_HD dd_t dd_mul_d(dd_t a, double b)
{
    dd_t p = dd_two_prod(a.hi, b);
    p.lo += a.lo * b;
    return dd_fast_two_sum(p.hi, p.lo);
}

// exact scaling by a power of two
DD_HD dd_t dd_ldexp(dd_t a, int e) { return dd_make(ldexp(a.hi, e), ldexp(a.lo, e)); }

// long division with three partial quotients
DD_HD dd_t dd_div(dd_t a, dd_t b)
{
    double q1 = a.hi / b.hi;
    dd_t r = dd_sub(a, dd_mul_d(b, q1));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul_d(b, q2));
    double q3 = r.hi / b.hi;
    dd_t q = dd_fast_two_sum(q1, q2);
    return dd_add_d(q, q3);
}

DD_HD dd_t dd_div_d(dd_t a, double b)
{
    double q1 = a.hi / b;
    dd_t r = dd_sub(a, dd_two_prod(q1, b));
    double q2 = r.hi / b;
    r = dd_sub(r, dd_two_prod(q2, b));
    double q3 = r.hi / b;
    dd_t q = dd_fast_two_sum(q1, q2);
    return dd_add_d(q, q3);
}

// sqrt by one Newton correction of the double root: y + (a - y^2)/(2y)
DD_HD dd_t dd_sqrt(dd_t a)
{
    if (!(a.hi > 0.0)) return dd_from(0.0);
    double y = sqrt(a.hi);
    dd_t r = dd_sub(a, dd_two_prod(y, y));
    return dd_fast_two_sum(y, r.hi / (2.0 * y));
}

// ln 2 and pi to ~107 bits (hi + lo); checked against multiprecision values in the unit tests
#define DD_LN2_HI 0x1.62e42fefa39efp-1
#define DD_LN2_LO 0x1.abc9e3b39803fp-56
#define DD_PI_HI 0x1.921fb54442d18p+1
#define DD_PI_LO 0x1.1a62633145c07p-53

// exp(a) for |a| < ~700: a = k ln2 + r, e^r = (e^(r/1024))^1024 with
// e^(r/1024) - 1 from its Taylor polynomial (terms to r^10/10!) and ten
// squarings of (1 + p) carried as p <- 2p + p^2.
DD_HD dd_t dd_exp(dd_t a)
{
    if (a.hi > 709.0) return dd_from(INFINITY);
    if (a.hi < -745.0) return dd_from(0.0);
    const double k = rint(a.hi / DD_LN2_HI);
    const dd_t ln2 = dd_make(DD_LN2_HI, DD_LN2_LO);
    dd_t r = dd_sub(a, dd_mul_d(ln2, k));
    r = dd_ldexp(r, -10);
    dd_t p = dd_from(1.0);
    for (int n = 10; n >= 2; --n)  // p = 1 + (r/n) p, Horner form of sum r^j/j!
        p = dd_add_d(dd_mul(dd_div_d(r, (double)n), p), 1.0);
    p = dd_mul(r, p);  // e^r - 1
    for (int i = 0; i < 10; ++i) p = dd_add(dd_ldexp(p, 1), dd_mul(p, p));
    return dd_ldexp(dd_add_d(p, 1.0), (int)k);
}

// log(a), a > 0: x0 = log(a.hi); u = a e^(-x0) - 1; log a = x0 + u - u^2/2 (+ O(u^3))
DD_HD dd_t dd_log(dd_t a)
{
    if (!(a.hi > 0.0)) return dd_from(NAN);
    const double x0 = log(a.hi);
    dd_t u = dd_add_d(dd_mul(a, dd_exp(dd_from(-x0))), -1.0);
    dd_t r = dd_add(dd_from(x0), u);
    return dd_add_d(r, -0.5 * u.hi * u.hi);
}

// asinh(t) = log(t + sqrt(t^2 + 1)) for t >= 0 (callers pass |t|)
DD_HD dd_t dd_asinh_nonneg(dd_t t)
{
    dd_t s = dd_sqrt(dd_add_d(dd_mul(t, t), 1.0));
    return dd_log(dd_add(t, s));
}

// atan(t) for t >= 0: halve the angle until t <= 1/16, then
// atan t = t sum_k (-t^2)^k/(2k+1), k = 0..13 (error < 2^-110 relative).
DD_HD dd_t dd_atan_nonneg(dd_t t)
{
    if (t.hi > 1e100) t = dd_from(1e100);
    int h = 0;
    while (t.hi > 0.0625 && h < 12) {
        dd_t den = dd_add_d(dd_sqrt(dd_add_d(dd_mul(t, t), 1.0)), 1.0);
        t = dd_div(t, den);
        ++h;
    }
    const dd_t u = dd_mul(t, t);
    dd_t p = dd_div_d(dd_from(1.0), 27.0);
    for (int k = 12; k >= 0; --k)
        p = dd_sub(dd_div_d(dd_from(1.0), (double)(2 * k + 1)), dd_mul(u, p));
    return dd_ldexp(dd_mul(t, p), h);
}

DD_HD int dd_is_pos(dd_t a) { return a.hi > 0.0; }

// Newell et al. (1993) f, even in x, y, z; arguments are non-negative here
// (callers pass |x|, |y|, |z|).  A term is dropped when its polynomial
// prefactor vanishes (its limit), which also avoids 0/0 in the arguments.
DD_HD dd_t dd_newell_f(dd_t x, dd_t y, dd_t z)
{
    const dd_t x2 = dd_mul(x, x), y2 = dd_mul(y, y), z2 = dd_mul(z, z);
    const dd_t R = dd_sqrt(dd_add(dd_add(x2, y2), z2));
    dd_t acc = dd_from(0.0);
    const dd_t z2mx2 = dd_sub(z2, x2), y2mx2 = dd_sub(y2, x2);
    if (dd_is_pos(y) && (z2mx2.hi != 0.0 || z2mx2.lo != 0.0)) {
        dd_t arg = dd_div(y, dd_sqrt(dd_add(x2, z2)));
        acc = dd_add(acc, dd_mul(dd_ldexp(dd_mul(y, z2mx2), -1), dd_asinh_nonneg(arg)));
    }
    if (dd_is_pos(z) && (y2mx2.hi != 0.0 || y2mx2.lo != 0.0)) {
        dd_t arg = dd_div(z, dd_sqrt(dd_add(x2, y2)));
        acc = dd_add(acc, dd_mul(dd_ldexp(dd_mul(z, y2mx2), -1), dd_asinh_nonneg(arg)));
    }
    if (dd_is_pos(x) && dd_is_pos(y) && dd_is_pos(z)) {
        dd_t yz = dd_mul(y, z);
        dd_t arg = dd_div(yz, dd_mul(x, R));
        acc = dd_sub(acc, dd_mul(dd_mul(x, yz), dd_atan_nonneg(arg)));
    }
    dd_t poly = dd_sub(dd_sub(dd_ldexp(x2, 1), y2), z2);
    acc = dd_add(acc, dd_div_d(dd_mul(poly, R), 6.0));
    return acc;
}

// Newell et al. (1993) g for non-negative x, y, z (the caller applies the
// sign: g is odd in x and in y, even in z).
DD_HD dd_t dd_newell_g(dd_t x, dd_t y, dd_t z)
{
    const dd_t x2 = dd_mul(x, x), y2 = dd_mul(y, y), z2 = dd_mul(z, z);
    const dd_t R = dd_sqrt(dd_add(dd_add(x2, y2), z2));
    const int px = dd_is_pos(x), py = dd_is_pos(y), pz = dd_is_pos(z);
    dd_t acc = dd_from(0.0);
    if (px && py && pz) {
        dd_t arg = dd_div(z, dd_sqrt(dd_add(x2, y2)));
        acc = dd_add(acc, dd_mul(dd_mul(dd_mul(x, y), z), dd_asinh_nonneg(arg)));
    }
    if (px && py) {
        dd_t arg = dd_div(x, dd_sqrt(dd_add(y2, z2)));
        dd_t pre = dd_div_d(dd_mul(y, dd_sub(dd_mul_d(z2, 3.0), y2)), 6.0);
        acc = dd_add(acc, dd_mul(pre, dd_asinh_nonneg(arg)));
        arg = dd_div(y, dd_sqrt(dd_add(x2, z2)));
        pre = dd_div_d(dd_mul(x, dd_sub(dd_mul_d(z2, 3.0), x2)), 6.0);
        acc = dd_add(acc, dd_mul(pre, dd_asinh_nonneg(arg)));
    }
    if (px && py && pz) {
        dd_t zR = dd_mul(z, R);
        dd_t t = dd_atan_nonneg(dd_div(dd_mul(x, y), zR));
        acc = dd_sub(acc, dd_mul(dd_div_d(dd_mul(z2, z), 6.0), t));
        t = dd_atan_nonneg(dd_div(dd_mul(x, z), dd_mul(y, R)));
        acc = dd_sub(acc, dd_mul(dd_ldexp(dd_mul(z, y2), -1), t));
        t = dd_atan_nonneg(dd_div(dd_mul(y, z), dd_mul(x, R)));
        acc = dd_sub(acc, dd_mul(dd_ldexp(dd_mul(z, x2), -1), t));
    }
    acc = dd_sub(acc, dd_div_d(dd_mul(dd_mul(x, y), R), 3.0));
    return acc;
}
