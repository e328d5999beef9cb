// Host build of the library's double-double header, for unit tests against
// multiprecision values (compiled by tests/test_dd_host.py with g++).
#include "../paper_1405_2728_gb300/csrc/dd.cuh"

extern "C" {
static void put(dd_t r, double *out) { out[0] = r.hi; out[1] = r.lo; }
void h_exp(double hi, double lo, double *out) { put(dd_exp(dd_make(hi, lo)), out); }
void h_log(double hi, double lo, double *out) { put(dd_log(dd_make(hi, lo)), out); }
void h_atan(double hi, double lo, double *out) { put(dd_atan_nonneg(dd_make(hi, lo)), out); }
void h_asinh(double hi, double lo, double *out) { put(dd_asinh_nonneg(dd_make(hi, lo)), out); }
void h_sqrt(double hi, double lo, double *out) { put(dd_sqrt(dd_make(hi, lo)), out); }
void h_div(double ah, double al, double bh, double bl, double *out) { put(dd_div(dd_make(ah, al), dd_make(bh, bl)), out); }
void h_f(double x, double y, double z, double *out) { put(dd_newell_f(dd_from(x), dd_from(y), dd_from(z)), out); }
void h_g(double x, double y, double z, double *out) { put(dd_newell_g(dd_from(x), dd_from(y), dd_from(z)), out); }
void h_consts(double *out) { out[0] = DD_LN2_HI; out[1] = DD_LN2_LO; out[2] = DD_PI_HI; out[3] = DD_PI_LO; }
}
