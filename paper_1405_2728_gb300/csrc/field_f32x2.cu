// Field kernels and their launchers instantiated for one precision:
// double fields, double-word FFT arithmetic (MM_F32X2).
#include "field_launch.cuh"

MM_DEFINE_FIELD_ENTRIES(f32x2, double, dfloat)
