// Field kernels and their launchers instantiated for one precision:
// double-word fields and arithmetic (MM_F32X2); the caller's arrays are double.
#include "field_launch.cuh"

MM_DEFINE_FIELD_ENTRIES(f32x2, dfloat, dfloat)
