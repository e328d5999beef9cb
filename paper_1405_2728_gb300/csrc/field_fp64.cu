// Field kernels and their launchers instantiated for one precision:
// double fields, double FFT arithmetic (MM_FP64).
#include "field_launch.cuh"

MM_DEFINE_FIELD_ENTRIES(fp64, double, double)
