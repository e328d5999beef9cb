// Field kernels and their launchers instantiated for one precision:
// float fields, float FFT arithmetic (MM_FP32).
#include "field_launch.cuh"

MM_DEFINE_FIELD_ENTRIES(fp32, float, float)
