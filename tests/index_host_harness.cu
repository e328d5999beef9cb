// Host build of the field kernels' index helpers (csrc/common.cuh, csrc/fft.cuh),
// for unit tests of their arithmetic on the CPU (compiled by
// tests/test_index_host.py with nvcc; nothing here runs on a GPU).
#include "../paper_1405_2728_gb300/csrc/fft.cuh"

extern "C" {
void h_fastdiv_init(int d, unsigned *mul, int *shift)
{
    FastDiv f;
    f.init(d);
    *mul = f.mul;
    *shift = f.shift;
}
int h_spos_float(int i) { return spos<float2>(i); }
int h_spos_double(int i) { return spos<double2>(i); }
int h_row_stride(int L, int esz) { return row_stride(L, esz); }
}
