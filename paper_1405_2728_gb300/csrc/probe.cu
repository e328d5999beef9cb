// Instrumentation: measured fused-multiply-add throughput of the FP64 and FP32
// pipes of the current device.  The field kernels of the double path are
// bound by the FP64 units (not by HBM), so their roofline needs this peak,
// which the copy-bandwidth and GEMM figures do not give.
//
// Each thread runs NCH independent FMA chains x <- x * a + b (a just below 1,
// so the chains converge and stay normal); the chains keep the pipe busy
// without depending on memory.  The grid fills every SM with several CTAs.
#include "common.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int NCH = 16;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_chains(int iters, T a, T b, T *sink)
{
    T x[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < NCH; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < NCH; ++c) s += x[c];
    // the store keeps the chains alive; every thread writes its own slot
    sink[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

template <typename T>
int time_chains(int blocks, int iters, T *sink, double *tflops)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a)) return MM_ERR_CUDA;
    if (cudaEventCreate(&b)) { cudaEventDestroy(a); return MM_ERR_CUDA; }
    const T fa = (T)0.9999999, fb = (T)1e-7;
    float best = 1e30f;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < 6 && !e; ++r) {  // first launch warms the clocks; best of the rest
        cudaEventRecord(a, 0);
        k_fma_chains<T><<<blocks, PROBE_THREADS>>>(iters, fa, fb, sink);
        cudaEventRecord(b, 0);
        if ((e = cudaGetLastError()) || (e = cudaEventSynchronize(b))) break;
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        if (r > 0 && t < best) best = t;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e) { mm_set_cuda_error(e, "mm_probe_fma"); return MM_ERR_CUDA; }
    const double fl = 2.0 * NCH * (double)iters * blocks * PROBE_THREADS;
    *tflops = fl / (best * 1e-3) / 1e12;
    return MM_OK;
}

} // namespace

extern "C" MM_API int mm_probe_fma(double tflops_out[2])
{
    if (!tflops_out) return MM_ERR_ARG;
    const int blocks = mm_sm_count() * 8;
    double *sink = nullptr;
    cudaError_t e = cudaMalloc((void **)&sink, sizeof(double) * (size_t)blocks * PROBE_THREADS);
    if (e) { mm_set_cuda_error(e, "cudaMalloc"); return MM_ERR_OOM; }
    // about 5 ms per launch at the nominal rates (2 FP64 and 128 FP32 FMA
    // per SM per clock)
    int rc = time_chains<double>(blocks, 624, sink, &tflops_out[0]);
    if (rc == MM_OK) rc = time_chains<float>(blocks, 624 * 64, (float *)sink, &tflops_out[1]);
    cudaFree(sink);
    return rc;
}
