// Mixed-precision hysteresis sweep (an extension; the paper uses one
// precision).  Per field value, the float problem minimises from the current
// state to a loose tolerance.  The double problem then takes its result and
// minimises to the final tolerance.  The float field arithmetic is ~10x
// faster per evaluation.  Its rounding noise, though, makes the last decades
// of the stop rule (Section 2) slow: the step-size sums become differences of
// noisy gradients, so the cheap phase stops at the loose tolerance.
//
// Both problems must describe the same grid and material; each keeps its own
// device-side minimiser loop (CUDA graph).  The state moves between them by
// a conversion kernel that reads the source problem's current iterate (the
// buffer its minimiser state points at) and writes the destination's
// iterate 0.  Everything of one sweep is issued on one stream; the host
// waits once, for the records.
#include <cmath>
#include <new>
#include <vector>

#include "common.cuh"

namespace {

// element conversions between the iterate types of the two problems
__device__ __forceinline__ void put(float &d, double v) { d = (float)v; }
__device__ __forceinline__ void put(double &d, float v) { d = v; }
__device__ __forceinline__ void put(float &d, dfloat v) { d = __fadd_rn(v.hi, v.lo); }  // nearest float to hi + lo
__device__ __forceinline__ void put(dfloat &d, float v) { d = dfloat(v, 0.0f); }

template <typename S, typename D>
__global__ void k_transfer(const MinState *st, const S *b0, const S *b1, D *dst, long n3)
{
    const S *src = (st->base ^ (int)(st->k & 1)) ? b1 : b0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n3; i += (long)gridDim.x * blockDim.x)
        put(dst[i], src[i]);
}

template <typename S, typename D> void launch_transfer(mm_problem *from, mm_problem *to, long n3, cudaStream_t s)
{
    k_transfer<S, D><<<mm_grid_for(n3, 256, 8), 256, 0, s>>>(from->st, (const S *)from->mbuf[0],
                                                            (const S *)from->mbuf[1], (D *)to->mbuf[0], n3);
}

// current iterate of `from` -> iterate 0 of `to` (converted): the float
// problem and the double (or double-word) one, in either direction
int transfer(mm_problem *from, mm_problem *to, cudaStream_t s)
{
    const long n3 = 3 * from->g.N;
    if (from->precision == MM_FP64) launch_transfer<double, float>(from, to, n3, s);
    else if (from->precision == MM_F32X2) launch_transfer<dfloat, float>(from, to, n3, s);
    else if (to->precision == MM_FP64) launch_transfer<float, double>(from, to, n3, s);
    else launch_transfer<float, dfloat>(from, to, n3, s);
    cudaError_t e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "k_transfer"); return MM_ERR_CUDA; }
    return MM_OK;
}

int status_of_rec(int s)
{
    switch (s) {
    case MMS_CONVERGED: return MM_OK;
    case MMS_MAXITER: return MM_ERR_NOT_CONVERGED;
    case MMS_NONFINITE: return MM_ERR_NONFINITE;
    case MMS_TIMEOUT: return MM_ERR_TIMEOUT;
    }
    return MM_ERR_CUDA;
}

bool opts_valid(const mm_min_opts *o) { return mm_opts_ok(o); }

int ensure_records(mm_problem *p, int n)
{
    if (p->rec_cap >= n) return MM_OK;
    if (p->rec_dev) { cudaFree(p->rec_dev); p->bytes -= (long)sizeof(StepRecord) * p->rec_cap; p->rec_dev = nullptr; }
    cudaError_t e = cudaMalloc((void **)&p->rec_dev, sizeof(StepRecord) * (size_t)n);
    if (e) { p->rec_cap = 0; mm_set_cuda_error(e, "cudaMalloc(records)"); return MM_ERR_OOM; }
    p->bytes += (long)sizeof(StepRecord) * n;
    p->rec_cap = n;
    return MM_OK;
}

int read_records(mm_problem *p, int n, int start, std::vector<StepRecord> &rec, cudaStream_t s)
{
    rec.resize((size_t)n);
    cudaError_t e = cudaMemcpyAsync(rec.data() + start, p->rec_dev + start, sizeof(StepRecord) * (size_t)(n - start),
                                    cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) { mm_set_cuda_error(e, "mm_hysteresis_sweep_mixed"); return MM_ERR_CUDA; }
    return MM_OK;
}

void fill_result(const StepRecord &r, mm_min_result &o, int launches_extra)
{
    o.iters = r.iters; o.heff_evals = r.evals; o.max_torque = r.max_torque; o.energy = r.energy;
    o.converged = r.status == MMS_CONVERGED; o.status = status_of_rec(r.status);
    o.kernel_launches = r.launches + launches_extra;
}

} // namespace

extern "C" MM_API int mm_hysteresis_sweep_mixed(mm_problem *lo, mm_problem *hi, void *m, const double *H_list, int n,
                                                int start, const mm_min_opts *opts_lo, const mm_min_opts *opts_hi,
                                                double *mavg, mm_min_result *per_step_lo, mm_min_result *per_step_hi,
                                                void *stream)
{
    if (!lo || !hi || !m || !H_list || !mavg || n < 1 || start < 0 || start >= n || !opts_valid(opts_lo) ||
        !opts_valid(opts_hi))
        return MM_ERR_ARG;
    if (lo->precision != MM_FP32 || !mm_double_fields(hi) || lo->g.nx != hi->g.nx || lo->g.ny != hi->g.ny ||
        lo->g.nz != hi->g.nz)
        return MM_ERR_ARG;
    for (int j = start; j < n; ++j)
        if (!std::isfinite(H_list[3 * j]) || !std::isfinite(H_list[3 * j + 1]) || !std::isfinite(H_list[3 * j + 2]))
            return MM_ERR_ARG;
    if (!lo->graph_ready || !hi->graph_ready) return MM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t F = 3 * (size_t)hi->g.N * sizeof(double);
    const bool mdev = mm_is_device_ptr(m);
    int rc;
    if ((rc = ensure_records(lo, n)) || (rc = ensure_records(hi, n))) return rc;
    if ((rc = mm_load_iterate(hi, m, mdev, s))) return rc;
    // the double problem's current iterate is now buffer 0 (base 0, k 0)
    if ((rc = mm_launch_init_state(hi, H_list + 3 * start, opts_hi, 1, s))) return rc;
    for (int j = start; j < n; ++j) {
        if ((rc = transfer(hi, lo, s)) || (rc = mm_launch_init_state(lo, H_list + 3 * j, opts_lo, 1, s))) return rc;
        if ((rc = mm_launch_loop(lo, s))) return rc;
        if ((rc = mm_launch_record(lo, j, s))) return rc;
        if ((rc = transfer(lo, hi, s)) || (rc = mm_launch_init_state(hi, H_list + 3 * j, opts_hi, 1, s))) return rc;
        if ((rc = mm_launch_loop(hi, s))) return rc;
        if ((rc = mm_launch_record(hi, j, s))) return rc;
    }
    if ((rc = mm_launch_copy_result(hi, mdev ? m : hi->stage_out, s))) return rc;
    if (!mdev && (rc = mm_copy_user(m, hi->stage_out, F, false, true, s))) return rc;
    std::vector<StepRecord> rl, rh;
    if ((rc = read_records(lo, n, start, rl, s)) || (rc = read_records(hi, n, start, rh, s))) return rc;
    int first_bad = MM_OK;
    for (int j = start; j < n; ++j) {
        const StepRecord &r = rh[j];
        for (int c = 0; c < 3; ++c) mavg[3 * j + c] = r.mavg[c];
        const int st = status_of_rec(r.status);
        if (st != MM_OK && first_bad == MM_OK) first_bad = st;
        if (per_step_lo) fill_result(rl[j], per_step_lo[j], 3);  // transfer, init, record
        if (per_step_hi) fill_result(rh[j], per_step_hi[j], 3);
    }
    return first_bad;
}
