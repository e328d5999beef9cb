// Effective-field and minimiser-step kernels (sm_103a).
//
// One evaluation of H_eff (Eq. effective_field; Sections 3 and 4) is three
// kernels over the zero-padded grid for films (bulk grids replace k_yz by
// the three passes of bulk.cu); in the minimiser (Section 2) the last of
// them also finishes the iteration:
//
//  k_xfwd     per (z, tile of TYF rows): optional minimiser step (the closed
//             form of the midpoint scheme, Eq. implicit_gradient_descent, or
//             the renormalised explicit step) fused with the real-to-complex
//             FFT along x of the three components, zero padding nx -> Px,
//             written transposed to the spectrum W[kx][z][y][c].
//  k_yz       per x-frequency kx: FFT along y (padding ny -> Py) in shared
//             memory; then per ky, in registers, the z direction as a direct
//             convolution with the tensor transformed along x and y
//             (H^ = -Ms N m^, nz <= 4, normalisation folded into the tensor);
//             then the inverse FFT along y keeping the first ny rows.
//  k_xinv     per (z, tile of TY rows): complex-to-real inverse FFT along x keeping nx
//             values, then the local terms: exchange (six-point stencil, free
//             faces), uniaxial anisotropy, Zeeman.  Depending on the mode it
//             writes H, or accumulates the energy terms, or forms the projected
//             gradient g = m x (m x H) (Eq. projected_direction) with the
//             Barzilai-Borwein sums s.s, s.y, y.y (Eq. stepsize), max |m x H|,
//             the energy and sum m.  Each CTA stores its partial sums; the last
//             CTA to finish sums them in a fixed order (deterministic), picks
//             the step size tau^1 / tau^2 alternately (Eq. stepsize), applies
//             the stop rule and sets the device-side loop condition.
//
// Sums are accumulated in double on the double path.  On the float path each
// per-cell product enters its sum exactly (TwoProduct with one FMA) and the
// sums are compensated float pairs (TwoSum, Knuth), about 46 significant
// bits; the double-word path (MM_F32X2) sums in double-word arithmetic.
// Partial sums are always combined across CTAs in double.
#include <cstdio>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "fft.cuh"
#include "field_kernels.cuh"

namespace {

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
__global__ void k_init_state(MinState *st, double tau0, double tol_abs, double h0, double h1, double h2,
                             long max_iter, int step_kind, unsigned long long timeout_ns, int reset_base,
                             int tau_rule, double kappa)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (reset_base) st->base = 0;
    else st->base = st->base ^ (int)(st->k & 1);   // continue from the previous result
    st->tau0 = tau0; st->tol_abs = tol_abs;
    st->Hext[0] = h0; st->Hext[1] = h1; st->Hext[2] = h2;
    st->Hextf[0] = (float)h0; st->Hextf[1] = (float)h1; st->Hextf[2] = (float)h2;
    st->Hextw[0] = dfloat(h0); st->Hextw[1] = dfloat(h1); st->Hextw[2] = dfloat(h2);
    st->max_iter = max_iter; st->step_kind = step_kind;
    st->tau_rule = tau_rule; st->kappa = kappa;
    st->timeout_ns = timeout_ns; st->t_start_ns = 0;
    st->k = 0; st->tau = tau0; st->tauf = (float)tau0; st->tauw = dfloat(tau0); st->status = MMS_RUNNING; st->evals = 0; st->launches = 1;
    st->max_torque = 0;
}

__global__ void k_record(const MinState *st, StepRecord *rec, int step)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    StepRecord r;
    r.mavg[0] = st->mavg[0]; r.mavg[1] = st->mavg[1]; r.mavg[2] = st->mavg[2];
    r.max_torque = st->max_torque; r.energy = st->energy[4];
    r.iters = st->k; r.evals = st->evals; r.launches = st->launches + 1; r.status = st->status;
    rec[step] = r;
}

// the current iterate, in the caller's element type
template <typename T>
__global__ void k_copy_result(const MinState *st, const T *b0, const T *b1, typename io_of<T>::type *dst, long n3)
{
    const T *src = (st->base ^ (int)(st->k & 1)) ? b1 : b0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n3; i += (long)gridDim.x * blockDim.x)
        dst[i] = to_io(src[i]);
}

// double-word fields to the caller's double
__global__ void k_dfloat_to_double(double *dst, const dfloat *src, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = df_to_double(src[i]);
}

template <typename T>
__global__ void k_twiddle(typename cvec<T>::type *tw, int L)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= L) return;
    double s, c;
    sincospi(2.0 * (double)t / (double)L, &s, &c);
    typename cvec<T>::type w;
    w.x = (T)c; w.y = (T)(-s);
    tw[t] = w;
}

template <typename T>
__global__ void k_convert(T *dst, const double *src, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

} // namespace

// ---------------------------------------------------------------------------
// exported to api.cu
// ---------------------------------------------------------------------------
// the three precisions: (field type, FFT arithmetic)
#define DISPATCH3(p, fn, args) \
    ((p)->precision == MM_FP64 ? mm_fields_##fn##_fp64 args \
                               : ((p)->precision == MM_FP32 ? mm_fields_##fn##_fp32 args : mm_fields_##fn##_f32x2 args))
#define DISPATCH(p, expr_d, expr_f) (mm_double_fields(p) ? (expr_d) : (expr_f))


// Shared-memory needs of a launch shape (bytes), for the planner.
size_t mm_smem_x_for(const mm_problem *p, int ty)
{
    Geom g = p->g;
    g.TY = ty;
    return DISPATCH(p, smem_x_t<double>(g), smem_x_t<float>(g));
}
size_t mm_smem_yz_for(const mm_problem *p)
{
    return DISPATCH(p, smem_yz_t<double>(p->g), smem_yz_t<float>(p->g));
}
int mm_yz_thread_bound(const mm_problem *p) { return DISPATCH(p, YZBound<double>::v, YZBound<float>::v); }

int mm_heff_configure(mm_problem *p)
{
    // limits for the largest admissible tile (shared memory grows with it)
    Geom g = p->g;
    g.TY = g.TYF = p->tys[p->nty - 1];
    const size_t sx = DISPATCH(p, smem_x_t<double>(g), smem_x_t<float>(g));
    const size_t sxf = DISPATCH(p, smem_xf_t<double>(g), smem_xf_t<float>(g));
    const size_t syz = p->g.bulk ? 0 : mm_smem_yz_for(p);
    cudaError_t e = DISPATCH3(p, configure, (g, sxf, sx, syz));
    if (!e && p->g.bulk) e = mm_bulk_configure(p);
    if (e) { mm_set_cuda_error(e, "cudaFuncSetAttribute"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_autotune(mm_problem *p, const int *tys, int nty, const int *rbs, int nrb, cudaStream_t s)
{
    cudaError_t e = DISPATCH3(p, autotune, (p, tys, nty, rbs, nrb, s));
    if (e) { mm_set_cuda_error(e, "autotune"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_field(mm_problem *p, const void *m, void *H, const double *hext, int mode, cudaStream_t s,
                    double hscale)
{
    cudaError_t e = DISPATCH3(p, chain, (p, m, H, hext, mode, s, hscale));
    if (e) { mm_set_cuda_error(e, "field kernels"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_min_body(mm_problem *p, cudaGraphConditionalHandle h, cudaStream_t s, int use_cond)
{
    cudaError_t e = DISPATCH3(p, min_body, (p, h, s, use_cond));
    if (e) { mm_set_cuda_error(e, "minimiser body"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_kernel_stage_times(mm_problem *p, int reps, double *ms, const char **names, int *count, cudaStream_t s)
{
    static const char *film[3] = {"xfwd_step", "yz_conv", "xinv_local_bb"};
    static const char *bulk[5] = {"xfwd_step", "y_fwd", "z_conv", "y_inv", "xinv_local_bb"};
    const int nst = p->g.bulk ? 5 : 3;
    if (*count < nst) return MM_ERR_ARG;
    cudaError_t e = DISPATCH3(p, stage_times, (p, reps, ms, s));
    if (e) { mm_set_cuda_error(e, "stage timing"); return MM_ERR_CUDA; }
    for (int i = 0; i < nst; ++i) names[i] = p->g.bulk ? bulk[i] : film[i];
    *count = nst;
    return MM_OK;
}

int mm_launch_loop(mm_problem *p, cudaStream_t s)
{
    const cudaError_t e = cudaGraphLaunch(p->gexec, s);
    if (e) { mm_set_cuda_error(e, "cudaGraphLaunch"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_init_state(mm_problem *p, const double Hext[3], const mm_min_opts *o, int reset_base, cudaStream_t s)
{
    double tau0 = o->tau0 > 0 ? o->tau0 : 1e-2 / p->g.Ms;
    unsigned long long to = o->timeout_s > 0 ? (unsigned long long)(o->timeout_s * 1e9) : 0ull;
    const double kappa = o->tau_kappa > 0 ? o->tau_kappa : 0.5;
    k_init_state<<<1, 32, 0, s>>>(p->st, tau0, o->tol * p->g.Ms, Hext[0], Hext[1], Hext[2], o->max_iter,
                                  o->step_kind, to, reset_base, o->tau_rule, kappa);
    cudaError_t e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "k_init_state"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_record(mm_problem *p, int step, cudaStream_t s)
{
    k_record<<<1, 32, 0, s>>>(p->st, p->rec_dev, step);
    cudaError_t e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "k_record"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_copy_result(mm_problem *p, void *dst, cudaStream_t s)
{
    const long n3 = 3 * p->g.N;
    const int blocks = mm_grid_for(n3, 256, 8);
    if (p->precision == MM_F32X2)
        k_copy_result<dfloat><<<blocks, 256, 0, s>>>(p->st, (const dfloat *)p->mbuf[0],
                                                    (const dfloat *)p->mbuf[1], (double *)dst, n3);
    else if (p->precision == MM_FP64)
        k_copy_result<double><<<blocks, 256, 0, s>>>(p->st, (const double *)p->mbuf[0],
                                                    (const double *)p->mbuf[1], (double *)dst, n3);
    else
        k_copy_result<float><<<blocks, 256, 0, s>>>(p->st, (const float *)p->mbuf[0],
                                                   (const float *)p->mbuf[1], (float *)dst, n3);
    cudaError_t e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "k_copy_result"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_twiddles(mm_problem *p, cudaStream_t s)
{
    const Geom &g = p->g;
    const int L[3] = {g.Px, g.Py, g.Pz};
    void *dst[3] = {p->tw_px, p->tw_py, p->tw_pz};
    for (int i = 0; i < 3; ++i) {
        const int blocks = (L[i] + 255) / 256;
        if (p->precision == MM_F32X2) k_twiddle<dfloat><<<blocks, 256, 0, s>>>((dcomplex *)dst[i], L[i]);
        else if (p->precision == MM_FP64) k_twiddle<double><<<blocks, 256, 0, s>>>((double2 *)dst[i], L[i]);
        else k_twiddle<float><<<blocks, 256, 0, s>>>((float2 *)dst[i], L[i]);
    }
    cudaError_t e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "k_twiddle"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_iterate_in(mm_problem *p, void *dst, const double *src, long n, cudaStream_t s)
{
    if (p->precision != MM_F32X2) return MM_ERR_ARG;   // the other precisions store the caller's type
    k_convert<dfloat><<<mm_grid_for(n, 256, 8), 256, 0, s>>>((dfloat *)dst, src, n);
    cudaError_t e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "k_convert"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_iterate_out(mm_problem *p, double *dst, const void *src, long n, cudaStream_t s)
{
    if (p->precision != MM_F32X2) return MM_ERR_ARG;
    k_dfloat_to_double<<<mm_grid_for(n, 256, 8), 256, 0, s>>>(dst, (const dfloat *)src, n);
    cudaError_t e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "k_dfloat_to_double"); return MM_ERR_CUDA; }
    return MM_OK;
}

int mm_launch_convert(mm_problem *p, void *dst, const double *src, long n, cudaStream_t s)
{
    const int blocks = mm_grid_for(n, 256, 8);
    if (mm_double_fields(p)) k_convert<double><<<blocks, 256, 0, s>>>((double *)dst, src, n);
    else k_convert<float><<<blocks, 256, 0, s>>>((float *)dst, src, n);
    cudaError_t e = cudaGetLastError();
    if (e) { mm_set_cuda_error(e, "k_convert"); return MM_ERR_CUDA; }
    return MM_OK;
}
