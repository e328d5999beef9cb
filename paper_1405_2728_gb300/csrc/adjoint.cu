// Differentiation of the minimiser's result (an extension; the paper has no
// counterpart): the energy gradient dU/dm = -mu0 Ms V H_eff for automatic
// differentiation, and the implicit adjoint of a converged minimum.
//
// At a minimum the torque vanishes, P_m H(m; K) = 0 with P_m w = w - (m.w) m.
// Differentiating with respect to the per-cell anisotropy K gives
//   A dm = P_m(dH/dK) dK,   A v = (m.H) v - P_m(L v),
// where L v = H_eff(v) without the external field (every other term of H_eff
// is linear in m).  A is symmetric on tangent fields and positive definite at
// a stable minimum, so for an objective J(m), dJ/dK_i = lambda . P_m(dH/dK_i)
// with A lambda = P_m(dJ/dm), solved by conjugate gradients.  Each product A v
// is one field evaluation of v through the FFT kernels plus a fused per-cell
// kernel; inner products are deterministic two-stage reductions in double.
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

constexpr int DOT_THREADS = 256;
constexpr int DOT_BLOCKS = 152 * 4;

template <typename T>
__global__ void __launch_bounds__(DOT_THREADS) k_dot(const T *a, const T *b, long n, double *partials)
{
    __shared__ double sh[DOT_THREADS];
    double acc = 0.0;
    for (long i = blockIdx.x * (long)DOT_THREADS + threadIdx.x; i < n; i += (long)gridDim.x * DOT_THREADS)
        acc += (double)a[i] * (double)b[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = DOT_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(DOT_THREADS) k_sum(const double *partials, int n, double *out)
{
    __shared__ double sh[DOT_THREADS];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += DOT_THREADS) acc += partials[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = DOT_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// Av = P_m((m.H) v - Lv), equal to (m.H) v - P_m(Lv) for tangent v.  The
// outer projection removes normal components that rounding leaves in the CG
// vectors; unprojected they are multiplied by m.H (down to -0.4 Ms near the
// ends of a film) at every product and eventually destroy positivity.
template <typename T>
__global__ void k_hvp(const T *m, const T *H, const T *v, const T *Lv, T *Av, long N)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const T m0 = m[i], m1 = m[N + i], m2 = m[2 * N + i];
        const T mh = m0 * H[i] + m1 * H[N + i] + m2 * H[2 * N + i];
        const T t0 = mh * v[i] - Lv[i], t1 = mh * v[N + i] - Lv[N + i], t2 = mh * v[2 * N + i] - Lv[2 * N + i];
        const T mt = m0 * t0 + m1 * t1 + m2 * t2;
        Av[i] = t0 - mt * m0;
        Av[N + i] = t1 - mt * m1;
        Av[2 * N + i] = t2 - mt * m2;
    }
}

// out = P_m(w)
template <typename T>
__global__ void k_project(const T *m, const T *w, T *out, long N)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const T m0 = m[i], m1 = m[N + i], m2 = m[2 * N + i];
        const T mw = m0 * w[i] + m1 * w[N + i] + m2 * w[2 * N + i];
        out[i] = w[i] - mw * m0;
        out[N + i] = w[N + i] - mw * m1;
        out[2 * N + i] = w[2 * N + i] - mw * m2;
    }
}

// x += alpha p; r -= alpha Ap
template <typename T>
__global__ void k_cg_update(T *x, T *r, const T *p, const T *Ap, double alpha, long n)
{
    const T a = (T)alpha;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        x[i] += a * p[i];
        r[i] -= a * Ap[i];
    }
}

// p = r + beta p
template <typename T>
__global__ void k_xpay(T *p, const T *r, double beta, long n)
{
    const T b = (T)beta;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        p[i] = r[i] + b * p[i];
}

// dJ/dK_i = lam_i . P_m(dH_i/dK_i), dH_i/dK_i = coef (m_i.u_i) u_i, coef = 2/(mu0 Ms)
template <typename T>
__global__ void k_dJdK(const T *m, const T *lam, const T *uc, double u0, double u1, double u2, double coef,
                       double *out, long N)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const double m0 = m[i], m1 = m[N + i], m2 = m[2 * N + i];
        double a0 = u0, a1 = u1, a2 = u2;
        if (uc) { a0 = uc[i]; a1 = uc[N + i]; a2 = uc[2 * N + i]; }
        const double mu = m0 * a0 + m1 * a1 + m2 * a2;
        // P_m(u) = u - (m.u) m
        const double p0 = a0 - mu * m0, p1 = a1 - mu * m1, p2 = a2 - mu * m2;
        out[i] = coef * mu * ((double)lam[i] * p0 + (double)lam[N + i] * p1 + (double)lam[2 * N + i] * p2);
    }
}

int grid_for(long n) { return mm_grid_for(n, 256, 8); }

struct Scratch {
    double *partials = nullptr, *scalars = nullptr, *scalars_host = nullptr;
    ~Scratch()
    {
        if (partials) cudaFree(partials);
        if (scalars) cudaFree(scalars);
        if (scalars_host) cudaFreeHost(scalars_host);
    }
    int init()
    {
        if (cudaMalloc((void **)&partials, sizeof(double) * DOT_BLOCKS) ||
            cudaMalloc((void **)&scalars, sizeof(double) * 4) ||
            cudaMallocHost((void **)&scalars_host, sizeof(double) * 4)) {
            cudaGetLastError();
            return MM_ERR_OOM;
        }
        return MM_OK;
    }
};

template <typename T>
cudaError_t dot_into(const T *a, const T *b, long n, Scratch &sc, int slot, cudaStream_t s)
{
    k_dot<T><<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(a, b, n, sc.partials);
    k_sum<<<1, DOT_THREADS, 0, s>>>(sc.partials, DOT_BLOCKS, sc.scalars + slot);
    return cudaGetLastError();
}

int ensure_adjoint_buffers(mm_problem *p)
{
    const size_t F = 3 * (size_t)p->g.N * p->esz;
    for (int i = 0; i < 2; ++i) {
        if (p->adj[i]) continue;
        cudaError_t e = cudaMalloc(&p->adj[i], F);
        if (e) { p->adj[i] = nullptr; mm_set_cuda_error(e, "cudaMalloc(adjoint)"); return MM_ERR_OOM; }
        p->bytes += (long)F;
    }
    return MM_OK;
}

bool vec3_ok(const double *h) { return h && std::isfinite(h[0]) && std::isfinite(h[1]) && std::isfinite(h[2]); }

// Field buffers used by the adjoint: mbuf[0] = m, mbuf[1] = H(m), gbuf[0] = x,
// gbuf[1] = r, stage_in = p, stage_out = L p, adj[0] = A p, adj[1] = spare.
template <typename T>
int adjoint_t(mm_problem *p, const void *m, const double Hext[3], const void *dJdm, double *dJdK, double tol,
              long max_iter, long *iters, double *resid, cudaStream_t s)
{
    const long N = p->g.N, n3 = 3 * N;
    const size_t F = 3 * (size_t)N * sizeof(T);
    int rc;
    if ((rc = ensure_adjoint_buffers(p))) return rc;
    Scratch sc;
    if ((rc = sc.init())) return rc;
    T *mm_ = (T *)p->mbuf[0], *H = (T *)p->mbuf[1], *x = (T *)p->gbuf[0], *r = (T *)p->gbuf[1];
    T *pp = (T *)p->stage_in, *Lp = (T *)p->stage_out, *Ap = (T *)p->adj[0], *tmp = (T *)p->adj[1];
    if ((rc = mm_copy_user(mm_, m, F, true, mm_is_device_ptr(m), s))) return rc;
    if ((rc = mm_copy_user(tmp, dJdm, F, true, mm_is_device_ptr(dJdm), s))) return rc;
    const double zero[3] = {0.0, 0.0, 0.0};
    if ((rc = mm_launch_field(p, mm_, H, Hext, MODE_HEFF, s))) return rc;
    const int gN = grid_for(N), gn = grid_for(n3);
    k_project<T><<<gN, 256, 0, s>>>(mm_, tmp, r, N);      // r = b = P(dJ/dm), x = 0
    cudaMemsetAsync(x, 0, F, s);
    cudaMemcpyAsync(pp, r, F, cudaMemcpyDeviceToDevice, s);
    cudaError_t e;
    if ((e = dot_into(r, r, n3, sc, 0, s))) { mm_set_cuda_error(e, "adjoint"); return MM_ERR_CUDA; }
    cudaMemcpyAsync(sc.scalars_host, sc.scalars, sizeof(double), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s))) { mm_set_cuda_error(e, "adjoint"); return MM_ERR_CUDA; }
    double rr = sc.scalars_host[0];
    const double bb = rr;
    long it = 0;
    int status = MM_OK;
    while (rr > tol * tol * bb && rr > 0.0) {
        if (it >= max_iter) { status = MM_ERR_NOT_CONVERGED; break; }
        if ((rc = mm_launch_field(p, pp, Lp, zero, MODE_HEFF, s))) return rc;
        k_hvp<T><<<gN, 256, 0, s>>>(mm_, H, pp, Lp, Ap, N);
        if ((e = dot_into(pp, Ap, n3, sc, 1, s))) { mm_set_cuda_error(e, "adjoint"); return MM_ERR_CUDA; }
        cudaMemcpyAsync(sc.scalars_host + 1, sc.scalars + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s))) { mm_set_cuda_error(e, "adjoint"); return MM_ERR_CUDA; }
        const double pAp = sc.scalars_host[1];
        if (!(std::isfinite(pAp) && pAp > 0.0)) { status = MM_ERR_NONFINITE; break; }  // not a minimum
        const double alpha = rr / pAp;
        k_cg_update<T><<<gn, 256, 0, s>>>(x, r, pp, Ap, alpha, n3);
        if ((e = dot_into(r, r, n3, sc, 0, s))) { mm_set_cuda_error(e, "adjoint"); return MM_ERR_CUDA; }
        cudaMemcpyAsync(sc.scalars_host, sc.scalars, sizeof(double), cudaMemcpyDeviceToHost, s);
        if ((e = cudaStreamSynchronize(s))) { mm_set_cuda_error(e, "adjoint"); return MM_ERR_CUDA; }
        const double rr_new = sc.scalars_host[0];
        k_xpay<T><<<gn, 256, 0, s>>>(pp, r, rr_new / rr, n3);
        rr = rr_new;
        ++it;
    }
    if (iters) *iters = it;
    if (resid) *resid = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    // dJ/dK into a device double buffer, then to the caller
    const bool odev = mm_is_device_ptr(dJdK);
    double *out = odev ? dJdK : (double *)tmp;  // tmp holds >= N doubles (3N elements of T >= 4 bytes)
    k_dJdK<T><<<gN, 256, 0, s>>>(mm_, x, (const T *)p->uc, p->g.u[0], p->g.u[1], p->g.u[2], p->g.can, out, N);
    if (!odev && (rc = mm_copy_user(dJdK, out, sizeof(double) * N, false, true, s))) return rc;
    if ((e = cudaGetLastError()) || (e = cudaStreamSynchronize(s))) { mm_set_cuda_error(e, "adjoint"); return MM_ERR_CUDA; }
    return status;
}

template <typename T>
int hvp_t(mm_problem *p, const void *m, const double Hext[3], const void *v, void *Av, cudaStream_t s)
{
    const long N = p->g.N;
    const size_t F = 3 * (size_t)N * sizeof(T);
    int rc;
    if ((rc = ensure_adjoint_buffers(p))) return rc;
    T *mm_ = (T *)p->adj[0], *vv = (T *)p->adj[1], *H = (T *)p->stage_in, *Lv = (T *)p->stage_out;
    if ((rc = mm_copy_user(mm_, m, F, true, mm_is_device_ptr(m), s))) return rc;
    if ((rc = mm_copy_user(vv, v, F, true, mm_is_device_ptr(v), s))) return rc;
    const double zero[3] = {0.0, 0.0, 0.0};
    if ((rc = mm_launch_field(p, mm_, H, Hext, MODE_HEFF, s))) return rc;
    if ((rc = mm_launch_field(p, vv, Lv, zero, MODE_HEFF, s))) return rc;
    const bool odev = mm_is_device_ptr(Av);
    T *out = odev ? (T *)Av : (T *)p->mbuf[1];
    k_hvp<T><<<grid_for(N), 256, 0, s>>>(mm_, H, vv, Lv, out, N);
    if (!odev && (rc = mm_copy_user(Av, out, F, false, true, s))) return rc;
    cudaError_t e = cudaGetLastError();
    if (!e) e = cudaStreamSynchronize(s);
    if (e) { mm_set_cuda_error(e, "mm_hessian_vec"); return MM_ERR_CUDA; }
    return MM_OK;
}

} // namespace

extern "C" MM_API int mm_hessian_vec(mm_problem *p, const void *m, const double Hext[3], const void *v, void *Av,
                                     void *stream)
{
    if (!p || !m || !v || !Av || !vec3_ok(Hext)) return MM_ERR_ARG;
    return p->precision == MM_FP64 ? hvp_t<double>(p, m, Hext, v, Av, (cudaStream_t)stream)
                                   : hvp_t<float>(p, m, Hext, v, Av, (cudaStream_t)stream);
}

extern "C" MM_API int mm_adjoint_dK(mm_problem *p, const void *m, const double Hext[3], const void *dJdm,
                                    double *dJdK, double tol, long max_iter, long *iters, double *resid,
                                    void *stream)
{
    if (!p || !m || !dJdm || !dJdK || !vec3_ok(Hext) || !(tol > 0) || max_iter < 1) return MM_ERR_ARG;
    return p->precision == MM_FP64
               ? adjoint_t<double>(p, m, Hext, dJdm, dJdK, tol, max_iter, iters, resid, (cudaStream_t)stream)
               : adjoint_t<float>(p, m, Hext, dJdm, dJdK, tol, max_iter, iters, resid, (cudaStream_t)stream);
}

extern "C" MM_API int mm_energy_gradient(mm_problem *p, const void *m, const double Hext[3], double scale,
                                         void *G_out, void *stream)
{
    if (!p || !m || !G_out || !vec3_ok(Hext) || !std::isfinite(scale)) return MM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t F = 3 * (size_t)p->g.N * p->esz;
    const double V = p->g.dx * p->g.dy * p->g.dz;
    const double hs = -MM_MU0 * p->g.Ms * V * scale;  // dU/dm_i = -mu0 Ms V H_i
    const bool mdev = mm_is_device_ptr(m), gdev = mm_is_device_ptr(G_out);
    const void *msrc = m;
    int rc;
    if (!mdev) {
        if ((rc = mm_copy_user(p->stage_in, m, F, true, false, s))) return rc;
        msrc = p->stage_in;
    }
    void *dst = gdev ? G_out : p->stage_out;
    if ((rc = mm_launch_field(p, msrc, dst, Hext, MODE_HEFF, s, hs))) return rc;
    if (!gdev && (rc = mm_copy_user(G_out, dst, F, false, true, s))) return rc;
    if (!mdev || !gdev) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e) { mm_set_cuda_error(e, "mm_energy_gradient"); return MM_ERR_CUDA; }
    }
    return MM_OK;
}

extern "C" MM_API int mm_set_anisotropy(mm_problem *p, const double *K_cell, void *stream)
{
    if (!p || !K_cell) return MM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const long N = p->g.N;
    const bool fresh = (p->Kc == nullptr);
    if (fresh) {
        cudaError_t e = cudaMalloc(&p->Kc, (size_t)N * p->esz);
        if (e) { p->Kc = nullptr; mm_set_cuda_error(e, "cudaMalloc(K_cell)"); return MM_ERR_OOM; }
        p->bytes += (long)((size_t)N * p->esz);
    }
    double *tmp = nullptr;
    const bool kdev = mm_is_device_ptr(K_cell);
    if (p->precision == MM_FP64) {
        int rc = mm_copy_user(p->Kc, K_cell, sizeof(double) * N, true, kdev, s);
        if (rc) return rc;
    } else {
        if (cudaMalloc((void **)&tmp, sizeof(double) * N)) { cudaGetLastError(); return MM_ERR_OOM; }
        int rc = mm_copy_user(tmp, K_cell, sizeof(double) * N, true, kdev, s);
        if (!rc) rc = mm_launch_convert(p, p->Kc, tmp, N, s);
        cudaStreamSynchronize(s);
        cudaFree(tmp);
        if (rc) return rc;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e) { mm_set_cuda_error(e, "mm_set_anisotropy"); return MM_ERR_CUDA; }
    // the minimiser graph bakes the per-cell pointer in: recapture it once
    if (fresh) return mm_rebuild_graph(p);
    return MM_OK;
}
