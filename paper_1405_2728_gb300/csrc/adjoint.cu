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
// The CG loop itself runs on the device (a conditional WHILE graph node).
#include <cmath>
#include <vector>

#include "common.cuh"

namespace {

constexpr int DOT_THREADS = 256;

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

// ---------------------------------------------------------------------------
// Conjugate gradients on the device.  One graph launch runs the whole solve:
// a conditional WHILE node whose body is one product A p (a field evaluation
// of p through the FFT kernels, then k_hvp_dot) and the CG updates.  The
// scalars live in CgState; one-CTA kernels sum the per-CTA partial dot
// products in a fixed order (deterministic), pick alpha and beta, apply the
// stop rule and set the loop condition, so the host waits once per solve.
// ---------------------------------------------------------------------------
enum { CG_RUNNING = 0, CG_CONVERGED = 1, CG_MAXITER = 2, CG_NOTPOS = 3 };

struct CgState {
    double rr, bb, pAp, alpha, beta, tol2;
    long it, max_iter;
    int status;
};

// one CTA: sum of n partials in a fixed order (thread t takes t, t + 256, ...,
// then a tree over the threads)
__device__ double block_sum_fixed(const double *partials, int n)
{
    __shared__ double sh[DOT_THREADS];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += DOT_THREADS) acc += __ldcg(partials + i);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = DOT_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    return sh[0];
}

// per-CTA partial of a.b (grid-stride, fixed grid: deterministic)
template <typename T>
__device__ void block_dot_store(double acc, double *partials)
{
    __shared__ double sh[DOT_THREADS];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = DOT_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// r.r of the start residual; the solve starts unless it is already below tol
__global__ void __launch_bounds__(DOT_THREADS) k_cg_start(CgState *st, const double *partials, int n, double tol2,
                                                          long max_iter)
{
    const double rr = block_sum_fixed(partials, n);
    if (threadIdx.x != 0) return;
    st->rr = rr; st->bb = rr; st->tol2 = tol2; st->it = 0; st->max_iter = max_iter;
    st->alpha = 0.0; st->beta = 0.0; st->pAp = 0.0;
    st->status = (!(rr > 0.0) || rr <= tol2 * rr) ? CG_CONVERGED : (max_iter < 1 ? CG_MAXITER : CG_RUNNING);
}

// Ap = P_m((m.H) p - Lp) (see k_hvp) and the CTA's partial of p.Ap
template <typename T>
__global__ void __launch_bounds__(DOT_THREADS) k_hvp_dot(const T *m, const T *H, const T *v, const T *Lv, T *Av,
                                                         long N, double *partials, const CgState *st)
{
    double acc = 0.0;
    if (st->status == CG_RUNNING) {
        for (long i = blockIdx.x * (long)DOT_THREADS + threadIdx.x; i < N; i += (long)gridDim.x * DOT_THREADS) {
            const T m0 = m[i], m1 = m[N + i], m2 = m[2 * N + i];
            const T mh = m0 * H[i] + m1 * H[N + i] + m2 * H[2 * N + i];
            const T t0 = mh * v[i] - Lv[i], t1 = mh * v[N + i] - Lv[N + i], t2 = mh * v[2 * N + i] - Lv[2 * N + i];
            const T mt = m0 * t0 + m1 * t1 + m2 * t2;
            const T a0 = t0 - mt * m0, a1 = t1 - mt * m1, a2 = t2 - mt * m2;
            Av[i] = a0; Av[N + i] = a1; Av[2 * N + i] = a2;
            acc += (double)v[i] * (double)a0 + (double)v[N + i] * (double)a1 + (double)v[2 * N + i] * (double)a2;
        }
    }
    block_dot_store<T>(acc, partials);
}

// alpha = r.r / p.Ap; a non-positive p.Ap means m is not a minimum
__global__ void __launch_bounds__(DOT_THREADS) k_cg_alpha(CgState *st, const double *partials, int n,
                                                          cudaGraphConditionalHandle h)
{
    const double pAp = block_sum_fixed(partials, n);
    if (threadIdx.x != 0) return;
    if (st->status != CG_RUNNING) { cudaGraphSetConditional(h, 0u); return; }
    st->pAp = pAp;
    if (!(isfinite(pAp) && pAp > 0.0)) {
        st->status = CG_NOTPOS;
        st->alpha = 0.0;
        cudaGraphSetConditional(h, 0u);
        return;
    }
    st->alpha = st->rr / pAp;
}

// x += alpha p; r -= alpha Ap; the CTA's partial of r.r
template <typename T>
__global__ void __launch_bounds__(DOT_THREADS) k_cg_update_dot(T *x, T *r, const T *p, const T *Ap, long n,
                                                               double *partials, const CgState *st)
{
    double acc = 0.0;
    if (st->status == CG_RUNNING) {
        const T a = (T)st->alpha;
        for (long i = blockIdx.x * (long)DOT_THREADS + threadIdx.x; i < n; i += (long)gridDim.x * DOT_THREADS) {
            x[i] += a * p[i];
            const T ri = r[i] - a * Ap[i];
            r[i] = ri;
            acc += (double)ri * (double)ri;
        }
    }
    block_dot_store<T>(acc, partials);
}

// beta = r.r(new) / r.r(old); stop rule |r| <= tol |b| or the iteration cap
__global__ void __launch_bounds__(DOT_THREADS) k_cg_beta(CgState *st, const double *partials, int n,
                                                         cudaGraphConditionalHandle h)
{
    const double rr_new = block_sum_fixed(partials, n);
    if (threadIdx.x != 0) return;
    if (st->status != CG_RUNNING) { cudaGraphSetConditional(h, 0u); return; }
    st->it += 1;
    st->beta = rr_new / st->rr;
    st->rr = rr_new;
    unsigned go = 1u;
    if (rr_new <= st->tol2 * st->bb) { st->status = CG_CONVERGED; go = 0u; }
    else if (st->it >= st->max_iter) { st->status = CG_MAXITER; go = 0u; }
    cudaGraphSetConditional(h, go);
}

// p = r + beta p (only while the solve continues)
template <typename T>
__global__ void k_xpay_dev(T *p, const T *r, long n, const CgState *st)
{
    if (st->status != CG_RUNNING) return;
    const T b = (T)st->beta;
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

// r.r partials of a vector (start residual)
template <typename T>
__global__ void __launch_bounds__(DOT_THREADS) k_dot_self(const T *r, long n, double *partials)
{
    double acc = 0.0;
    for (long i = blockIdx.x * (long)DOT_THREADS + threadIdx.x; i < n; i += (long)gridDim.x * DOT_THREADS)
        acc += (double)r[i] * (double)r[i];
    block_dot_store<T>(acc, partials);
}

int grid_for(long n) { return mm_grid_for(n, 256, 8); }

int ensure_adjoint_buffers(mm_problem *p)
{
    const size_t F = 3 * (size_t)p->g.N * p->esz;
    for (int i = 0; i < 2; ++i) {
        if (p->adj[i]) continue;
        cudaError_t e = cudaMalloc(&p->adj[i], F);
        if (e) { p->adj[i] = nullptr; mm_set_cuda_error(e, "cudaMalloc(adjoint)"); return MM_ERR_OOM; }
        p->bytes += (long)F;
    }
    if (!p->adj_state) {
        p->adj_nblk = mm_sm_count() * 4;
        cudaError_t e = cudaMalloc(&p->adj_state, sizeof(CgState));
        if (!e) e = cudaMalloc((void **)&p->adj_partials, sizeof(double) * p->adj_nblk);
        if (e) { mm_set_cuda_error(e, "cudaMalloc(adjoint state)"); return MM_ERR_OOM; }
        p->bytes += (long)(sizeof(CgState) + sizeof(double) * p->adj_nblk);
    }
    return MM_OK;
}

bool vec3_ok(const double *h) { return h && std::isfinite(h[0]) && std::isfinite(h[1]) && std::isfinite(h[2]); }

// Field buffers used by the adjoint: mbuf[0] = m, mbuf[1] = H(m), gbuf[0] = x,
// gbuf[1] = r, stage_in = p, stage_out = L p, adj[0] = A p, adj[1] = dJ/dm.
template <typename T>
cudaError_t capture_cg_body(mm_problem *p, cudaStream_t cs)
{
    const long N = p->g.N, n3 = 3 * N;
    T *mm_ = (T *)p->mbuf[0], *H = (T *)p->mbuf[1], *x = (T *)p->gbuf[0], *r = (T *)p->gbuf[1];
    T *pp = (T *)p->stage_in, *Lp = (T *)p->stage_out, *Ap = (T *)p->adj[0];
    CgState *st = (CgState *)p->adj_state;
    const double zero[3] = {0.0, 0.0, 0.0};
    if (mm_launch_field(p, pp, Lp, zero, MODE_HEFF, cs)) return cudaErrorUnknown;
    k_hvp_dot<T><<<p->adj_nblk, DOT_THREADS, 0, cs>>>(mm_, H, pp, Lp, Ap, N, p->adj_partials, st);
    k_cg_alpha<<<1, DOT_THREADS, 0, cs>>>(st, p->adj_partials, p->adj_nblk, p->adj_cond);
    k_cg_update_dot<T><<<p->adj_nblk, DOT_THREADS, 0, cs>>>(x, r, pp, Ap, n3, p->adj_partials, st);
    k_cg_beta<<<1, DOT_THREADS, 0, cs>>>(st, p->adj_partials, p->adj_nblk, p->adj_cond);
    k_xpay_dev<T><<<grid_for(n3), 256, 0, cs>>>(pp, r, n3, st);
    return cudaGetLastError();
}

template <typename T>
int build_cg_graph(mm_problem *p)
{
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e) { mm_set_cuda_error(e, "cudaStreamCreate"); return MM_ERR_CUDA; }
    int rc = MM_OK;
    do {
        if ((e = cudaGraphCreate(&p->adj_graph, 0))) break;
        if ((e = cudaGraphConditionalHandleCreate(&p->adj_cond, p->adj_graph, 1, cudaGraphCondAssignDefault))) break;
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = p->adj_cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        if ((e = cudaGraphAddNode(&node, p->adj_graph, nullptr, nullptr, 0, &np))) break;
        cudaGraph_t body = np.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed))) break;
        const cudaError_t le = capture_cg_body<T>(p, cs);
        cudaGraph_t out = body;
        e = cudaStreamEndCapture(cs, &out);
        if (le) { e = le; break; }
        if (e) break;
        if ((e = cudaGraphInstantiate(&p->adj_exec, p->adj_graph, 0))) break;
    } while (0);
    if (e) { mm_set_cuda_error(e, "adjoint graph"); rc = MM_ERR_CUDA; mm_adjoint_invalidate(p); }
    cudaStreamDestroy(cs);
    return rc;
}

template <typename T>
int adjoint_t(mm_problem *p, const void *m, const double Hext[3], const void *dJdm, double *dJdK, double tol,
              long max_iter, long *iters, double *resid, cudaStream_t s)
{
    const long N = p->g.N, n3 = 3 * N;
    const size_t F = 3 * (size_t)N * sizeof(T);
    int rc;
    if ((rc = ensure_adjoint_buffers(p))) return rc;
    if (!p->adj_exec && (rc = build_cg_graph<T>(p))) return rc;
    T *mm_ = (T *)p->mbuf[0], *H = (T *)p->mbuf[1], *x = (T *)p->gbuf[0], *r = (T *)p->gbuf[1];
    T *pp = (T *)p->stage_in, *tmp = (T *)p->adj[1];
    CgState *st = (CgState *)p->adj_state;
    if ((rc = mm_copy_user(mm_, m, F, true, mm_is_device_ptr(m), s))) return rc;
    if ((rc = mm_copy_user(tmp, dJdm, F, true, mm_is_device_ptr(dJdm), s))) return rc;
    if ((rc = mm_launch_field(p, mm_, H, Hext, MODE_HEFF, s))) return rc;
    const int gN = grid_for(N);
    cudaError_t e;
    k_project<T><<<gN, 256, 0, s>>>(mm_, tmp, r, N);      // r = b = P(dJ/dm), x = 0, p = r
    if ((e = cudaMemsetAsync(x, 0, F, s)) || (e = cudaMemcpyAsync(pp, r, F, cudaMemcpyDeviceToDevice, s))) {
        mm_set_cuda_error(e, "adjoint");
        return MM_ERR_CUDA;
    }
    k_dot_self<T><<<p->adj_nblk, DOT_THREADS, 0, s>>>(r, n3, p->adj_partials);
    k_cg_start<<<1, DOT_THREADS, 0, s>>>(st, p->adj_partials, p->adj_nblk, tol * tol, max_iter);
    if ((e = cudaGetLastError())) { mm_set_cuda_error(e, "adjoint start"); return MM_ERR_CUDA; }
    if ((e = cudaGraphLaunch(p->adj_exec, s))) { mm_set_cuda_error(e, "adjoint graph launch"); return MM_ERR_CUDA; }
    // dJ/dK into a device double buffer, then to the caller
    const bool odev = mm_is_device_ptr(dJdK);
    double *out = odev ? dJdK : (double *)tmp;  // tmp holds >= N doubles (3N elements of T >= 4 bytes)
    k_dJdK<T><<<gN, 256, 0, s>>>(mm_, x, (const T *)p->uc, p->g.u[0], p->g.u[1], p->g.u[2], p->g.can, out, N);
    if (!odev && (rc = mm_copy_user(dJdK, out, sizeof(double) * N, false, true, s))) return rc;
    CgState hs;
    if ((e = cudaGetLastError()) || (e = cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s))) {
        mm_set_cuda_error(e, "adjoint");
        return MM_ERR_CUDA;
    }
    if (iters) *iters = hs.it;
    if (resid) *resid = hs.bb > 0 ? std::sqrt(hs.rr / hs.bb) : 0.0;
    switch (hs.status) {
    case CG_CONVERGED: return MM_OK;
    case CG_MAXITER: return MM_ERR_NOT_CONVERGED;
    case CG_NOTPOS: return MM_ERR_NONFINITE;
    }
    return MM_ERR_CUDA;
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
    return mm_double_fields(p) ? hvp_t<double>(p, m, Hext, v, Av, (cudaStream_t)stream)
                                   : hvp_t<float>(p, m, Hext, v, Av, (cudaStream_t)stream);
}

extern "C" MM_API int mm_adjoint_dK(mm_problem *p, const void *m, const double Hext[3], const void *dJdm,
                                    double *dJdK, double tol, long max_iter, long *iters, double *resid,
                                    void *stream)
{
    if (!p || !m || !dJdm || !dJdK || !vec3_ok(Hext) || !(tol > 0) || max_iter < 1) return MM_ERR_ARG;
    return mm_double_fields(p)
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
    if (mm_double_fields(p)) {
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
    // the loop graphs bake the per-cell pointer in: recapture them once
    if (fresh) {
        mm_adjoint_invalidate(p);
        return mm_rebuild_graph(p);
    }
    return MM_OK;
}

void mm_adjoint_invalidate(mm_problem *p)
{
    if (p->adj_exec) { cudaGraphExecDestroy(p->adj_exec); p->adj_exec = nullptr; }
    if (p->adj_graph) { cudaGraphDestroy(p->adj_graph); p->adj_graph = nullptr; }
}
