// C ABI of libmmgb (include/mm.h): argument checking, memory ownership,
// setup of a problem (tensor spectrum, twiddles, per-cell material), the
// device-resident minimiser loop as a CUDA graph with a conditional WHILE
// node (Section 2 iterated on the device until the stop rule holds), and the
// hysteresis driver of Section 4.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"
#include "fft.cuh"
#include <nvtx3/nvToolsExt.h>

namespace {
// NVTX range around each entry point (a no-op unless a profiler is attached);
// lets profilers select e.g. the kernels of mm_kernel_times only.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
}


static thread_local char g_cuda_err[256] = "";

void mm_set_cuda_error(cudaError_t e, const char *where)
{
    snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
    cudaGetLastError();  // clear the sticky-free error slot of the runtime
}

extern "C" const char *mm_last_cuda_error(void) { return g_cuda_err; }

extern "C" const char *mm_status_string(int s)
{
    switch (s) {
    case MM_OK: return "ok";
    case MM_ERR_ARG: return "invalid argument";
    case MM_ERR_OOM: return "out of device memory";
    case MM_ERR_CUDA: return "CUDA runtime error";
    case MM_ERR_NOT_CONVERGED: return "not converged within max_iter";
    case MM_ERR_NONFINITE: return "non-finite value in the minimiser";
    case MM_ERR_TIMEOUT: return "minimiser wall-clock limit reached";
    case MM_ERR_UNSUPPORTED: return "grid outside what this build supports";
    }
    return "unknown status";
}

namespace {

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) {                        \
            mm_set_cuda_error(e_, what);                \
            return MM_ERR_CUDA;                         \
        }                                               \
    } while (0)

int next_pow2(int v) { int p = 1; while (p < v) p <<= 1; return p; }

// stored tensor: film layout C * max(1, Pz/2) * 6 * (Py/2+1), bulk layout C * (Pz/2+1) * (Py/2+1) * 6
size_t tensor_bytes(const Geom &g, size_t esz)
{
    return (g.bulk ? (size_t)g.C * (g.Pz / 2 + 1) * (g.Py / 2 + 1) * 6
                   : (size_t)g.C * (g.Pz > 1 ? g.Pz / 2 : 1) * 6 * (g.Py / 2 + 1)) * esz;
}
int ilog2i(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

bool grid_ok(const mm_grid *g)
{
    return g && g->nx >= 1 && g->ny >= 1 && g->nz >= 1 && std::isfinite(g->dx) && std::isfinite(g->dy) &&
           std::isfinite(g->dz) && g->dx > 0 && g->dy > 0 && g->dz > 0 &&
           (long)g->nx * g->ny * g->nz <= (1L << 31) / 3;
}

} // namespace

// Is ptr device-accessible memory (device or managed)?  Host memory
// (pageable or pinned) is staged.
bool mm_is_device_ptr(const void *ptr)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool mm_opts_ok(const mm_min_opts *o)
{
    return o && std::isfinite(o->tol) && o->tol >= 0 && std::isfinite(o->tau0) && o->max_iter >= 0 &&
           (o->step_kind == MM_STEP_CAYLEY || o->step_kind == MM_STEP_NORMALIZE) && std::isfinite(o->timeout_s) &&
           (o->tau_rule == MM_TAU_ALTERNATE || o->tau_rule == MM_TAU_ADAPTIVE) && std::isfinite(o->tau_kappa) &&
           o->tau_kappa <= 1.0;
}

int mm_sm_count()
{
    static int cached[256];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) { cudaGetLastError(); return 1; }
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
            cudaGetLastError();
            return 1;
        }
        cached[dev] = n;
    }
    return cached[dev];
}

int mm_grid_for(long n, int threads, int per_sm)
{
    const long want = (n + threads - 1) / threads;
    const long cap = (long)mm_sm_count() * per_sm;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

namespace {
#define is_device_ptr mm_is_device_ptr

int dalloc(mm_problem *p, void **ptr, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) { *ptr = nullptr; mm_set_cuda_error(e, "cudaMalloc"); return MM_ERR_OOM; }
    p->bytes += (long)bytes;
    return MM_OK;
}

void free_problem(mm_problem *p)
{
    if (!p) return;
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->graph) cudaGraphDestroy(p->graph);
    mm_adjoint_invalidate(p);
    void *bufs[] = {p->mbuf[0], p->mbuf[1], p->gbuf[0], p->gbuf[1], p->W, p->Nhat, p->tw_px, p->tw_py,
                    p->tw_pz, p->W2, p->Kc, p->uc, p->partials, p->st, p->Hext_dev, p->stage_in, p->stage_out,
                    p->rec_dev, p->counter, p->adj[0], p->adj[1], p->adj_state, p->adj_partials};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (p->st_host) cudaFreeHost(p->st_host);
    delete p;
}

// Geometry and launch shape; returns MM_ERR_UNSUPPORTED outside this build's envelope.
int plan(mm_problem *p)
{
    Geom &g = p->g;
    const mm_grid &gr = p->grid;
    g.nx = gr.nx; g.ny = gr.ny; g.nz = gr.nz;
    g.Px = next_pow2(2 * gr.nx - 1); if (g.Px < 2) g.Px = 2;
    g.Py = next_pow2(2 * gr.ny - 1);
    g.Pz = next_pow2(2 * gr.nz - 1);
    g.Hx = g.Px / 2; g.C = g.Hx + 1;
    g.lhx = ilog2i(g.Hx); g.lpy = ilog2i(g.Py);
    g.Gx = g.Hx >= 8 ? g.Hx / 8 : 1;
    g.Gy = g.Py >= 8 ? g.Py / 8 : 1;
    g.N = (long)gr.nx * gr.ny * gr.nz;
    g.dx = gr.dx; g.dy = gr.dy; g.dz = gr.dz;
    g.Ms = p->mat.Ms;
    const double c = 2.0 * p->mat.A / (MM_MU0 * p->mat.Ms);
    g.cex_x = c / (gr.dx * gr.dx); g.cex_y = c / (gr.dy * gr.dy); g.cex_z = c / (gr.dz * gr.dz);
    g.can = 2.0 / (MM_MU0 * p->mat.Ms);
    g.K = p->mat.K;
    g.u[0] = p->mat.u[0]; g.u[1] = p->mat.u[1]; g.u[2] = p->mat.u[2];
    g.fcex_x = (float)g.cex_x; g.fcex_y = (float)g.cex_y; g.fcex_z = (float)g.cex_z;
    g.fcan = (float)g.can; g.fK = (float)g.K;
    g.fu[0] = (float)g.u[0]; g.fu[1] = (float)g.u[1]; g.fu[2] = (float)g.u[2];
    g.wcex[0] = dfloat(g.cex_x); g.wcex[1] = dfloat(g.cex_y); g.wcex[2] = dfloat(g.cex_z);
    g.wcan = dfloat(g.can); g.wK = dfloat(g.K);
    for (int c = 0; c < 3; ++c) g.wu[c] = dfloat(g.u[c]);
    g.fd_nx.init(gr.nx); g.fd_ny.init(gr.ny);
    g.fd_padx.init(g.Px - gr.nx > 0 ? g.Px - gr.nx : 1);
    g.fd_pady.init(g.Py - gr.ny > 0 ? g.Py - gr.ny : 1);
    // the float x-inverse kernel stages its stencil rows with 16-byte copies
    g.stage = p->precision == MM_FP32 && gr.nx % 4 == 0;
    g.fd_nc.init(g.stage ? gr.nx / 4 : 1);
    if (g.Px > 4096 || g.Py > 4096 || g.Pz > 4096) return MM_ERR_UNSUPPORTED;
    // shared-memory row strides: double rows pad one element per 8, float rows
    // are XOR-swizzled within a stride of L+1 (fft.cuh)
    const int vsz = p->precision == MM_FP32 ? 8 : 16;  // bytes per complex element
    g.rsx = row_stride(g.Hx, vsz);
    g.rsy = row_stride(g.Py, vsz);
    g.rsz = row_stride(g.Pz, vsz);
    if (g.rsx <= g.Hx || g.rsy <= g.Py || g.rsz <= g.Pz) return MM_ERR_UNSUPPORTED;  // the kernels index rows with these strides
    g.lpz = ilog2i(g.Pz);
    g.Gz = g.Pz >= 8 ? g.Pz / 8 : 1;
    // admissible launch shapes; mm_autotune picks among them after setup
    const size_t smax = MM_SMEM_CAP;
    g.bulk = 0;
    p->nrb = 0;
    if (g.Pz <= 8) {
        // film layout: y rows per batch in the y-z kernel, divisors of 3 nz
        // with RB*Gy threads within the kernel's bound
        const int maxT = mm_yz_thread_bound(p), nrow = 3 * g.nz;
        for (int rb = nrow; rb >= 1 && p->nrb < 16; --rb)
            if (nrow % rb == 0 && rb * g.Gy <= maxT) p->rbs[p->nrb++] = rb;
        if (p->nrb) {
            g.RB = p->rbs[0];
            if (mm_smem_yz_for(p) > smax) p->nrb = 0;
        }
    }
    if (!p->nrb) {
        // bulk layout: separate y and z passes (double and float only)
        if (p->precision == MM_F32X2) return MM_ERR_UNSUPPORTED;
        g.bulk = 1;
        g.RB = 1;
        p->rbs[0] = 1;
        p->nrb = 1;
        const int maxT = mm_bulk_thread_bound(p);
        if (g.Gy > maxT || g.Gz > maxT) return MM_ERR_UNSUPPORTED;
        // z planes per y-pass CTA: up to 4, as many rows as one pass of threads covers
        g.ZB = 0;
        for (int zb = 4; zb >= 1; zb /= 2)
            if (zb <= g.nz && 3 * zb * g.Gy <= maxT && mm_bulk_smem_y(p, zb) <= smax) { g.ZB = zb; break; }
        if (!g.ZB) {
            if (mm_bulk_smem_y(p, 1) > smax) return MM_ERR_UNSUPPORTED;
            g.ZB = 1;
        }
        g.RBY = 3 * g.ZB;
        if (g.RBY * g.Gy > maxT) g.RBY = maxT / g.Gy;
        // y frequencies per z-pass CTA: runs of KB*3 complex values along y
        // coalesce; keep two CTAs per SM (<= 113 KiB each) where possible
        g.KB = 0;
        for (int kb = 16; kb >= 1; kb /= 2)
            if (kb <= g.Py && mm_bulk_smem_z(p, kb) <= 113 * 1024) { g.KB = kb; break; }
        if (!g.KB) {
            if (mm_bulk_smem_z(p, 1) > smax) return MM_ERR_UNSUPPORTED;
            g.KB = 1;
        }
        g.RBZ = 3 * g.KB;
        if (g.RBZ * g.Gz > maxT) g.RBZ = maxT / g.Gz;
    }
    g.nbody = g.bulk ? 5 : 3;
    // y rows per CTA in the x kernels: powers of two up to 16 (and up to the
    // next power of two of ny) within 768 threads and the shared-memory cap
    p->nty = 0;
    for (int ty = 1; ty <= 16 && ty <= next_pow2(gr.ny); ty *= 2)
        if (3 * ty * g.Gx <= 768 && mm_smem_x_for(p, ty) <= smax) p->tys[p->nty++] = ty;
    if (!p->nty) return MM_ERR_UNSUPPORTED;
    // untuned problems (below the autotuner's size) take the smallest tile:
    // the most CTAs per stage, which is what their latency-bound kernels need
    // (the 32 x 16 x 1 film: 49 us per evaluation against 69 us with the
    // widest tile); the autotuner replaces it on larger problems
    g.TY = g.TYF = p->tys[0];
    g.lty = g.ltyf = ilog2i(g.TY);
    // partial sums are sized for the smallest tile (most CTAs)
    p->nblk_x = ((gr.ny + p->tys[0] - 1) / p->tys[0]) * gr.nz;
    return MM_OK;
}

int build_graph(mm_problem *p)
{
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
    int rc = MM_OK;
    cudaGraph_t body = nullptr;
    do {
        if (cudaGraphCreate(&p->graph, 0)) { rc = MM_ERR_CUDA; break; }
        if (cudaGraphConditionalHandleCreate(&p->cond, p->graph, 1, cudaGraphCondAssignDefault)) { rc = MM_ERR_CUDA; break; }
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = p->cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        if (cudaGraphAddNode(&node, p->graph, nullptr, nullptr, 0, &np)) { rc = MM_ERR_CUDA; break; }
        body = np.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) { rc = MM_ERR_CUDA; break; }
        int lr = mm_launch_min_body(p, p->cond, cs, 1);
        cudaGraph_t out = body;
        cudaError_t ee = cudaStreamEndCapture(cs, &out);
        if (lr != MM_OK || ee) { rc = MM_ERR_CUDA; break; }
        if (cudaGraphInstantiate(&p->gexec, p->graph, 0)) { rc = MM_ERR_CUDA; break; }
        p->graph_ready = 1;
        ++p->graph_gen;
    } while (0);
    if (rc != MM_OK) {
        cudaError_t e = cudaGetLastError();
        if (e) mm_set_cuda_error(e, "minimiser graph");
    }
    cudaStreamDestroy(cs);
    return rc;
}

} // namespace

// Drop and recapture the minimiser graph (after a kernel parameter such as
// the per-cell anisotropy pointer changed).
int mm_rebuild_graph(mm_problem *p)
{
    if (p->gexec) { cudaGraphExecDestroy(p->gexec); p->gexec = nullptr; }
    if (p->graph) { cudaGraphDestroy(p->graph); p->graph = nullptr; }
    p->graph_ready = 0;
    return build_graph(p);
}

// Copy bytes between a caller buffer and a device buffer (either may be host memory).
int mm_copy_user(void *dst, const void *src, size_t bytes, bool dst_dev, bool src_dev, cudaStream_t s)
{
    cudaMemcpyKind k = dst_dev ? (src_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice)
                               : (src_dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, k, s);
    if (e) { mm_set_cuda_error(e, "cudaMemcpyAsync"); return MM_ERR_CUDA; }
    return MM_OK;
}

// The caller's m into iterate buffer 0: a copy in the problem's element
// type, or for MM_F32X2 a conversion of the caller's doubles to double-word
// pairs (host arrays pass through the input staging buffer).
int mm_load_iterate(mm_problem *p, const void *m, bool mdev, cudaStream_t s)
{
    const size_t F = 3 * (size_t)p->g.N * p->esz;
    if (p->precision != MM_F32X2) return mm_copy_user(p->mbuf[0], m, F, true, mdev, s);
    const void *src = m;
    if (!mdev) {
        int rc = mm_copy_user(p->stage_in, m, F, true, false, s);
        if (rc) return rc;
        src = p->stage_in;
    }
    return mm_launch_iterate_in(p, p->mbuf[0], (const double *)src, 3 * p->g.N, s);
}

namespace {
#define copy_user mm_copy_user

bool opts_ok(const mm_min_opts *o) { return mm_opts_ok(o); }

bool vec_ok(const double *h) { return h && std::isfinite(h[0]) && std::isfinite(h[1]) && std::isfinite(h[2]); }

// Record a failed runtime call and return rc.  Recording also reads the
// runtime's last-error slot, so the failure does not resurface at the next
// launch check.
int failed(cudaError_t e, const char *where, int rc)
{
    mm_set_cuda_error(e, where);
    return rc;
}

int status_of(int s)
{
    switch (s) {
    case MMS_CONVERGED: return MM_OK;
    case MMS_MAXITER: return MM_ERR_NOT_CONVERGED;
    case MMS_NONFINITE: return MM_ERR_NONFINITE;
    case MMS_TIMEOUT: return MM_ERR_TIMEOUT;
    }
    return MM_ERR_CUDA;
}

} // namespace

extern "C" int mm_newell(const mm_grid *grid, double *N_out, void *stream)
{
    NvtxRange nvtx_("mm_newell");
    if (!grid_ok(grid) || !N_out) return MM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * 6 * (size_t)grid->nx * grid->ny * grid->nz;
    const bool dev = is_device_ptr(N_out);
    double *d = N_out;
    if (!dev) {
        cudaError_t e = cudaMalloc((void **)&d, bytes);
        if (e) { mm_set_cuda_error(e, "cudaMalloc"); return MM_ERR_OOM; }
    }
    int rc = mm_newell_device(grid, d, s);
    if (rc == MM_OK && !dev) rc = copy_user(N_out, d, bytes, false, true, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (!dev) cudaFree(d);
    if (rc == MM_OK && e) { mm_set_cuda_error(e, "mm_newell"); rc = MM_ERR_CUDA; }
    return rc;
}

extern "C" int mm_setup_geometry(const mm_grid *grid, const mm_material *mat, int precision, void *stream,
                                 mm_problem **out)
{
    NvtxRange nvtx_("mm_setup_geometry");
    if (!out || !grid_ok(grid) || !mat) return MM_ERR_ARG;
    if (precision != MM_FP64 && precision != MM_FP32 && precision != MM_F32X2) return MM_ERR_ARG;
    if (!(std::isfinite(mat->Ms) && mat->Ms > 0) || !(std::isfinite(mat->A) && mat->A >= 0) || !std::isfinite(mat->K))
        return MM_ERR_ARG;
    const double un = std::sqrt(mat->u[0] * mat->u[0] + mat->u[1] * mat->u[1] + mat->u[2] * mat->u[2]);
    if (!mat->u_cell && !(std::fabs(un - 1.0) < 1e-9)) return MM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;

    mm_problem *p = new (std::nothrow) mm_problem;
    if (!p) return MM_ERR_OOM;
    memset((void *)p, 0, sizeof *p);
    p->grid = *grid;
    p->mat = *mat;
    p->mat.K_cell = nullptr;
    p->mat.u_cell = nullptr;
    p->precision = precision;
    p->esz = precision == MM_FP32 ? 4 : 8;   // MM_F32X2: fields and tensor as float pairs (8 bytes), like double
    int rc = plan(p);
    if (rc != MM_OK) { delete p; return rc; }
    cudaGetDevice(&p->dev);
    const Geom &g = p->g;
    const size_t F = 3 * (size_t)g.N * p->esz;
    const size_t vsz = 2 * p->esz;
    const size_t Wb = (size_t)g.C * 3 * g.nz * g.ny * vsz;
    const size_t Tb = tensor_bytes(g, p->esz);
    do {
        if ((rc = dalloc(p, &p->mbuf[0], F)) || (rc = dalloc(p, &p->mbuf[1], F)) ||
            (rc = dalloc(p, &p->gbuf[0], F)) || (rc = dalloc(p, &p->gbuf[1], F)) ||
            (rc = dalloc(p, &p->W, Wb)) || (rc = dalloc(p, &p->Nhat, Tb)) ||
            (g.bulk && (rc = dalloc(p, &p->W2, (size_t)g.C * 3 * g.nz * g.Py * vsz))) ||
            (rc = dalloc(p, &p->tw_px, g.Px * vsz)) || (rc = dalloc(p, &p->tw_py, g.Py * vsz)) ||
            (rc = dalloc(p, &p->tw_pz, g.Pz * vsz)) ||
            (rc = dalloc(p, (void **)&p->partials, sizeof(double) * RED_NSLOT * (size_t)p->nblk_x)) ||
            (rc = dalloc(p, (void **)&p->st, sizeof(MinState))) ||
            (rc = dalloc(p, (void **)&p->counter, 64)) ||
            (rc = dalloc(p, (void **)&p->Hext_dev, 4 * sizeof(double))) ||
            (rc = dalloc(p, &p->stage_in, F)) || (rc = dalloc(p, &p->stage_out, F)))
            break;
        cudaError_t ce;
        if ((ce = cudaMallocHost((void **)&p->st_host, sizeof(MinState)))) { rc = failed(ce, "cudaMallocHost", MM_ERR_OOM); break; }
        if ((ce = cudaMemsetAsync(p->st, 0, sizeof(MinState), s)) || (ce = cudaMemsetAsync(p->counter, 0, 64, s)) ||
            (ce = cudaMemsetAsync(p->gbuf[0], 0, F, s)) || (ce = cudaMemsetAsync(p->gbuf[1], 0, F, s))) {
            rc = failed(ce, "cudaMemsetAsync", MM_ERR_CUDA);
            break;
        }
        // per-cell material, converted to the working precision
        if (mat->K_cell || mat->u_cell) {
            double *tmp = nullptr;
            if ((ce = cudaMalloc((void **)&tmp, 3 * sizeof(double) * (size_t)g.N))) { rc = failed(ce, "cudaMalloc", MM_ERR_OOM); break; }
            if (mat->K_cell && rc == MM_OK) {
                if ((rc = dalloc(p, &p->Kc, (size_t)g.N * p->esz)) == MM_OK &&
                    (rc = copy_user(tmp, mat->K_cell, sizeof(double) * g.N, true, is_device_ptr(mat->K_cell), s)) == MM_OK)
                    rc = mm_launch_convert(p, p->Kc, tmp, g.N, s);
            }
            if (mat->u_cell && rc == MM_OK) {
                if ((rc = dalloc(p, &p->uc, 3 * (size_t)g.N * p->esz)) == MM_OK &&
                    (rc = copy_user(tmp, mat->u_cell, 3 * sizeof(double) * g.N, true, is_device_ptr(mat->u_cell), s)) == MM_OK)
                    rc = mm_launch_convert(p, p->uc, tmp, 3 * g.N, s);
            }
            cudaStreamSynchronize(s);
            cudaFree(tmp);
            if (rc != MM_OK) break;
        }
        if ((rc = mm_launch_twiddles(p, s)) != MM_OK) break;
        double *Nd = nullptr;
        if ((ce = cudaMalloc((void **)&Nd, sizeof(double) * 6 * (size_t)g.N))) { rc = failed(ce, "cudaMalloc", MM_ERR_OOM); break; }
        rc = mm_newell_device(&p->grid, Nd, s);
        if (rc == MM_OK) rc = mm_tensor_spectrum(p, Nd, s);
        cudaError_t e = cudaStreamSynchronize(s);
        cudaFree(Nd);
        if (rc != MM_OK) break;
        if (e) { mm_set_cuda_error(e, "setup"); rc = MM_ERR_CUDA; break; }
        if ((rc = mm_heff_configure(p)) != MM_OK) break;
        if ((ce = cudaMemsetAsync(p->mbuf[0], 0, F, s))) { rc = failed(ce, "cudaMemsetAsync", MM_ERR_CUDA); break; }
        // Problems below 65 536 cells are launch-latency bound and their kernel
        // times are mostly noise, so a timed choice would change from run to run.
        // The shape changes the order of the partial sums, and through it the
        // rounding that decides a minimiser's branch at a switching field.
        // They keep the planner's defaults (smallest tile, largest row batch).
        if (p->g.N >= 65536) {
            NvtxRange nvtx_tune("mm_autotune");
            if ((rc = mm_autotune(p, p->tys, p->nty, p->rbs, p->nrb, s)) != MM_OK) break;
        }
        if ((rc = build_graph(p)) != MM_OK) break;
    } while (0);
    if (rc != MM_OK) {
        cudaStreamSynchronize(s);
        free_problem(p);
        return rc;
    }
    *out = p;
    return MM_OK;
}

extern "C" int mm_destroy(mm_problem *p)
{
    if (!p) return MM_OK;
    cudaDeviceSynchronize();
    free_problem(p);
    return MM_OK;
}

extern "C" int mm_problem_info(const mm_problem *p, mm_info *info)
{
    if (!p || !info) return MM_ERR_ARG;
    const Geom &g = p->g;
    info->nx = g.nx; info->ny = g.ny; info->nz = g.nz;
    info->px = g.Px; info->py = g.Py; info->pz = g.Pz;
    info->precision = p->precision;
    info->cells = g.N;
    info->workspace_bytes = p->bytes;
    info->spectrum_bytes = (long)g.C * 3 * g.nz * g.ny * 2 * (long)p->esz;
    info->tensor_bytes = (long)tensor_bytes(g, p->esz);
    info->x_tile_rows = g.TY;
    info->yz_batch_rows = g.RB;
    info->bulk_layout = g.bulk;
    info->x_fwd_tile_rows = g.TYF;
    return MM_OK;
}

// Field evaluation with caller buffers (staged when on the host).
static int field_call(mm_problem *p, const void *m, const double Hext[3], void *H, int mode, cudaStream_t s)
{
    const size_t F = 3 * (size_t)p->g.N * p->esz;
    const bool mdev = is_device_ptr(m);
    const void *msrc = m;
    int rc;
    if (!mdev) {
        if ((rc = copy_user(p->stage_in, m, F, true, false, s))) return rc;
        msrc = p->stage_in;
    }
    void *hdst = nullptr;
    bool hdev = true;
    if (mode == MODE_HEFF) {
        hdev = is_device_ptr(H);
        hdst = hdev ? H : p->stage_out;
    }
    if ((rc = mm_launch_field(p, msrc, hdst, Hext, mode, s))) return rc;
    if (mode == MODE_HEFF && !hdev) {
        if ((rc = copy_user(H, p->stage_out, F, false, true, s))) return rc;
    }
    if (!mdev || !hdev) CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return MM_OK;
}

extern "C" int mm_heff(mm_problem *p, const void *m, const double Hext[3], void *H_out, void *stream)
{
    NvtxRange nvtx_("mm_heff");
    if (!p || !m || !H_out || !vec_ok(Hext)) return MM_ERR_ARG;
    return field_call(p, m, Hext, H_out, MODE_HEFF, (cudaStream_t)stream);
}

extern "C" int mm_energy(mm_problem *p, const void *m, const double Hext[3], double E_out[5], void *stream)
{
    NvtxRange nvtx_("mm_energy");
    if (!p || !m || !E_out || !vec_ok(Hext)) return MM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = field_call(p, m, Hext, nullptr, MODE_ENERGY, s);
    if (rc) return rc;
    CK(cudaMemcpyAsync(p->st_host, p->st, sizeof(MinState), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    for (int i = 0; i < 5; ++i) E_out[i] = p->st_host->energy[i];
    return MM_OK;
}

static void fill_result(const MinState &st, mm_min_result *r, long extra_launches)
{
    r->iters = st.k;
    r->heff_evals = st.evals;
    r->max_torque = st.max_torque;
    r->energy = st.energy[4];
    r->converged = st.status == MMS_CONVERGED;
    r->status = status_of(st.status);
    r->kernel_launches = st.launches + extra_launches;
}

extern "C" int mm_minimize(mm_problem *p, void *m, const double Hext[3], const mm_min_opts *opts,
                           mm_min_result *res, void *stream)
{
    NvtxRange nvtx_("mm_minimize");
    if (!p || !m || !vec_ok(Hext) || !opts_ok(opts)) return MM_ERR_ARG;
    if (!p->graph_ready) return MM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t F = 3 * (size_t)p->g.N * p->esz;
    const bool mdev = is_device_ptr(m);
    int rc;
    if ((rc = mm_load_iterate(p, m, mdev, s))) return rc;
    if ((rc = mm_launch_init_state(p, Hext, opts, 1, s))) return rc;
    if ((rc = mm_launch_loop(p, s))) return rc;
    if ((rc = mm_launch_copy_result(p, mdev ? m : p->stage_out, s))) return rc;
    if (!mdev && (rc = copy_user(m, p->stage_out, F, false, true, s))) return rc;
    CK(cudaMemcpyAsync(p->st_host, p->st, sizeof(MinState), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    const MinState st = *p->st_host;
    if (res) fill_result(st, res, 1);
    return status_of(st.status);
}

extern "C" int mm_hysteresis_sweep(mm_problem *p, void *m, const double *H_list, int n, int start,
                                   const mm_min_opts *opts, double *mavg, mm_min_result *per_step, void *stream)
{
    NvtxRange nvtx_("mm_hysteresis_sweep");
    if (!p || !m || !H_list || !mavg || n < 1 || start < 0 || start >= n || !opts_ok(opts)) return MM_ERR_ARG;
    for (int i = start; i < n; ++i)
        if (!vec_ok(H_list + 3 * i)) return MM_ERR_ARG;
    if (!p->graph_ready) return MM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t F = 3 * (size_t)p->g.N * p->esz;
    const bool mdev = is_device_ptr(m);
    int rc;
    if (p->rec_cap < n) {
        if (p->rec_dev) { cudaFree(p->rec_dev); p->bytes -= (long)sizeof(StepRecord) * p->rec_cap; p->rec_dev = nullptr; }
        if ((rc = dalloc(p, (void **)&p->rec_dev, sizeof(StepRecord) * (size_t)n))) { p->rec_cap = 0; return rc; }
        p->rec_cap = n;
    }
    if ((rc = mm_load_iterate(p, m, mdev, s))) return rc;
    for (int i = start; i < n; ++i) {
        if ((rc = mm_launch_init_state(p, H_list + 3 * i, opts, i == start, s))) return rc;
        if ((rc = mm_launch_loop(p, s))) return rc;
        if ((rc = mm_launch_record(p, i, s))) return rc;
    }
    if ((rc = mm_launch_copy_result(p, mdev ? m : p->stage_out, s))) return rc;
    if (!mdev && (rc = copy_user(m, p->stage_out, F, false, true, s))) return rc;
    StepRecord *rec = new (std::nothrow) StepRecord[n];
    if (!rec) return MM_ERR_OOM;
    cudaError_t e = cudaMemcpyAsync(rec + start, p->rec_dev + start, sizeof(StepRecord) * (n - start),
                                    cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) { delete[] rec; mm_set_cuda_error(e, "sweep"); return MM_ERR_CUDA; }
    int first_bad = MM_OK;
    for (int i = start; i < n; ++i) {
        const StepRecord &r = rec[i];
        for (int c = 0; c < 3; ++c) mavg[3 * i + c] = r.mavg[c];
        const int st = status_of(r.status);
        if (st != MM_OK && first_bad == MM_OK) first_bad = st;
        if (per_step) {
            mm_min_result &o = per_step[i];
            o.iters = r.iters; o.heff_evals = r.evals; o.max_torque = r.max_torque; o.energy = r.energy;
            o.converged = r.status == MMS_CONVERGED; o.status = st;
            o.kernel_launches = r.launches + 1 + (i == n - 1 ? 1 : 0);
        }
    }
    delete[] rec;
    return first_bad;
}

extern "C" int mm_kernel_times(mm_problem *p, const void *m, const double Hext[3], int reps, double *ms_out,
                               const char **names, int *count, void *stream)
{
    NvtxRange nvtx_("mm_kernel_times");
    if (!p || !m || !vec_ok(Hext) || reps < 1 || !ms_out || !names || !count) return MM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    if ((rc = mm_load_iterate(p, m, is_device_ptr(m), s))) return rc;
    mm_min_opts o = {0.0, 0.0, 1L << 40, MM_STEP_CAYLEY, 0.0, MM_TAU_ALTERNATE, 0.0};
    if ((rc = mm_launch_init_state(p, Hext, &o, 1, s))) return rc;
    rc = mm_kernel_stage_times(p, reps, ms_out, names, count, s);
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return rc;
}

extern "C" int mm_min_inspect(mm_problem *p, mm_min_state *out, void *m_k, void *m_prev, void *g_k, void *g_prev,
                              void *stream)
{
    NvtxRange nvtx_("mm_min_inspect");
    if (!p || !out) return MM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(p->st_host, p->st, sizeof(MinState), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    const MinState st = *p->st_host;
    // buffers of iterate k: m in mbuf[base ^ (k & 1)], g in gbuf[k & 1]
    const int cur = st.base ^ (int)(st.k & 1), gk = (int)(st.k & 1);
    const size_t F = 3 * (size_t)p->g.N * p->esz;
    void *dst[4] = {m_k, m_prev, g_k, g_prev};
    void *src[4] = {p->mbuf[cur], p->mbuf[cur ^ 1], p->gbuf[gk], p->gbuf[gk ^ 1]};
    for (int i = 0; i < 4; ++i) {
        if (!dst[i]) continue;
        const bool ddev = is_device_ptr(dst[i]);
        int rc;
        if (p->precision == MM_F32X2) {   // double-word storage: converted to the caller's double
            void *d = ddev ? dst[i] : p->stage_out;
            rc = mm_launch_iterate_out(p, (double *)d, src[i], 3 * p->g.N, s);
            if (!rc && !ddev) rc = copy_user(dst[i], p->stage_out, F, false, true, s);
        } else {
            rc = copy_user(dst[i], src[i], F, ddev, true, s);
        }
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    out->k = st.k;
    out->status = status_of(st.status == MMS_RUNNING ? MMS_CONVERGED : st.status);
    out->tau = st.tau;
    out->ss = st.bb[0];
    out->sy = st.bb[1];
    out->yy = st.bb[2];
    out->max_torque = st.max_torque;
    return MM_OK;
}
