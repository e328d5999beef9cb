// Shared device/host definitions of libmmgb: complex helpers, kernel
// parameter blocks, the device-resident minimiser state and the host-side
// problem object.
#pragma once

#include <cuda_runtime.h>
#include <type_traits>
#include <stdint.h>

#include "../../include/mm.h"
#include "dfloat.cuh"

#define MM_MU0 (4e-7 * 3.14159265358979323846)

// ---------------------------------------------------------------------------
// complex values: double2 / float2 (re = x, im = y)
// ---------------------------------------------------------------------------
template <typename T> struct cvec;
template <> struct cvec<double> { typedef double2 type; };
template <> struct cvec<float> { typedef float2 type; };
template <> struct cvec<dfloat> { typedef dcomplex type; };

template <typename V> __device__ __forceinline__ V cmake(decltype(V().x) a, decltype(V().x) b) { V r; r.x = a; r.y = b; return r; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) { V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r; }
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) { V r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r; }
template <typename V> __device__ __forceinline__ V cconj(V a) { V r; r.x = a.x; r.y = -a.y; return r; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename V> __device__ __forceinline__ V cmul_mi(V a)
{
    V r;
    if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
    return r;
}

// ---------------------------------------------------------------------------
// minimiser state, resident in device memory (one per problem)
// ---------------------------------------------------------------------------
enum { MMS_RUNNING = 0, MMS_CONVERGED = 1, MMS_MAXITER = 2, MMS_NONFINITE = 3, MMS_TIMEOUT = 4 };

// Reduction slots written per CTA by the local-terms kernel (double each).
enum {
    RED_SS = 0,      // sum s.s   (s = m_k - m_{k-1})
    RED_SY,          // sum s.y   (y = g_k - g_{k-1})
    RED_YY,          // sum y.y
    RED_T2MAX,       // max |m x H|^2
    RED_ED,          // sum m.H_demag
    RED_EEX,         // sum m.H_exchange
    RED_EAN,         // sum K (1 - (m.u)^2)
    RED_EZ,          // sum m.H_ext
    RED_MX, RED_MY, RED_MZ,  // sum m
    RED_PAD,         // unused: a CTA's row of partials stays a multiple of 16 bytes
    RED_NSLOT
};

struct MinState {
    // control, written by the host-side init kernel
    double tau0, tol_abs;     // tol_abs = tol * Ms (compared with |m x H|)
    double Hext[3];
    long max_iter;
    int step_kind;
    int base;                 // m buffer holding iterate 0
    unsigned long long t_start_ns, timeout_ns;
    // evolving
    long k;                   // current iterate index (evaluations so far - 1 once evaluated)
    double tau;               // step size for the next update
    int status;               // MMS_*
    long evals;
    double max_torque;        // max |m x H| / Ms at iterate k
    double energy[5];         // demag, exchange, anisotropy, zeeman, total (J) at iterate k
    double mavg[3];
    long launches;            // kernels launched by the loop body so far
    float Hextf[3];           // Hext and tau rounded once for the float kernels,
    float tauf;
    dfloat Hextw[3];          // and converted once to double-word pairs for the double-word
    dfloat tauw;              // kernels (a conversion per thread would run on the FP64 pipe)
    double bb[3];             // sums s.s, s.y, y.y over cells at iterate k (0 at k = 0)
    int tau_rule;             // MM_TAU_ALTERNATE or MM_TAU_ADAPTIVE
    double kappa;             // threshold of the adaptive rule
};

// Per-step record of a sweep
struct StepRecord {
    double mavg[3];
    double max_torque, energy;
    long iters, evals, launches;
    int status;
};

// ---------------------------------------------------------------------------
// Division by a runtime divisor d >= 1 through a precomputed multiplier
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, round-up variant): for 0 <= n < 2^31,
// n / d = (umulhi(n, mul) + n) >> shift with shift = ceil(log2 d) and
// mul = floor(2^32 (2^shift - d) / d) + 1.
// ---------------------------------------------------------------------------
struct FastDiv {
    unsigned mul;
    int shift;
    int d;
    __host__ __device__ void init(int dv)
    {
        d = dv;
        int l = 0;
        while ((1u << l) < (unsigned)dv) ++l;
        shift = l;
        mul = (unsigned)((((unsigned long long)1 << 32) * (((unsigned long long)1 << l) - (unsigned long long)dv)) /
                         (unsigned long long)dv + 1ull);
    }
#ifdef __CUDACC__
    __device__ __forceinline__ int div(int n) const
    {
        return (int)((__umulhi((unsigned)n, mul) + (unsigned)n) >> shift);
    }
#endif
};

// ---------------------------------------------------------------------------
// Geometry shared by the field kernels (passed by value)
// ---------------------------------------------------------------------------
struct Geom {
    int nx, ny, nz;
    int Px, Py, Pz;        // padded FFT lengths
    int Hx, C;             // Hx = Px/2 (packed complex length), C = Hx + 1 x-frequencies
    int lhx, lpy;          // log2(Hx), log2(Py)
    int Gx, Gy;            // threads per FFT row: max(1, L/8)
    int TY;                // y rows per CTA of the x-inverse kernel
    int TYF, ltyf;         // y rows per CTA of the x-forward kernel, log2
    int RB;                // y rows transformed at once in the y-z kernel (divides 3 nz)
    int rsx, rsy;          // smem row strides (complex elements) of the x and y FFT rows
    // bulk layout (grids whose padded y-z plane does not fit one CTA): the
    // y-z stage runs as three passes, y forward / z convolution / y inverse
    int bulk;              // 0: film layout (one y-z kernel), 1: bulk layout
    int ZB;                // z planes per CTA of the y passes
    int RBY;               // y rows transformed at once in the y passes
    int KB;                // y frequencies per CTA of the z pass
    int RBZ;               // z rows transformed at once in the z pass
    int lpz, Gz, rsz;      // log2(Pz), threads per z row, smem stride of a z row
    int nbody;             // kernels per minimiser iteration (3 film, 5 bulk)
    long N;                // cells
    double dx, dy, dz;
    double Ms;
    double cex_x, cex_y, cex_z;   // 2A/(mu0 Ms d^2) per axis
    double can;                    // 2/(mu0 Ms) (times K per cell)
    double K;                      // uniform K
    double u[3];                   // uniform axis
    // the same constants rounded once to float for the float kernels (a
    // conversion per thread would run on the slow FP64 pipe)
    float fcex_x, fcex_y, fcex_z, fcan, fK, fu[3];
    dfloat wcex[3], wcan, wK, wu[3];   // and as double-word pairs for the double-word kernels
    int lty;                       // log2(TY)
    FastDiv fd_nx, fd_ny, fd_padx, fd_pady;  // divisors nx, ny, Px - nx, Py - ny
    int stage;                     // k_xinv (float) stages its stencil rows with 16-byte cp.async
    FastDiv fd_nc;                 // 16-byte chunks per x row when staging
};

__host__ __device__ __forceinline__ int mm_ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

#ifdef __CUDACC__
// asynchronous global -> shared copies (cp.async); both addresses aligned to
// the copy size; complete for the issuing thread at cp_async_wait_all()
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's most recent commit groups are pending
template <int N> __device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
#endif

// value of a double constant in the kernel's precision (float copy for float)
template <typename T> __host__ __device__ __forceinline__ T pick(double d, float f)
{
    if constexpr (sizeof(T) == 4) return f;
    else return d;
}
// the same with the double-word copy for the double-word kernels
template <typename T> __host__ __device__ __forceinline__ T pick(double d, float f, dfloat w)
{
    if constexpr (std::is_same<T, dfloat>::value) return w;
    else return pick<T>(d, f);
}



// Field evaluation modes of the x-inverse/local kernel
enum { MODE_HEFF = 0, MODE_ENERGY = 1, MODE_MIN = 2 };

// Element type of the caller's arrays for fields stored as T: T itself,
// double for double-word storage (the ABI's arrays of an MM_F32X2 problem
// are double; its iterates are kept as float pairs)
template <typename T> struct io_of { typedef T type; };
template <> struct io_of<dfloat> { typedef double type; };

// T: element type of the minimiser's fields m and g and of the local terms
// (double, float, or dfloat for MM_F32X2); F: arithmetic type of the FFTs and
// the convolution, whose complex values fill the spectrum buffers and the
// tensor; IO: the caller's element type (m for MODE_HEFF/ENERGY, H, per-cell
// material)
template <typename T, typename F = T>
struct FieldPtrs {
    typedef typename cvec<F>::type V;
    typedef typename io_of<T>::type IO;
    const IO *m_src;       // field input for MODE_HEFF/ENERGY, or NULL (then mbuf by state)
    IO *H_out;             // MODE_HEFF output
    T *mbuf[2];            // minimiser iterate buffers
    T *gbuf[2];            // projected-gradient buffers
    V *W;                  // spectrum [C][nz][ny][3] (x-frequency slowest, component fastest)
    V *W2;                 // bulk layout only: y-transformed spectrum [C][nz][Py][3]
    const F *Nhat;         // tensor: film [C][max(1,Pz/2)][6][Py/2+1] (x-y transform at real z offsets, scaled by
                           // -Ms/(Px Py)); bulk [C][Pz/2+1][Py/2+1][6] (octant of the 3-D spectrum,
                           // scaled by -Ms/(Px Py Pz))
    const V *tw_px;        // exp(-2 pi i t/Px), t < Px
    const V *tw_py;        // exp(-2 pi i t/Py), t < Py
    const V *tw_pz;        // exp(-2 pi i t/Pz), t < Pz
    const IO *Kc;          // per-cell K or NULL
    const IO *uc;          // per-cell axis [3][N] or NULL
    double *partials;      // [nblocks][RED_NSLOT]
    MinState *st;          // minimiser state (MODE_MIN and updates)
    unsigned *counter;     // CTAs of the current x-inverse launch that have finished (reset by the last)
    double hscale;         // MODE_HEFF writes hscale * H (1 for the field itself)
};

// ---------------------------------------------------------------------------
// host-side problem object
// ---------------------------------------------------------------------------
struct mm_problem {
    mm_grid grid;
    mm_material mat;
    int precision;
    Geom g;
    size_t esz;            // sizeof(T)
    // device memory
    void *mbuf[2], *gbuf[2];
    void *W;
    void *W2;              // bulk layout only
    void *Nhat;
    void *tw_px, *tw_py, *tw_pz;
    void *Kc, *uc;
    double *partials;
    unsigned *counter;     // completion counter of the x-inverse kernel
    int nblk_x;            // CTAs of the x kernels (= partial slots)
    int tys[8], nty;       // admissible rows-per-tile of the x kernels
    void *adj[2];          // two more field buffers for the adjoint solver (allocated on first use)
    int rbs[16], nrb;      // admissible rows-per-batch of the y-z kernel
    MinState *st;
    MinState *st_host;     // pinned mirror
    double *Hext_dev;
    void *stage_in, *stage_out;    // staging for host m / H
    StepRecord *rec_dev;   // sweep records (capacity rec_cap)
    int rec_cap;
    long bytes;
    // graph of the device-side minimiser loop
    cudaGraph_t graph;
    cudaGraphExec_t gexec;
    cudaGraphConditionalHandle cond;
    int graph_ready;
    int graph_gen;         // incremented at every capture of the minimiser graph
    int dev;
    // device-side conjugate-gradient loop of the adjoint (built on first use)
    cudaGraph_t adj_graph;
    cudaGraphExec_t adj_exec;
    cudaGraphConditionalHandle adj_cond;
    void *adj_state;       // CgState (adjoint.cu)
    double *adj_partials;  // per-CTA partial dot products
    int adj_nblk;
};

// one minimisation on the device: a launch of the problem's minimiser graph (heff.cu)
int mm_launch_loop(mm_problem *p, cudaStream_t s);

// drop the adjoint's loop graph (it bakes in kernel parameters such as the
// per-cell anisotropy pointer); rebuilt on the next mm_adjoint_dK
void mm_adjoint_invalidate(mm_problem *p);

// field-kernel entry points of each precision (field_fp64.cu, field_fp32.cu, field_f32x2.cu)
#define MM_DECLARE_FIELD_ENTRIES(SFX)                                                                          \
    cudaError_t mm_fields_configure_##SFX(const Geom &g, size_t sxf, size_t sx, size_t syz);                  \
    cudaError_t mm_fields_autotune_##SFX(mm_problem *p, const int *tys, int nty, const int *rbs, int nrb,      \
                                         cudaStream_t s);                                                      \
    cudaError_t mm_fields_chain_##SFX(mm_problem *p, const void *m, void *H, const double *hext, int mode,    \
                                      cudaStream_t s, double hscale);                                         \
    cudaError_t mm_fields_min_body_##SFX(mm_problem *p, cudaGraphConditionalHandle h, cudaStream_t s,         \
                                         int use_cond);                                                        \
    cudaError_t mm_fields_stage_times_##SFX(mm_problem *p, int reps, double *ms, cudaStream_t s);
MM_DECLARE_FIELD_ENTRIES(fp64)
MM_DECLARE_FIELD_ENTRIES(fp32)
MM_DECLARE_FIELD_ENTRIES(f32x2)

// Largest dynamic shared memory any field-kernel launch may use (the
// planner keeps every launch shape within it).  Kernels get this limit as
// their MaxDynamicSharedMemorySize attribute once and for all: the attribute
// belongs to the kernel function, shared by every problem of the process, so
// setting it to one problem's own need would refuse the larger launches of
// problems configured before it.  It only permits launches; nothing is
// reserved by it.
#define MM_SMEM_CAP (200 * 1024)

// launchers implemented in heff.cu
int mm_launch_min_body(mm_problem *p, cudaGraphConditionalHandle h, cudaStream_t s, int use_cond);
int mm_kernel_stage_times(mm_problem *p, int reps, double *ms, const char **names, int *count, cudaStream_t s);
int mm_launch_init_state(mm_problem *p, const double Hext[3], const mm_min_opts *o, int reset_base, cudaStream_t s);
int mm_launch_record(mm_problem *p, int step, cudaStream_t s);
int mm_launch_copy_result(mm_problem *p, void *dst, cudaStream_t s);
size_t mm_smem_x_for(const mm_problem *p, int ty);
size_t mm_smem_yz_for(const mm_problem *p);
int mm_yz_thread_bound(const mm_problem *p);
int mm_heff_configure(mm_problem *p);
int mm_autotune(mm_problem *p, const int *tys, int nty, const int *rbs, int nrb, cudaStream_t s);
int mm_launch_twiddles(mm_problem *p, cudaStream_t s);
int mm_launch_field(mm_problem *p, const void *m, void *H, const double *hext, int mode, cudaStream_t s,
                    double hscale = 1.0);
// double values into the problem's material type (per-cell K and axes:
// float for MM_FP32, else double)
int mm_launch_convert(mm_problem *p, void *dst, const double *src, long n, cudaStream_t s);
// MM_F32X2 only: the caller's double values into double-word iterate storage, and back
int mm_launch_iterate_in(mm_problem *p, void *dst, const double *src, long n, cudaStream_t s);
int mm_launch_iterate_out(mm_problem *p, double *dst, const void *src, long n, cudaStream_t s);
int mm_rebuild_graph(mm_problem *p);
// implemented in bulk.cu: the three y-z passes of the bulk layout (pass -1:
// all three in order; 0, 1, 2: only that one)
cudaError_t mm_bulk_conv(const Geom &g, const FieldPtrs<double> &P, cudaStream_t s, int pass);
cudaError_t mm_bulk_conv(const Geom &g, const FieldPtrs<float> &P, cudaStream_t s, int pass);
size_t mm_bulk_smem_y(const mm_problem *p, int zb);
size_t mm_bulk_smem_z(const mm_problem *p, int kb);
int mm_bulk_thread_bound(const mm_problem *p);
cudaError_t mm_bulk_configure(const mm_problem *p);
// implemented in newell.cu
int mm_newell_device(const mm_grid *g, double *N_dev, cudaStream_t s);
int mm_tensor_spectrum(mm_problem *p, const double *N_dev, cudaStream_t s);

// helpers (api.cu)
bool mm_is_device_ptr(const void *ptr);
// fields of this problem are double (MM_FP64, MM_F32X2) rather than float
inline bool mm_double_fields(const mm_problem *p) { return p->precision != MM_FP32; }
// options of a minimisation within range (finite tolerances, known rules)
bool mm_opts_ok(const mm_min_opts *o);
// streaming multiprocessors of the current device (queried once per device)
int mm_sm_count();
// grid of a grid-stride loop over n elements with `threads` per CTA: enough
// CTAs for n, at most `per_sm` resident CTAs on every SM of the device
int mm_grid_for(long n, int threads, int per_sm);
int mm_copy_user(void *dst, const void *src, size_t bytes, bool dst_dev, bool src_dev, cudaStream_t s);
// the caller's m (host or device, the ABI's element type) into iterate buffer 0
int mm_load_iterate(mm_problem *p, const void *m, bool mdev, cudaStream_t s);
// error bookkeeping (api.cu)
void mm_set_cuda_error(cudaError_t e, const char *where);
