/*
 * mm.h -- C ABI of libmmgb.so: energy-minimising hysteresis for
 * finite-difference micromagnetics on one NVIDIA GB300 (sm_103a).
 *
 * The method is the one of Abert, Wautischer, Bruckner, Satz and Suess,
 * "Efficient Energyminimization in Finite-Difference Micromagnetics:
 * Speeding up Hysteresis Computations" (arXiv 1405.2728):
 *   - effective field H_eff = -(1/(mu0 Ms)) dU/dm, Eq. (effective_field), with
 *     the demagnetisation field as an FFT convolution on a regular cuboid grid
 *     (Section 3), exchange, uniaxial anisotropy and Zeeman terms (Section 4);
 *   - projected gradient g = m x (m x H_eff), Eq. (projected_direction) and the
 *     auxiliary fields of Eq. (stepsize);
 *   - norm-preserving midpoint step, Eq. (implicit_gradient_descent), solved in
 *     closed form;
 *   - Barzilai-Borwein step sizes tau^1, tau^2 of Eq. (stepsize) used
 *     alternately, a small first step and a sup-norm stop rule (Section 2);
 *   - the hysteresis driver: one minimisation per field value, warm-started
 *     from the previous magnetisation (Section 4).
 *
 * Conventions shared by every call
 * --------------------------------
 * Units: SI.  Lengths in m, Ms and fields in A/m, A in J/m, K in J/m^3,
 *   energies in J.  mu0 = 4 pi 1e-7 exactly.
 * Layout: a vector field is structure-of-arrays [3][nz][ny][nx] (component,
 *   then z, y, x with x fastest), contiguous, N = nx*ny*nz cells per component.
 *   Scalars per cell are [nz][ny][nx].
 * Element type: double for MM_FP64 problems, float for MM_FP32 problems.
 * Pointers marked "host or device" may be either: the library asks the CUDA
 *   runtime which one it is.  Device pointers are used in place; host
 *   memory (preferably pinned) is staged through library-owned device buffers
 *   inside the call.  Device pointers must be 16-byte aligned.
 * Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   All device work of a call is issued on it.  Calls that return host
 *   results synchronise that stream before returning; mm_heff with device
 *   pointers returns without synchronising.
 * Ownership: the caller owns every m, H and K/u buffer it passes; the library
 *   keeps no reference to them after the call returns.  The library owns the
 *   problem object and everything in it (tensor spectra, FFT twiddles,
 *   workspaces, CUDA graphs), released by mm_destroy.
 * Errors: every call returns an mm_status code and never aborts the process.
 *   On MM_ERR_ARG / MM_ERR_UNSUPPORTED nothing is written.  MM_ERR_CUDA
 *   means a CUDA runtime call failed (mm_last_cuda_error tells which); the
 *   problem should then be destroyed.
 * Threading: a problem object must not be used by two host threads at once.
 */
#ifndef MMGB_MM_H
#define MMGB_MM_H

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MM_API __attribute__((visibility("default")))
#else
#define MM_API
#endif

typedef struct mm_problem mm_problem; /* opaque, owned by the library */

typedef enum {
    MM_OK = 0,
    MM_ERR_ARG = -1,            /* invalid argument (null, non-positive size, non-unit axis, misaligned) */
    MM_ERR_OOM = -2,            /* device allocation failed */
    MM_ERR_CUDA = -3,           /* a CUDA runtime call failed */
    MM_ERR_NOT_CONVERGED = -4,  /* max_iter steps taken without meeting tol; m holds the last iterate */
    MM_ERR_NONFINITE = -5,      /* a non-finite torque, energy or step size appeared */
    MM_ERR_TIMEOUT = -6,        /* the minimiser's wall-clock limit (timeout_s) passed; m holds the last iterate */
    MM_ERR_UNSUPPORTED = -7     /* valid but outside what this build supports (see mm_setup_geometry) */
} mm_status;

/* Element type and arithmetic of the field path.  MM_F32X2 (an extension):
 * the caller's arrays are double as for MM_FP64; inside, the iterates, the
 * FFTs, the demagnetisation convolution, the local terms, the step and the
 * per-CTA sums use double-float arithmetic (pairs of floats, about 48
 * significant bits, run on the FP32 pipes), and the sums across CTAs,
 * the step size and the stop rule are double; film-layout grids only (see
 * mm_setup_geometry). */
enum { MM_FP64 = 0, MM_FP32 = 1, MM_F32X2 = 2 };
enum { MM_STEP_CAYLEY = 0, MM_STEP_NORMALIZE = 1 };  /* update rule, see mm_min_opts */
enum { MM_TAU_ALTERNATE = 0, MM_TAU_ADAPTIVE = 1 };  /* step-size rule, see mm_min_opts */

/* Regular cuboid grid of nx*ny*nz cells of size dx*dy*dz (Section 3). */
typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
} mm_grid;

/* Material (Section 4): saturation magnetisation Ms > 0, exchange A >= 0,
 * uniaxial anisotropy K (any sign) with unit easy axis u.  Optional per-cell
 * overrides (host or device, double, read once by mm_setup_geometry):
 * K_cell [nz][ny][nx] replaces K; u_cell [3][nz][ny][nx] replaces u and must
 * hold unit vectors. */
typedef struct {
    double Ms, A, K;
    double u[3];
    const double *K_cell;
    const double *u_cell;
} mm_material;

/*
 * mm_newell -- the cell-averaged demagnetisation tensor of the grid (the
 * convolution kernel of the FFT demagnetisation field, Section 3; Newell,
 * Williams and Dunlop, J. Geophys. Res. 98 (1993) 9551), computed on the GPU
 * in double-double arithmetic and rounded to double.
 *
 * N_out (host or device, double): [6][nz][ny][nx], components xx, yy, zz, xy,
 * xz, yz at the non-negative offsets (i, j, k) cells, 0 <= i < nx etc.
 * Other offsets follow by symmetry: N_aa is even in every coordinate, N_ab is
 * odd in coordinate a and in coordinate b.  With this tensor the
 * demagnetisation field is H_d(r_i) = -Ms sum_j N(r_i - r_j) m_j.
 * Returns MM_OK, MM_ERR_ARG, MM_ERR_OOM or MM_ERR_CUDA; synchronises `stream`.
 */
MM_API int mm_newell(const mm_grid *grid, double *N_out, void *stream);

/*
 * mm_newell_static -- the same tensor as mm_newell, for callers that cannot
 * allocate device memory.  The paper has no counterpart; this call exists for
 * callers whose device memory is fully reserved by another allocator or
 * capped by a fixed budget, and for code on latency-critical streams that must
 * not call cudaMalloc/cudaFree (which may synchronise the whole device).
 * It calls no allocating routine: its double-double work table is a static
 * device array of 6 MiB compiled into the library, held by every GPU that
 * loads it until the process exits.
 * N_dev: DEVICE memory of the current device only (host pointers, and
 * device memory of another GPU, return MM_ERR_ARG), double, [6][nz][ny][nx],
 * same layout and values as mm_newell.
 * Limit: (nx+1)(ny+1)(nz+1) <= 65536 lattice points (e.g. 255 x 127 x 1,
 * 63 x 63 x 15); larger grids return MM_ERR_UNSUPPORTED and launch nothing.
 * Asynchronous on `stream`; returns after launching (launch errors give
 * MM_ERR_CUDA).  The first call on each device looks up the table's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  All calls on a device share the one table:
 * calls whose kernels overlap on the GPU (different streams without ordering)
 * race and give wrong results.
 */
MM_API int mm_newell_static(const mm_grid *grid, double *N_dev, void *stream);

/*
 * mm_setup_geometry -- create a problem: validates the grid and material,
 * allocates device workspaces, computes the Newell tensor (as mm_newell), its
 * Fourier spectrum on the zero-padded grid (padded size per axis: the smallest
 * power of two >= 2n-1, and >= 2 along x), times the admissible launch
 * shapes of the field kernels on this problem and keeps the fastest, and
 * captures the minimiser's CUDA graph.  precision = MM_FP64 or MM_FP32: element type of m/H and of the FFT
 * and stencil arithmetic; MM_F32X2: double arrays, double-float arithmetic
 * (see the enum).  The reductions (step-size sums, energies,
 * averages) are combined across CTAs in double and the step size is chosen in
 * double.  Within a CTA the MM_FP64 path accumulates in double; the MM_FP32
 * path adds every per-cell product exactly (an FMA-split product) into a
 * compensated float pair (about 46 significant bits), which mm_min_inspect
 * lets callers check against their own double reduction; the MM_F32X2 path
 * accumulates in double-float pairs.
 * Two layouts of the y-z stage of the convolution.  Film layout (nz <= 4 and
 * the padded y-z plane of one x-frequency, about 3 * nz * 9/8 * Py complex
 * values, within 200 KiB of shared memory; e.g. 512 x 256 x 4 in FP64 or
 * 1024 x 512 x 4 in FP32): one kernel per x-frequency.  Bulk layout (every
 * other grid, e.g. 256^3 cubes): separate y, z and inverse-y passes through
 * an extra spectrum buffer of C * nz * Py * 3 complex values.
 * Supported in this build (else MM_ERR_UNSUPPORTED): every padded length
 * <= 4096 (nx, ny, nz <= 2048) and one padded y row or z row, with its
 * twiddles, within 200 KiB of shared memory.
 * On success *out receives the new problem.  Synchronises `stream`.
 */
MM_API int mm_setup_geometry(const mm_grid *grid, const mm_material *mat, int precision, void *stream,
                      mm_problem **out);

/* mm_destroy -- free a problem and everything it owns (NULL is accepted). */
MM_API int mm_destroy(mm_problem *prob);

/*
 * mm_heff -- effective field, Eq. (effective_field) (Sections 3 and 4):
 *   H = H_demag + H_exchange + H_anisotropy + H_ext, with
 *   H_demag,i    = -Ms sum_j N(r_i - r_j) m_j        (zero-padded FFT convolution)
 *   H_exchange,i = (2A/(mu0 Ms)) sum_{j in nb(i)} (m_j - m_i)/d_ij^2   (six
 *                  neighbours; neighbours outside the grid are absent)
 *   H_aniso,i    = (2K_i/(mu0 Ms)) (m_i . u_i) u_i
 * m (host or device) [3][nz][ny][nx] unit vectors; Hext[3] (host, A/m);
 * H_out (host or device) [3][nz][ny][nx] in A/m.
 */
MM_API int mm_heff(mm_problem *prob, const void *m, const double Hext[3], void *H_out, void *stream);

/*
 * mm_energy -- the discrete energy whose cell gradient is mm_heff:
 *   E_demag = -(mu0 Ms V/2) sum m.H_demag, E_exchange = A V sum_{neighbour
 *   pairs} |m_j - m_i|^2/d^2, E_aniso = sum K_i V (1 - (m_i.u_i)^2),
 *   E_zeeman = -mu0 Ms V sum m.H_ext, with V = dx dy dz.
 * E_out (host) [5] = demag, exchange, anisotropy, Zeeman, total, in J.
 * Synchronises `stream`.
 */
MM_API int mm_energy(mm_problem *prob, const void *m, const double Hext[3], double E_out[5], void *stream);

/* Options of one minimisation (Section 2).
 * tol       stop when max_i |m_i x H_i| / Ms < tol (the sup-norm stop rule,
 *           evaluated on m_k before stepping).
 * tau0      first step size (the "reasonably small guess"), in m/A; <= 0
 *           selects 1e-2/Ms.
 * max_iter  at most this many steps (so at most max_iter+1 field evaluations).
 * step_kind MM_STEP_CAYLEY: the midpoint scheme, Eq. (implicit_gradient_descent),
 *           in closed form m' = [(1 - tau^2|g|^2/4) m - tau g]/(1 + tau^2|g|^2/4);
 *           MM_STEP_NORMALIZE: m' = (m - tau g)/|m - tau g|, the explicit
 *           projected step Eq. (projected_gradient_descent) renormalised.
 * timeout_s wall-clock limit of the device loop in seconds (<= 0: none).
 * tau_rule  MM_TAU_ALTERNATE: the alternation of Section 2;
 *           MM_TAU_ADAPTIVE: the "more elaborate switch" the paper cites but
 *           does not give, read as the adaptive Barzilai-Borwein rule of Zhou,
 *           Gao and Dai (Comput. Optim. Appl. 35 (2006) 69): tau^2 when
 *           tau^2/tau^1 = (s.y)^2/((s.s)(y.y)) < tau_kappa, else tau^1.
 * tau_kappa threshold of the adaptive rule, in (0, 1]; <= 0 selects 0.5.
 * Step sizes: tau_0 = tau0; for k >= 1, with s = m_k - m_{k-1} and
 * y = g_k - g_{k-1} summed over all cells, tau^1 = s.s/s.y on odd k and
 * tau^2 = s.y/y.y on even k (Eq. stepsize, alternating) or as tau_rule
 * selects; when that quotient is not finite and positive, sqrt(s.s/y.y),
 * else tau0. */
typedef struct {
    double tol;
    double tau0;
    long max_iter;
    int step_kind;
    double timeout_s;
    int tau_rule;
    double tau_kappa;
} mm_min_opts;

/* Outcome of one minimisation. */
typedef struct {
    long iters;          /* steps taken */
    long heff_evals;     /* effective-field evaluations (iters + 1) */
    double max_torque;   /* max_i |m_i x H_i| / Ms at the returned m */
    double energy;       /* total energy at the returned m, J */
    int converged;       /* 1 if max_torque < tol */
    int status;          /* mm_status of this minimisation */
    long kernel_launches;/* CUDA kernels this minimisation launched */
} mm_min_result;

/*
 * mm_minimize -- minimise the energy at fixed external field Hext (host, A/m)
 * starting from m (host or device, in/out, unit vectors), following Section 2.
 * The loop runs on the device (a CUDA graph with a device-side conditional
 * loop); the host waits once at the end.  res (host, nullable) receives the
 * outcome.  Returns MM_OK, MM_ERR_NOT_CONVERGED, MM_ERR_NONFINITE,
 * MM_ERR_TIMEOUT (m then holds the last iterate), MM_ERR_ARG or MM_ERR_CUDA.
 * Synchronises `stream`.
 */
MM_API int mm_minimize(mm_problem *prob, void *m, const double Hext[3], const mm_min_opts *opts,
                mm_min_result *res, void *stream);

/*
 * mm_hysteresis_sweep -- the hysteresis driver of Section 4: for field values
 * H_list[start..n-1] (host, [n][3], A/m) in order, minimise as mm_minimize
 * starting from the previous result (the step-size history restarts at every
 * field value) and record the average magnetisation <m> = (1/N) sum_i m_i in
 * mavg (host, [n][3]; entries before `start` untouched).  m (host or device,
 * in/out) holds the start state and receives the final state.  per_step
 * (host, nullable, [n]) receives each field value's outcome.  The whole sweep
 * is issued without host round trips; the host synchronises once at the end.
 * Returns MM_OK if every field value converged, else the first non-OK status
 * met (the sweep still runs to the end).  `start` allows resuming a sweep.
 */
MM_API int mm_hysteresis_sweep(mm_problem *prob, void *m, const double *H_list, int n, int start,
                        const mm_min_opts *opts, double *mavg, mm_min_result *per_step,
                        void *stream);

/*
 * Differentiation (an extension beyond the paper, whose method only minimises).
 *
 * mm_energy_gradient -- G_out = scale * dU/dm with dU/dm_i = -mu0 Ms V H_eff,i
 * (Eq. effective_field read cell-wise), the energy of mm_energy.  For
 * automatic differentiation scale is the incoming gradient of U.  m, G_out:
 * host or device [3][nz][ny][nx].
 */
MM_API int mm_energy_gradient(mm_problem *prob, const void *m, const double Hext[3], double scale, void *G_out,
                              void *stream);

/*
 * mm_hessian_vec -- the tangent-plane second derivative at m applied to a
 * tangent field v (units A/m; times mu0 Ms V it is the Riemannian Hessian of U):
 *   Av = P_m((m.H) v - L v)  (= (m.H) v - P_m(L v) for tangent v),  H = H_eff(m),
 *   L v = H_eff(v) without the external field,  P_m w = w - (m.w) m.
 * m, v, Av: host or device [3][nz][ny][nx].  Overwrites the minimiser's work
 * buffers (a later mm_minimize / mm_hysteresis_sweep starts from its own m).
 */
MM_API int mm_hessian_vec(mm_problem *prob, const void *m, const double Hext[3], const void *v, void *Av,
                          void *stream);

/*
 * mm_adjoint_dK -- implicit adjoint at a converged minimum m of mm_minimize:
 * the gradient of an objective J(m*(K)) with respect to the per-cell
 * anisotropy constants.  With the operator A of mm_hessian_vec it solves
 * A lambda = P_m(dJ/dm) by conjugate gradients (relative residual < tol, at
 * most max_iter iterations) and returns dJdK[i] = lambda_i . P_m(dH_i/dK_i),
 * dH_i/dK_i = (2/(mu0 Ms)) (m_i.u_i) u_i.  Example: J = <m_x> has
 * dJ/dm = (1/N, 0, 0) in every cell.
 * dJdm: host or device [3][nz][ny][nx] (problem precision); dJdK: host or
 * device double [nz][ny][nx]; iters, resid (host, nullable): CG iterations and
 * final relative residual.  Returns MM_OK, MM_ERR_NOT_CONVERGED (max_iter
 * reached), MM_ERR_NONFINITE (A not positive on the search direction: m is
 * not a minimum), MM_ERR_ARG, MM_ERR_OOM or MM_ERR_CUDA.  Synchronises `stream`.
 */
MM_API int mm_adjoint_dK(mm_problem *prob, const void *m, const double Hext[3], const void *dJdm, double *dJdK,
                         double tol, long max_iter, long *iters, double *resid, void *stream);

/*
 * mm_set_anisotropy -- replace the per-cell anisotropy constants
 * (host or device double [nz][ny][nx]) of an existing problem, e.g. for finite
 * differences or parameter studies.  Synchronises `stream`.
 */
MM_API int mm_set_anisotropy(mm_problem *prob, const double *K_cell, void *stream);

/*
 * mm_hysteresis_sweep_mixed -- the hysteresis driver of Section 4 in mixed
 * precision (an extension; the paper uses one precision).  For every field
 * value j >= start, the FP32 problem `lo` first minimises from the current
 * state with opts_lo (a loose tolerance).  The FP64 problem `hi` then
 * minimises from that result with opts_hi (the final tolerance).  The float
 * phase does most of the descent at the float rate.  The double phase
 * finishes the last decades of the stop rule, where float rounding slows the
 * step-size rule down.  lo and hi must come from mm_setup_geometry with the
 * same grid and material, precisions MM_FP32 and MM_FP64.
 * m (host or device, [3][nz][ny][nx] float64, in/out) is the starting state;
 * it receives the final one.  H_list, n, start, mavg as mm_hysteresis_sweep
 * (mavg from the FP64 phase).  per_step_lo / per_step_hi (host, nullable,
 * [n]) receive each phase's result; a float phase that stops at its
 * iteration cap is not an error.  Returns MM_OK if every FP64 phase
 * converged, else the first non-OK FP64 status.  Synchronises `stream`.
 */
MM_API int mm_hysteresis_sweep_mixed(mm_problem *lo, mm_problem *hi, void *m, const double *H_list, int n, int start,
                                     const mm_min_opts *opts_lo, const mm_min_opts *opts_hi, double *mavg,
                                     mm_min_result *per_step_lo, mm_min_result *per_step_hi, void *stream);

/*
 * Batched sweeps (an extension; the paper sweeps one sample).  A batch
 * references existing problems (of any sizes and precisions; the caller keeps
 * owning them and must not destroy them while the batch exists) and runs
 * their hysteresis sweeps together.  Three ways to run them (`kind` of
 * mm_batch_create_kind; mm_batch_create takes MM_BATCH_AUTO):
 * MM_BATCH_BRANCHES (what MM_BATCH_AUTO selects; any problems): one sweep
 * call is ONE graph launch.  The graph holds one independent branch per
 * problem: a device-side loop over the field values whose body sets the
 * minimiser state, runs the problem's own minimiser loop (its own kernels,
 * launch shapes and device-side stop rule, nested as a conditional node) and
 * records the result.  No host work per field value; the GPU interleaves the
 * branches.  Every problem's results equal its own mm_hysteresis_sweep bit
 * for bit.
 * MM_BATCH_GROUPED (every problem film-layout, MM_FP64 or MM_FP32, else
 * MM_ERR_UNSUPPORTED): one sweep call is ONE graph launch.  Its device-side
 * loop runs one minimiser iteration of every problem still running per pass
 * -- one grouped kernel launch per stage and precision over the work items
 * of all those problems -- and each problem moves on to its next field value
 * as soon as its minimisation at the current one ends, so problems advance
 * at their own pace.  Each work item runs the problem's own kernel body with
 * the problem's own tile, partial sums and state, so every problem's results
 * equal its own mm_hysteresis_sweep bit for bit.  Creation gives all members
 * of a precision the tile thread counts of the largest member (one CTA shape
 * per grouped launch): it may change the launch shapes of smaller members,
 * and recaptures their minimiser graphs, so their later single sweeps use
 * the same shapes.
 * MM_BATCH_STREAMS (any problems): each problem keeps its own minimiser graph
 * and gets a stream of its own; for every field value the batch issues every
 * problem's minimisation on its stream from the host.
 * mm_batch_create(_kind) returns MM_ERR_ARG for a null or repeated problem
 * (one problem's buffers cannot serve two work lists), for one whose setup
 * did not finish and for an unknown kind; the batch owns its tables, graph or
 * streams, released by mm_batch_destroy.  mm_batch_kind returns the kind a
 * batch runs (MM_BATCH_BRANCHES, _GROUPED or _STREAMS).
 *
 * mm_batch_sweep: as mm_hysteresis_sweep for every problem i with the same
 * field list H_list[n][3] (host, A/m): m_list[i] (host or device, in/out) is
 * problem i's magnetisation; mavg (host) [nprob][n][3]; per_step (host,
 * nullable) [nprob][n].  Work is ordered after earlier work on `stream`, and
 * `stream` is synchronised before returning.  Returns MM_OK if every
 * minimisation converged, else the first non-OK status.
 */
enum { MM_BATCH_AUTO = 0, MM_BATCH_BRANCHES = 1, MM_BATCH_GROUPED = 2, MM_BATCH_STREAMS = 3 };
typedef struct mm_batch mm_batch;
MM_API int mm_batch_create(mm_problem *const *probs, int nprob, mm_batch **out);
MM_API int mm_batch_create_kind(mm_problem *const *probs, int nprob, int kind, mm_batch **out);
MM_API int mm_batch_kind(const mm_batch *batch);
MM_API int mm_batch_destroy(mm_batch *batch);
MM_API int mm_batch_sweep(mm_batch *batch, void *const *m_list, const double *H_list, int n, int start,
                          const mm_min_opts *opts, double *mavg, mm_min_result *per_step, void *stream);

/* Sizes of a problem, for reporting and for callers that size buffers. */
typedef struct {
    int nx, ny, nz;
    int px, py, pz;            /* zero-padded FFT grid */
    int precision;
    long cells;
    long workspace_bytes;      /* device memory owned by the problem */
    long spectrum_bytes;       /* one padded field spectrum (3 components, x-half) */
    long tensor_bytes;         /* stored demagnetisation tensor (transformed; layout depends on bulk_layout) */
    int x_tile_rows;           /* launch shape picked by the setup autotuner: y rows per x-inverse CTA */
    int yz_batch_rows;         /* ... and y rows transformed together in the y-z kernel */
    int bulk_layout;           /* 1: y-z stage in three passes (bulk grids), 0: one film kernel */
    int x_fwd_tile_rows;       /* y rows per x-forward CTA (tuned separately) */
} mm_info;
MM_API int mm_problem_info(const mm_problem *prob, mm_info *info);

/*
 * mm_kernel_times -- instrumentation: evaluate H_eff plus one minimiser step
 * `reps` times on `stream` with CUDA events around each kernel, and report the
 * average device time of each kernel stage in ms.  names[i] are static
 * strings.  Used by the benchmark to turn algorithmic bytes/flops into
 * achieved rates.  *count (in: capacity of the arrays; out: stages written).
 * Leaves the problem's minimiser state undefined; synchronises `stream`.
 */
MM_API int mm_kernel_times(mm_problem *prob, const void *m, const double Hext[3], int reps, double *ms_out,
                    const char **names, int *count, void *stream);

/*
 * mm_min_inspect -- instrumentation: the minimiser's device state after the
 * last mm_minimize / mm_hysteresis_sweep on this problem (the last field
 * value of a sweep).  out (host) receives the iterate index k of the last
 * evaluation, the step size tau of the step that produced iterate k (tau0 at
 * k = 0), the Barzilai-Borwein sums of Eq. (stepsize) at iterate k over all
 * cells, s.s, s.y and y.y with s = m_k - m_{k-1} and y = g_k - g_{k-1}
 * (zero at k = 0), max_i |m_i x H_i| / Ms at iterate k and the mm_status of
 * that minimisation.  m_k, m_prev, g_k, g_prev (host or device, nullable,
 * problem precision, [3][nz][ny][nx]) receive m_k, m_{k-1}, g_k = m_k x
 * (m_k x H_k) and g_{k-1} as the kernels hold them (MM_F32X2: the
 * double-float pairs rounded to double; m_prev, g_prev
 * meaningful for k >= 1).  Lets callers check the step-size sums against
 * their own reduction of the same data.  Synchronises `stream`.
 */
typedef struct {
    long k;
    int status;
    double tau;
    double ss, sy, yy;
    double max_torque;
} mm_min_state;
MM_API int mm_min_inspect(mm_problem *prob, mm_min_state *out, void *m_k, void *m_prev, void *g_k, void *g_prev,
                          void *stream);

/*
 * mm_probe_fma -- instrumentation: measured fused-multiply-add throughput of
 * the current device, tflops_out (host) [2] = FP64, FP32 in TFLOP/s (2 flops
 * per FMA), from independent FMA chains filling every SM, best of five ~5 ms
 * launches on the legacy default stream.  The double-precision field kernels
 * are bound by the FP64 units, so this is their roofline peak.  Allocates a
 * small buffer; synchronises the device.  (Instrumentation; not in the paper.)
 */
MM_API int mm_probe_fma(double tflops_out[2]);

/* Human-readable text of a status code (static string). */
MM_API const char *mm_status_string(int status);

/* Text of the last CUDA error seen by this thread inside the library (static). */
MM_API const char *mm_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MMGB_MM_H */
