// Batched hysteresis sweeps (an extension; the paper runs one sample at a
// time): many independent problems, of uneven grid sizes and each with the
// launch shapes its own setup autotuner picked, swept together.
//
// Grouped launch (film-layout problems, the case of thin films).  For every
// field value the batch runs ONE graph launch: an init kernel sets every
// problem's minimiser state, then a conditional WHILE node loops over one
// minimiser iteration of ALL problems -- one grouped launch per kernel stage
// and precision (x-forward with the step, y-z convolution, x-inverse with the
// local terms and step-size sums) whose CTAs are the work items of every
// problem still running -- and a one-thread kernel that keeps the loop going
// while any problem runs; a record kernel stores every problem's result.
// Each work item runs the same device body as the problem's own kernel with
// the problem's own tile shape and thread count (CTAs are sized for the
// largest problem; the spare threads only join the barriers), and each
// problem keeps its own partial sums, counter and state, so every problem's
// result equals its own single sweep bit for bit.  A problem that has
// converged skips its work items until the field value ends.
//
// Branch graph (the default; any problems): one sweep call is ONE graph
// launch whose graph holds one independent branch per problem: a
// conditional WHILE node over the problem's field values whose body sets the
// minimiser state for the next value, runs the problem's own minimiser loop
// (a nested conditional WHILE node around its three kernels, the same body
// as its own minimiser graph) and records the result.  The branches share
// nothing, so the GPU interleaves the problems' kernels as it would
// independent streams, with no host launch per field value.
//
// Stream path: each problem's own minimiser graph on a stream of its own,
// all streams issued per field value so the problems overlap on the GPU.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "field_kernels.cuh"

namespace {

// one problem of a grouped launch, as the grouped kernels read it
template <typename T>
struct GFilm {
    Geom g;
    FieldPtrs<T> P;
    int nth_xf, nth_x, nth_yz;   // working threads of the three stages (the problem's own launch shapes)
    int gx_x, nblk_x;            // x-inverse grid: CTAs along y, CTAs in all
    int first[3], count[3];      // the problem's work items of each stage (x-forward, y-z, x-inverse)
};

// Problems still running in this iteration, as a compacted work list: the
// grouped kernels are persistent and walk virtual item indices 0 ..
// prefix[s][nact] - 1 of stage s; index v belongs to films[a] for the a with
// prefix[s][a] <= v < prefix[s][a + 1].  Layout in device memory:
// nact, films[nf], prefix[3][nf + 1] (ints).
struct GActive {
    int *base;
    int nf;
    __device__ int &nact() const { return base[0]; }
    __device__ int *films() const { return base + 1; }
    __device__ int *prefix(int s) const { return base + 1 + nf + s * (nf + 1); }
};

struct GItem { int film, bx, by; };

// A problem group as the init and advance kernels see it.  The descriptor
// layout does not depend on the field type (Geom, then pointers), so both
// precisions are read through the double view for the state and item counts.
struct GActive;


// per problem and sweep call: what the init kernel writes into its state
struct GInit {
    MinState *st;
    StepRecord *rec;
    double tau0, tol_abs;
    int j;                       // field value this problem is minimising (n once it is done)
};

// options of a sweep call, read by the init and advance kernels
struct GCtl {
    int n, start;                // field values H[start .. n-1]
    long max_iter;
    int step_kind, tau_rule;
    unsigned long long timeout_ns;
    double kappa;
};

template <typename T>
__device__ __forceinline__ void load_film(GFilm<T> &f, const GFilm<T> *src)
{
    const int nw = (int)(sizeof(GFilm<T>) / sizeof(int));
    for (int i = threadIdx.x; i < nw; i += blockDim.x)
        reinterpret_cast<int *>(&f)[i] = reinterpret_cast<const int *>(src)[i];
    __syncthreads();
}

// the work item behind virtual index v of stage s (binary search over the
// active problems' prefix sums)
struct GRef {
    const GFilm<double> *films;
    int nf;
    GActive act;
};
static_assert(sizeof(GFilm<double>) == sizeof(GFilm<float>), "descriptor layout is precision independent");

__device__ __forceinline__ GItem active_item(const GActive &A, const int *first, const GItem *items, int s, int v)
// first[s * nf + f]: where problem f's items start in stage s's item array
{
    const int *pre = A.prefix(s);
    int lo = 0, hi = A.nact() - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= v) lo = mid; else hi = mid - 1;
    }
    const int f = A.films()[lo];
    return items[first[s * A.nf + f] + (v - pre[lo])];
}

// Persistent grouped kernels: CTA b takes virtual items b, b + gridDim.x, ...
// of the problems still running.  Items of a stage are independent, so the
// order does not matter; the shared memory is reused item after item.
#define MM_GROUP_LOOP(STAGE)                                                                  \
    __shared__ __align__(16) GFilm<T> f;                                                      \
    const int total = A.prefix(STAGE)[A.nact()];                                              \
    for (int v = blockIdx.x; v < total; v += gridDim.x) {                                    \
        __syncthreads();                                                                      \
        const GItem it = active_item(A, first_of, items, STAGE, v);                           \
        load_film(f, films + it.film);

template <typename T>
__global__ void __launch_bounds__(768) k_xfwd_group(const GFilm<T> *films, const GItem *items, const int *first_of,
                                                    GActive A)
{
    MM_GROUP_LOOP(0)
        switch (lc_of(f.g.lhx)) {
#define C(L) case L: xfwd_body<T, T, true, L>(f.g, f.P, threadIdx.x, f.nth_xf, it.bx, it.by); break;
            MM_LC_CASES(C)
#undef C
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(YZBound<T>::v) k_yz_group(const GFilm<T> *films, const GItem *items,
                                                            const int *first_of, GActive A)
{
    MM_GROUP_LOOP(1)
    switch (f.g.Pz * 16 + lc_of(f.g.lpy)) {
#define C(L) case 1 * 16 + L: yz_body<T, T, 1, L>(f.g, f.P, threadIdx.x, f.nth_yz, it.bx); break; \
             case 4 * 16 + L: yz_body<T, T, 4, L>(f.g, f.P, threadIdx.x, f.nth_yz, it.bx); break; \
             case 8 * 16 + L: yz_body<T, T, 8, L>(f.g, f.P, threadIdx.x, f.nth_yz, it.bx); break;
        MM_LC_CASES(C)
#undef C
    }
    }
}

template <typename T>
__global__ void __launch_bounds__(768) k_xinv_group(const GFilm<T> *films, const GItem *items, const int *first_of,
                                                    GActive A)
{
    MM_GROUP_LOOP(2)
        const int bid = it.by * f.gx_x + it.bx;
        switch (lc_of(f.g.lhx)) {
#define C(L) case L: xinv_body<T, T, MODE_MIN, L>(f.g, f.P, 0.0, 0.0, 0.0, 0, 0, threadIdx.x, f.nth_x, it.bx, it.by, \
                                                    bid, f.nblk_x); break;
            MM_LC_CASES(C)
#undef C
        }
    }
}

// compacted work lists of the problems still running (one CTA); `first`
// lists, per problem, where its items start in each stage's item array
__device__ void build_active(const GFilm<double> *films, int nf, GActive A)
{
    if (threadIdx.x != 0 || nf == 0) return;
    int na = 0;
    int *pre0 = A.prefix(0), *pre1 = A.prefix(1), *pre2 = A.prefix(2);
    pre0[0] = pre1[0] = pre2[0] = 0;
    for (int f = 0; f < nf; ++f) {
        if (films[f].P.st->status != MMS_RUNNING) continue;
        A.films()[na] = f;
        pre0[na + 1] = pre0[na] + films[f].count[0];
        pre1[na + 1] = pre1[na] + films[f].count[1];
        pre2[na + 1] = pre2[na] + films[f].count[2];
        ++na;
    }
    A.nact() = na;
}

// the minimiser state of problem i for field value j, as k_init_state sets
// it for one problem (the first field value of a sweep call starts from the
// iterate in buffer 0; later ones continue from the last iterate)
__device__ void init_one(GInit *init, int i, int j, const double *H, const GCtl &c)
{
    MinState *st = init[i].st;
    if (j == c.start) st->base = 0;
    else st->base = st->base ^ (int)(st->k & 1);
    const double h0 = H[3 * j], h1 = H[3 * j + 1], h2 = H[3 * j + 2];
    st->tau0 = init[i].tau0; st->tol_abs = init[i].tol_abs;
    st->Hext[0] = h0; st->Hext[1] = h1; st->Hext[2] = h2;
    st->Hextf[0] = (float)h0; st->Hextf[1] = (float)h1; st->Hextf[2] = (float)h2;
    st->Hextw[0] = dfloat(h0); st->Hextw[1] = dfloat(h1); st->Hextw[2] = dfloat(h2);
    st->max_iter = c.max_iter; st->step_kind = c.step_kind;
    st->tau_rule = c.tau_rule; st->kappa = c.kappa;
    st->timeout_ns = c.timeout_ns; st->t_start_ns = 0;
    st->k = 0; st->tau = init[i].tau0; st->tauf = (float)init[i].tau0; st->tauw = dfloat(init[i].tau0); st->status = MMS_RUNNING; st->evals = 0;
    st->launches = 1;
    st->max_torque = 0;
    init[i].j = j;
}

// before the loop: every problem at the sweep's first field value
__global__ void k_group_init(GInit *init, int n, const double *H, const GCtl *ctl, const GRef *refs, int nrefs)
{
    const GCtl c = *ctl;
    for (int i = threadIdx.x; i < n; i += blockDim.x) init_one(init, i, c.start, H, c);
    __syncthreads();
    for (int r = 0; r < nrefs; ++r) build_active(refs[r].films, refs[r].nf, refs[r].act);
}

// After every iteration: each problem whose minimisation at its field value
// ended (converged, or stopped by its iteration cap, time limit or a
// non-finite value) records that field value and starts its next one, so
// problems advance through the sweep at their own pace; then the work lists
// of the next iteration, and the loop goes on while any problem runs.
__global__ void k_group_advance(GInit *init, int n, const double *H, const GCtl *ctl, const GRef *refs, int nrefs,
                                cudaGraphConditionalHandle h)
{
    const GCtl c = *ctl;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const MinState *st = init[i].st;
        const int j = init[i].j;
        if (st->status == MMS_RUNNING || j >= c.n) continue;
        StepRecord r;
        r.mavg[0] = st->mavg[0]; r.mavg[1] = st->mavg[1]; r.mavg[2] = st->mavg[2];
        r.max_torque = st->max_torque; r.energy = st->energy[4];
        r.iters = st->k; r.evals = st->evals; r.launches = st->launches + 1; r.status = st->status;
        init[i].rec[j] = r;
        if (j + 1 < c.n) init_one(init, i, j + 1, H, c);
        else init[i].j = c.n;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    int active = 0;
    for (int r = 0; r < nrefs; ++r) {
        build_active(refs[r].films, refs[r].nf, refs[r].act);
        if (refs[r].nf) active += refs[r].act.nact();
    }
    cudaGraphSetConditional(h, active > 0 ? 1u : 0u);
}

// Branch graph: problem i's next field value (its index init[i].j), and the
// nested minimiser loop's condition set to run
__global__ void k_branch_init(GInit *init, int i, const double *H, const GCtl *ctl, cudaGraphConditionalHandle inner)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    init_one(init, i, init[i].j, H, *ctl);
    cudaGraphSetConditional(inner, 1u);
}

// Branch graph: record problem i's field value and go on while values remain
__global__ void k_branch_record(GInit *init, int i, const GCtl *ctl, cudaGraphConditionalHandle outer)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const MinState *st = init[i].st;
    const int j = init[i].j;
    StepRecord r;
    r.mavg[0] = st->mavg[0]; r.mavg[1] = st->mavg[1]; r.mavg[2] = st->mavg[2];
    r.max_torque = st->max_torque; r.energy = st->energy[4];
    r.iters = st->k; r.evals = st->evals; r.launches = st->launches + 1; r.status = st->status;
    init[i].rec[j] = r;
    init[i].j = j + 1;
    cudaGraphSetConditional(outer, j + 1 < ctl->n ? 1u : 0u);
}

// device tables of one precision group
template <typename T>
struct Group {
    std::vector<int> members;        // indices into the batch's problem list
    std::vector<GFilm<T>> host;      // host copy of the descriptors (refreshed at every sweep)
    GFilm<T> *films = nullptr;
    GItem *items_xf = nullptr, *items_yz = nullptr, *items_x = nullptr;
    int *first = nullptr;            // [3][nf]: where each problem's items start per stage
    GActive act = {nullptr, 0};      // compacted work lists of the running problems
    int grid_xf = 1, grid_yz = 1, grid_x = 1;   // persistent grids (resident CTAs on every SM)
    int n_xf = 0, n_yz = 0, n_x = 0;
    int thr_xf = 32, thr_yz = 32, thr_x = 32;
    size_t sm_xf = 0, sm_yz = 0, sm_x = 0;
};

} // namespace

struct mm_batch {
    std::vector<mm_problem *> probs;
    int kind = MM_BATCH_BRANCHES;
    std::vector<int> gens;       // branch graph: the members' graph generations it was built from
    // stream path (bulk-layout problems present)
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t start_ev = nullptr;
    // grouped path
    // groups by precision and size class: large problems (>= 65536 cells)
    // and small ones; each group's stages run as a branch of its own in the
    // loop body, so the groups' kernels overlap on the GPU
    std::vector<Group<double>> g64;
    std::vector<Group<float>> g32;
    GRef *refs_dev = nullptr;
    int nrefs = 0;
    GInit *init_dev = nullptr;   // [nprob]
    GCtl *ctl_dev = nullptr;
    double *H_dev = nullptr;     // [cap][3]
    int H_cap = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond = 0;
};

namespace {

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

template <typename T> void free_group(Group<T> &G)
{
    if (G.films) cudaFree(G.films);
    if (G.items_xf) cudaFree(G.items_xf);
    if (G.items_yz) cudaFree(G.items_yz);
    if (G.items_x) cudaFree(G.items_x);
    if (G.first) cudaFree(G.first);
    if (G.act.base) cudaFree(G.act.base);
    G = Group<T>();
}

void free_batch(mm_batch *b)
{
    for (auto st : b->streams) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
    for (auto ev : b->done) cudaEventDestroy(ev);
    if (b->start_ev) cudaEventDestroy(b->start_ev);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto &G : b->g64) free_group(G);
    for (auto &G : b->g32) free_group(G);
    if (b->refs_dev) cudaFree(b->refs_dev);
    if (b->init_dev) cudaFree(b->init_dev);
    if (b->ctl_dev) cudaFree(b->ctl_dev);
    if (b->H_dev) cudaFree(b->H_dev);
    delete b;
}

template <typename T> cudaError_t upload(T **dst, const std::vector<T> &v)
{
    cudaError_t e = cudaMalloc((void **)dst, sizeof(T) * (v.size() ? v.size() : 1));
    if (!e && !v.empty()) e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    return e;
}

// The group's tables: one descriptor per problem (its Geom, buffers and
// launch shapes, as its own kernels are launched) and the work items of each
// stage, largest problems first.  Every grouped launch takes the largest
// thread count and shared memory of its stage.
template <typename T> cudaError_t build_group(mm_batch *b, Group<T> &G)
{
    // largest problems first: they lead every stage's work list
    std::stable_sort(G.members.begin(), G.members.end(),
                     [&](int a, int c) { return b->probs[a]->g.N > b->probs[c]->g.N; });
    const int nf = (int)G.members.size();
    std::vector<GFilm<T>> films(nf);
    std::vector<GItem> ixf, iyz, ix;
    std::vector<int> first(3 * (size_t)nf);
    for (int f = 0; f < nf; ++f) {
        mm_problem *p = b->probs[G.members[f]];
        const Geom &g = p->g;
        GFilm<T> &d = films[f];
        memset((void *)&d, 0, sizeof d);
        d.g = g;
        d.P = make_ptrs<T>(p);
        d.nth_xf = threads_xf<T>(g);
        d.nth_x = threads_x<T>(g);
        d.nth_yz = threads_yz<T>(g);
        d.gx_x = (g.ny + g.TY - 1) / g.TY;
        d.nblk_x = d.gx_x * g.nz;
        G.thr_xf = std::max(G.thr_xf, d.nth_xf);
        G.thr_x = std::max(G.thr_x, d.nth_x);
        G.thr_yz = std::max(G.thr_yz, d.nth_yz);
        G.sm_xf = std::max(G.sm_xf, smem_xf_t<T>(g));
        G.sm_x = std::max(G.sm_x, smem_x_t<T>(g));
        G.sm_yz = std::max(G.sm_yz, smem_yz_t<T>(g));
        const int gxf = (g.ny + g.TYF - 1) / g.TYF, gx = d.gx_x;
        first[0 * nf + f] = d.first[0] = (int)ixf.size();
        for (int z = 0; z < g.nz; ++z)
            for (int y = 0; y < gxf; ++y) ixf.push_back({f, y, z});
        first[1 * nf + f] = d.first[1] = (int)iyz.size();
        for (int k = 0; k < g.C; ++k) iyz.push_back({f, k, 0});
        first[2 * nf + f] = d.first[2] = (int)ix.size();
        for (int z = 0; z < g.nz; ++z)
            for (int y = 0; y < gx; ++y) ix.push_back({f, y, z});
        d.count[0] = (int)ixf.size() - d.first[0];
        d.count[1] = (int)iyz.size() - d.first[1];
        d.count[2] = (int)ix.size() - d.first[2];
    }
    G.n_xf = (int)ixf.size(); G.n_yz = (int)iyz.size(); G.n_x = (int)ix.size();
    G.host = films;
    cudaError_t e;
    if ((e = upload(&G.films, films)) || (e = upload(&G.items_xf, ixf)) || (e = upload(&G.items_yz, iyz)) ||
        (e = upload(&G.items_x, ix)) || (e = upload(&G.first, first)))
        return e;
    G.act.nf = nf;
    if ((e = cudaMalloc((void **)&G.act.base, sizeof(int) * (1 + nf + 3 * ((size_t)nf + 1))))) return e;
    if ((e = cudaMemset(G.act.base, 0, sizeof(int) * (1 + nf + 3 * ((size_t)nf + 1))))) return e;
    if (nf == 0) return cudaSuccess;
    if (G.sm_xf > MM_SMEM_CAP || G.sm_yz > MM_SMEM_CAP || G.sm_x > MM_SMEM_CAP) return cudaErrorInvalidValue;
    if ((e = cudaFuncSetAttribute(k_xfwd_group<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, MM_SMEM_CAP)) ||
        (e = cudaFuncSetAttribute(k_yz_group<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, MM_SMEM_CAP)) ||
        (e = cudaFuncSetAttribute(k_xinv_group<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, MM_SMEM_CAP)))
        return e;
    // persistent grids: as many CTAs as are resident on all SMs at once
    int r0 = 0, r1 = 0, r2 = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r0, k_xfwd_group<T>, G.thr_xf, G.sm_xf)) ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r1, k_yz_group<T>, G.thr_yz, G.sm_yz)) ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r2, k_xinv_group<T>, G.thr_x, G.sm_x)))
        return e;
    const int sms = mm_sm_count();
    G.grid_xf = std::max(1, std::min(G.n_xf, sms * std::max(1, r0)));
    G.grid_yz = std::max(1, std::min(G.n_yz, sms * std::max(1, r1)));
    G.grid_x = std::max(1, std::min(G.n_x, sms * std::max(1, r2)));
    return cudaSuccess;
}

// refresh the descriptors from the problems (a problem's per-cell anisotropy
// buffer may have been replaced since the batch was made)
template <typename T> cudaError_t refresh_group(mm_batch *b, Group<T> &G, cudaStream_t s)
{
    if (G.members.empty()) return cudaSuccess;
    for (size_t f = 0; f < G.members.size(); ++f) G.host[f].P = make_ptrs<T>(b->probs[G.members[f]]);
    return cudaMemcpyAsync(G.films, G.host.data(), sizeof(GFilm<T>) * G.host.size(), cudaMemcpyHostToDevice, s);
}

template <typename T> void launch_group(const Group<T> &G, cudaStream_t s)
{
    if (G.members.empty()) return;
    k_xfwd_group<T><<<G.grid_xf, G.thr_xf, G.sm_xf, s>>>(G.films, G.items_xf, G.first, G.act);
    k_yz_group<T><<<G.grid_yz, G.thr_yz, G.sm_yz, s>>>(G.films, G.items_yz, G.first, G.act);
    k_xinv_group<T><<<G.grid_x, G.thr_x, G.sm_x, s>>>(G.films, G.items_x, G.first, G.act);
}

// graph of a whole sweep call: init -> WHILE { grouped stages of both
// precisions; advance }.  One graph launch minimises every problem at every
// field value of the call.
int build_batch_graph(mm_batch *b)
{
    const int n = (int)b->probs.size();
    const int ng = (int)(b->g64.size() + b->g32.size());
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e) { mm_set_cuda_error(e, "cudaStreamCreate"); return MM_ERR_CUDA; }
    std::vector<cudaStream_t> br(ng, nullptr);
    std::vector<cudaEvent_t> ev(ng + 1, nullptr);
    do {
        for (int i = 0; i < ng && !e; ++i) e = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking);
        for (int i = 0; i <= ng && !e; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        if (e) break;
        if ((e = cudaGraphCreate(&b->graph, 0))) break;
        if ((e = cudaGraphConditionalHandleCreate(&b->cond, b->graph, 1, cudaGraphCondAssignDefault))) break;
        if ((e = cudaStreamBeginCaptureToGraph(cs, b->graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed))) break;
        k_group_init<<<1, 256, 0, cs>>>(b->init_dev, n, b->H_dev, b->ctl_dev, b->refs_dev, b->nrefs);
        cudaGraph_t g0 = b->graph;
        if ((e = cudaStreamEndCapture(cs, &g0))) break;
        cudaGraphNode_t init_node;
        size_t nn = 1;
        if ((e = cudaGraphGetNodes(b->graph, &init_node, &nn)) || nn != 1) { if (!e) e = cudaErrorUnknown; break; }
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = b->cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t cond_node;
        if ((e = cudaGraphAddNode(&cond_node, b->graph, &init_node, nullptr, 1, &np))) break;
        cudaGraph_t body = np.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed))) break;
        // one branch per group: fork from the capture stream, join before the advance kernel
        cudaEventRecord(ev[ng], cs);
        int gi = 0;
        for (auto &G : b->g64) {
            cudaStreamWaitEvent(br[gi], ev[ng], 0);
            launch_group(G, br[gi]);
            cudaEventRecord(ev[gi], br[gi]);
            ++gi;
        }
        for (auto &G : b->g32) {
            cudaStreamWaitEvent(br[gi], ev[ng], 0);
            launch_group(G, br[gi]);
            cudaEventRecord(ev[gi], br[gi]);
            ++gi;
        }
        for (int i = 0; i < ng; ++i) cudaStreamWaitEvent(cs, ev[i], 0);
        k_group_advance<<<1, 256, 0, cs>>>(b->init_dev, n, b->H_dev, b->ctl_dev, b->refs_dev, b->nrefs, b->cond);
        cudaGraph_t g1 = body;
        const cudaError_t le = cudaGetLastError();
        e = cudaStreamEndCapture(cs, &g1);
        if (le) { e = le; break; }
        if (e) break;
        if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0))) break;
    } while (0);
    for (auto x : br) if (x) cudaStreamDestroy(x);
    for (auto x : ev) if (x) cudaEventDestroy(x);
    cudaStreamDestroy(cs);
    if (e) { mm_set_cuda_error(e, "batch graph"); return MM_ERR_CUDA; }
    return MM_OK;
}

// Branch graph: per problem a WHILE over its field values { init; WHILE
// { its three minimiser kernels }; record }, the branches independent.
int build_branch_graph(mm_batch *b)
{
    const int n = (int)b->probs.size();
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e) { mm_set_cuda_error(e, "cudaStreamCreate"); return MM_ERR_CUDA; }
    int rc = MM_OK;
    auto while_node = [](cudaGraph_t g, cudaGraphConditionalHandle h, const cudaGraphNode_t *dep, size_t ndep,
                         cudaGraphNode_t *node, cudaGraph_t *body) -> cudaError_t {
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaError_t err = cudaGraphAddNode(node, g, dep, nullptr, ndep, &np);
        if (!err) *body = np.conditional.phGraph_out[0];
        return err;
    };
    do {
        if ((e = cudaGraphCreate(&b->graph, 0))) break;
        for (int i = 0; i < n && !e && rc == MM_OK; ++i) {
            mm_problem *p = b->probs[i];
            // outer loop over field values: runs at least once per launch (default 1)
            cudaGraphConditionalHandle ho, hi;
            cudaGraphNode_t outer, init_node, inner;
            cudaGraph_t obody, ibody;
            if ((e = cudaGraphConditionalHandleCreate(&ho, b->graph, 1, cudaGraphCondAssignDefault))) break;
            if ((e = while_node(b->graph, ho, nullptr, 0, &outer, &obody))) break;
            if ((e = cudaGraphConditionalHandleCreate(&hi, obody, 0, 0))) break;
            if ((e = cudaStreamBeginCaptureToGraph(cs, obody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed))) break;
            k_branch_init<<<1, 32, 0, cs>>>(b->init_dev, i, b->H_dev, b->ctl_dev, hi);
            cudaGraph_t out = obody;
            if ((e = cudaStreamEndCapture(cs, &out))) break;
            size_t nn = 1;
            if ((e = cudaGraphGetNodes(obody, &init_node, &nn)) || nn != 1) { if (!e) e = cudaErrorUnknown; break; }
            if ((e = while_node(obody, hi, &init_node, 1, &inner, &ibody))) break;
            if ((e = cudaStreamBeginCaptureToGraph(cs, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed))) break;
            const int lr = mm_launch_min_body(p, hi, cs, 1);
            out = ibody;
            e = cudaStreamEndCapture(cs, &out);
            if (lr != MM_OK) { rc = lr; break; }
            if (e) break;
            if ((e = cudaStreamBeginCaptureToGraph(cs, obody, &inner, nullptr, 1, cudaStreamCaptureModeRelaxed))) break;
            k_branch_record<<<1, 32, 0, cs>>>(b->init_dev, i, b->ctl_dev, ho);
            out = obody;
            const cudaError_t le = cudaGetLastError();
            e = cudaStreamEndCapture(cs, &out);
            if (le) e = le;
        }
        if (e || rc != MM_OK) break;
        if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0))) break;
    } while (0);
    cudaStreamDestroy(cs);
    if (e || rc != MM_OK) {
        if (e) mm_set_cuda_error(e, "batch branch graph");
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
        return rc != MM_OK ? rc : MM_ERR_CUDA;
    }
    b->gens.clear();
    for (auto *p : b->probs) b->gens.push_back(p->graph_gen);
    return MM_OK;
}

// One CTA shape per grouped launch: every member of a precision group takes
// the tile whose thread count is the largest not above that of the group's
// largest problem (which carries most of the work and keeps its own tuned
// tiles).  Without this, a launch sized for the widest tile of some small
// problem runs the large problem's items with most threads idle and one CTA
// per SM.  A member whose tiles change gets its minimiser graph recaptured,
// so its single sweeps use the same tiles (and give the same results) as
// its part of the batch.
int harmonise_tiles(mm_batch *b, const std::vector<int> &members)
{
    if (members.size() < 2) return MM_OK;
    mm_problem *big = b->probs[members[0]];
    for (int i : members)
        if (b->probs[i]->g.N > big->g.N) big = b->probs[i];
    const bool dbl = mm_double_fields(big);
    const int nxf = dbl ? threads_xf<double>(big->g) : threads_xf<float>(big->g);
    const int nx = dbl ? threads_x<double>(big->g) : threads_x<float>(big->g);
    const int nyz = big->g.RB * big->g.Gy;
    for (int i : members) {
        mm_problem *p = b->probs[i];
        if (p == big) continue;
        Geom g = p->g;
        int tyf = p->tys[0], ty = p->tys[0], rb = p->rbs[p->nrb - 1];
        for (int k = 0; k < p->nty; ++k) {   // ascending powers of two
            Geom t = g;
            t.TYF = t.TY = p->tys[k];
            if ((dbl ? threads_xf<double>(t) : threads_xf<float>(t)) <= nxf) tyf = p->tys[k];
            if ((dbl ? threads_x<double>(t) : threads_x<float>(t)) <= nx) ty = p->tys[k];
        }
        for (int k = p->nrb - 1; k >= 0; --k)  // descending: keep the largest that fits
            if (p->rbs[k] * g.Gy <= nyz) { rb = p->rbs[k]; }
        if (tyf == g.TYF && ty == g.TY && rb == g.RB) continue;
        g.TYF = tyf; g.ltyf = mm_ilog2(tyf);
        g.TY = ty; g.lty = mm_ilog2(ty);
        g.RB = rb;
        p->g = g;
        const int rc = mm_rebuild_graph(p);
        if (rc) return rc;
    }
    return MM_OK;
}

int create_grouped(mm_batch *b)
{
    // groups by precision and size class (the setup autotuner's threshold):
    // large problems keep their tuned tiles and carry most of the work; small
    // ones share wider tiles; each group's stages form a branch of their own
    std::vector<int> m64[2], m32[2];
    for (size_t i = 0; i < b->probs.size(); ++i) {
        const int large = b->probs[i]->g.N >= 65536;
        (b->probs[i]->precision == MM_FP64 ? m64[large] : m32[large]).push_back((int)i);
    }
    for (int c = 1; c >= 0; --c) {
        if (!m64[c].empty()) { b->g64.emplace_back(); b->g64.back().members = m64[c]; }
        if (!m32[c].empty()) { b->g32.emplace_back(); b->g32.back().members = m32[c]; }
    }
    int rc;
    for (auto &G : b->g64) if ((rc = harmonise_tiles(b, G.members))) return rc;
    for (auto &G : b->g32) if ((rc = harmonise_tiles(b, G.members))) return rc;
    cudaError_t e = cudaSuccess;
    for (auto &G : b->g64) if (!e) e = build_group(b, G);
    for (auto &G : b->g32) if (!e) e = build_group(b, G);
    if (e) { mm_set_cuda_error(e, "batch tables"); return MM_ERR_CUDA; }
    std::vector<GRef> refs;
    for (auto &G : b->g64) refs.push_back({G.films, (int)G.members.size(), G.act});
    for (auto &G : b->g32) refs.push_back({reinterpret_cast<const GFilm<double> *>(G.films), (int)G.members.size(), G.act});
    b->nrefs = (int)refs.size();
    if ((e = upload(&b->refs_dev, refs)) ||
        (e = cudaMalloc((void **)&b->init_dev, sizeof(GInit) * b->probs.size())) ||
        (e = cudaMalloc((void **)&b->ctl_dev, sizeof(GCtl))) || (e = cudaMalloc((void **)&b->H_dev, sizeof(double) * 3))) {
        mm_set_cuda_error(e, "cudaMalloc(batch)");
        return MM_ERR_OOM;
    }
    b->H_cap = 1;
    return MM_OK;
}

int create_branches(mm_batch *b)
{
    cudaError_t e;
    if ((e = cudaMalloc((void **)&b->init_dev, sizeof(GInit) * b->probs.size())) ||
        (e = cudaMalloc((void **)&b->ctl_dev, sizeof(GCtl))) || (e = cudaMalloc((void **)&b->H_dev, sizeof(double) * 3))) {
        mm_set_cuda_error(e, "cudaMalloc(batch)");
        return MM_ERR_OOM;
    }
    b->H_cap = 1;
    return build_branch_graph(b);
}

int create_streams(mm_batch *b)
{
    if (cudaEventCreateWithFlags(&b->start_ev, cudaEventDisableTiming)) return MM_ERR_CUDA;
    for (size_t i = 0; i < b->probs.size(); ++i) {
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) return MM_ERR_CUDA;
        b->streams.push_back(st);
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) return MM_ERR_CUDA;
        b->done.push_back(ev);
    }
    return MM_OK;
}

// the per-field-value records of every problem into mavg / per_step
int collect(mm_batch *b, int n, int start, double *mavg, mm_min_result *per_step, cudaStream_t s, long launches_each)
{
    std::vector<StepRecord> rec((size_t)n);
    int first_bad = MM_OK;
    for (size_t i = 0; i < b->probs.size(); ++i) {
        cudaError_t e = cudaMemcpyAsync(rec.data() + start, b->probs[i]->rec_dev + start,
                                        sizeof(StepRecord) * (size_t)(n - start), cudaMemcpyDeviceToHost, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) { mm_set_cuda_error(e, "mm_batch_sweep"); return MM_ERR_CUDA; }
        for (int j = start; j < n; ++j) {
            const StepRecord &r = rec[j];
            double *mv = mavg + 3 * ((size_t)i * n + j);
            mv[0] = r.mavg[0]; mv[1] = r.mavg[1]; mv[2] = r.mavg[2];
            const int stt = status_of_rec(r.status);
            if (stt != MM_OK && first_bad == MM_OK) first_bad = stt;
            if (per_step) {
                mm_min_result &o = per_step[(size_t)i * n + j];
                o.iters = r.iters; o.heff_evals = r.evals; o.max_torque = r.max_torque; o.energy = r.energy;
                o.converged = r.status == MMS_CONVERGED; o.status = stt;
                o.kernel_launches = launches_each >= 0 ? launches_each : r.launches + 1 + (j == n - 1 ? 1 : 0);
            }
        }
    }
    return first_bad;
}

int sweep_streams(mm_batch *b, void *const *m_list, const double *H_list, int n, int start, const mm_min_opts *opts,
                  cudaStream_t s)
{
    const size_t P = b->probs.size();
    // fork: every problem stream waits for the caller's stream
    cudaError_t e = cudaEventRecord(b->start_ev, s);
    for (size_t i = 0; i < P && !e; ++i) e = cudaStreamWaitEvent(b->streams[i], b->start_ev, 0);
    if (e) { mm_set_cuda_error(e, "mm_batch_sweep"); return MM_ERR_CUDA; }
    // issue everything; on a failure stop issuing, but still join every
    // problem stream to the caller's stream so that no work is left unordered
    int rc = MM_OK;
    for (size_t i = 0; i < P && rc == MM_OK; ++i) {
        rc = mm_load_iterate(b->probs[i], m_list[i], mm_is_device_ptr(m_list[i]), b->streams[i]);
    }
    for (int j = start; j < n && rc == MM_OK; ++j)
        for (size_t i = 0; i < P && rc == MM_OK; ++i) {
            mm_problem *p = b->probs[i];
            cudaStream_t si = b->streams[i];
            if ((rc = mm_launch_init_state(p, H_list + 3 * j, opts, j == start, si))) break;
            if ((rc = mm_launch_loop(p, si))) break;
            rc = mm_launch_record(p, j, si);
        }
    for (size_t i = 0; i < P && rc == MM_OK; ++i) {
        mm_problem *p = b->probs[i];
        cudaStream_t si = b->streams[i];
        const size_t F = 3 * (size_t)p->g.N * p->esz;
        const bool mdev = mm_is_device_ptr(m_list[i]);
        if ((rc = mm_launch_copy_result(p, mdev ? m_list[i] : p->stage_out, si))) break;
        if (!mdev) rc = mm_copy_user(m_list[i], p->stage_out, F, false, true, si);
    }
    // join: the caller's stream waits for every problem stream
    for (size_t i = 0; i < P; ++i) {
        if ((e = cudaEventRecord(b->done[i], b->streams[i])) || (e = cudaStreamWaitEvent(s, b->done[i], 0))) {
            mm_set_cuda_error(e, "mm_batch_sweep");
            if (rc == MM_OK) rc = MM_ERR_CUDA;
        }
    }
    return rc;
}

// grouped path and branch graph: one graph launch per sweep call
int sweep_graph(mm_batch *b, void *const *m_list, const double *H_list, int n, int start, const mm_min_opts *opts,
                cudaStream_t s)
{
    const size_t P = b->probs.size();
    cudaError_t e;
    bool stale = false;   // the branch graph holds the members' kernel parameters: recapture after a member's
    if (b->kind == MM_BATCH_BRANCHES)   // own graph was recaptured (e.g. a new per-cell anisotropy buffer)
        for (size_t i = 0; i < P; ++i) stale = stale || b->gens[i] != b->probs[i]->graph_gen;
    if (stale) {
        cudaStreamSynchronize(s);
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    }
    if (b->H_cap < n) {
        // the graph bakes in the field buffer's address: recapture it with the new one
        double *nh = nullptr;
        if ((e = cudaMalloc((void **)&nh, sizeof(double) * 3 * (size_t)n))) { mm_set_cuda_error(e, "cudaMalloc"); return MM_ERR_OOM; }
        cudaStreamSynchronize(s);
        cudaFree(b->H_dev);
        b->H_dev = nh;
        b->H_cap = n;
        if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
        if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    }
    if (!b->exec) {
        int rc = b->kind == MM_BATCH_BRANCHES ? build_branch_graph(b) : build_batch_graph(b);
        if (rc) return rc;
    }
    // per-sweep tables: states, records, tau0 and the stop threshold of every problem
    std::vector<GInit> init(P);
    for (size_t i = 0; i < P; ++i) {
        mm_problem *p = b->probs[i];
        init[i].st = p->st;
        init[i].rec = p->rec_dev;
        init[i].tau0 = opts->tau0 > 0 ? opts->tau0 : 1e-2 / p->g.Ms;
        init[i].tol_abs = opts->tol * p->g.Ms;
        init[i].j = start;
    }
    GCtl ctl;
    ctl.n = n;
    ctl.start = start;
    ctl.max_iter = opts->max_iter;
    ctl.step_kind = opts->step_kind;
    ctl.tau_rule = opts->tau_rule;
    ctl.timeout_ns = opts->timeout_s > 0 ? (unsigned long long)(opts->timeout_s * 1e9) : 0ull;
    ctl.kappa = opts->tau_kappa > 0 ? opts->tau_kappa : 0.5;
    e = cudaSuccess;
    for (auto &G : b->g64) if (!e) e = refresh_group(b, G, s);   // (no groups in a branch graph)
    for (auto &G : b->g32) if (!e) e = refresh_group(b, G, s);
    if (e ||
        (e = cudaMemcpyAsync(b->init_dev, init.data(), sizeof(GInit) * P, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(b->ctl_dev, &ctl, sizeof ctl, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(b->H_dev, H_list, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, s))) {
        mm_set_cuda_error(e, "mm_batch_sweep");
        return MM_ERR_CUDA;
    }
    int rc = MM_OK;
    for (size_t i = 0; i < P && rc == MM_OK; ++i) {
        rc = mm_load_iterate(b->probs[i], m_list[i], mm_is_device_ptr(m_list[i]), s);
    }
    // the whole sweep call: one graph launch
    if (rc == MM_OK && (e = cudaGraphLaunch(b->exec, s))) { mm_set_cuda_error(e, "cudaGraphLaunch(batch)"); rc = MM_ERR_CUDA; }
    for (size_t i = 0; i < P && rc == MM_OK; ++i) {
        mm_problem *p = b->probs[i];
        const size_t F = 3 * (size_t)p->g.N * p->esz;
        const bool mdev = mm_is_device_ptr(m_list[i]);
        if ((rc = mm_launch_copy_result(p, mdev ? m_list[i] : p->stage_out, s))) break;
        if (!mdev) rc = mm_copy_user(m_list[i], p->stage_out, F, false, true, s);
    }
    return rc;
}

} // namespace

extern "C" MM_API int mm_batch_create_kind(mm_problem *const *probs, int n, int kind, mm_batch **out)
{
    if (!probs || n < 1 || !out || kind < MM_BATCH_AUTO || kind > MM_BATCH_STREAMS) return MM_ERR_ARG;
    // a problem listed twice would have its buffers used by two work lists at once
    std::vector<mm_problem *> sorted(probs, probs + n);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return MM_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!probs[i] || !probs[i]->graph_ready) return MM_ERR_ARG;
    // grouped launches serve film-layout problems in double or float
    bool all_film = true;
    for (int i = 0; i < n; ++i) all_film = all_film && !probs[i]->g.bulk && probs[i]->precision != MM_F32X2;
    if (kind == MM_BATCH_GROUPED && !all_film) return MM_ERR_UNSUPPORTED;
    mm_batch *b = new (std::nothrow) mm_batch;
    if (!b) return MM_ERR_OOM;
    b->probs.assign(probs, probs + n);
    b->kind = kind == MM_BATCH_AUTO ? MM_BATCH_BRANCHES : kind;
    int rc = b->kind == MM_BATCH_BRANCHES ? create_branches(b)
           : b->kind == MM_BATCH_GROUPED  ? create_grouped(b)
                                          : create_streams(b);
    if (rc == MM_ERR_CUDA && kind == MM_BATCH_AUTO) {
        // a runtime that cannot build the nested graph: the grouped launches
        // (film-layout problems) or the streams instead
        free_batch(b);
        cudaGetLastError();
        if (!(b = new (std::nothrow) mm_batch)) return MM_ERR_OOM;
        b->probs.assign(probs, probs + n);
        b->kind = all_film ? MM_BATCH_GROUPED : MM_BATCH_STREAMS;
        rc = all_film ? create_grouped(b) : create_streams(b);
    }
    if (rc) {
        if (rc == MM_ERR_CUDA && !mm_last_cuda_error()[0]) mm_set_cuda_error(cudaGetLastError(), "mm_batch_create");
        free_batch(b);
        return rc;
    }
    *out = b;
    return MM_OK;
}

extern "C" MM_API int mm_batch_create(mm_problem *const *probs, int n, mm_batch **out)
{
    return mm_batch_create_kind(probs, n, MM_BATCH_AUTO, out);
}

extern "C" MM_API int mm_batch_kind(const mm_batch *b) { return b ? b->kind : MM_ERR_ARG; }

extern "C" MM_API int mm_batch_destroy(mm_batch *b)
{
    if (!b) return MM_OK;
    cudaDeviceSynchronize();
    free_batch(b);
    return MM_OK;
}

extern "C" MM_API int mm_batch_sweep(mm_batch *b, void *const *m_list, const double *H_list, int n, int start,
                                     const mm_min_opts *opts, double *mavg, mm_min_result *per_step, void *stream)
{
    if (!b || !m_list || !H_list || !mavg || n < 1 || start < 0 || start >= n || !opts) return MM_ERR_ARG;
    if (!mm_opts_ok(opts)) return MM_ERR_ARG;
    for (int j = 0; j < 3 * n; ++j)
        if (!std::isfinite(H_list[j])) return MM_ERR_ARG;
    const size_t P = b->probs.size();
    for (size_t i = 0; i < P; ++i)
        if (!m_list[i]) return MM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    for (size_t i = 0; i < P; ++i)
        if ((rc = ensure_records(b->probs[i], n))) return rc;
    if (b->kind != MM_BATCH_STREAMS) {
        // the records' addresses are written per sweep into the init table,
        // after ensure_records may have moved them
        rc = sweep_graph(b, m_list, H_list, n, start, opts, s);
    } else {
        rc = sweep_streams(b, m_list, H_list, n, start, opts, s);
    }
    if (rc != MM_OK) {
        cudaStreamSynchronize(s);
        return rc;
    }
    // per problem the record keeps its own count (grouped: the grouped
    // kernels and the condition kernel are shared by all problems)
    return collect(b, n, start, mavg, per_step, s, -1);
}
