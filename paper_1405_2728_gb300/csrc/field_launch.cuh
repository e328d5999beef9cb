// Host-side launchers of the field kernels for one precision (field type T,
// FFT arithmetic F), and the entry points each precision's translation unit
// exports: the three precisions are compiled in separate units so that the
// library builds in parallel.
#pragma once

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "fft.cuh"
#include "field_kernels.cuh"

namespace {

// ---------------------------------------------------------------------------
// host-side launch helpers
// ---------------------------------------------------------------------------
template <typename T, typename F, bool MIN>
cudaError_t launch_xfwd(const Geom &g, const FieldPtrs<T, F> &P, cudaStream_t s)
{
    const dim3 grid((g.ny + g.TYF - 1) / g.TYF, g.nz);
    const int thr = threads_xf<T>(g);
    const size_t sm = smem_xf_t<T>(g);
    switch (lc_of_f<F>(g.lhx)) {
#define C(L) case L: if constexpr (lc_compiled<F>(L)) k_xfwd<T, F, MIN, L><<<grid, thr, sm, s>>>(g, P); break;
        MM_LC_CASES(C)
#undef C
    }
    return cudaGetLastError();
}

template <typename T, typename F, int MODE>
cudaError_t launch_xinv(const Geom &g, const FieldPtrs<T, F> &P, cudaStream_t s, const double *hext,
                        cudaGraphConditionalHandle h, int use_cond)
{
    const dim3 grid((g.ny + g.TY - 1) / g.TY, g.nz);
    const int thr = threads_x<T>(g);
    const size_t sm = smem_x_t<T>(g);
    const double h0 = hext ? hext[0] : 0.0, h1 = hext ? hext[1] : 0.0, h2 = hext ? hext[2] : 0.0;
    switch (lc_of_f<F>(g.lhx)) {
#define C(L) case L: if constexpr (lc_compiled<F>(L)) k_xinv<T, F, MODE, L><<<grid, thr, sm, s>>>(g, P, h0, h1, h2, h, use_cond); break;
        MM_LC_CASES(C)
#undef C
    }
    return cudaGetLastError();
}

template <typename T, typename F, int PZ>
cudaError_t launch_yz(const Geom &g, const FieldPtrs<T, F> &P, cudaStream_t s)
{
    switch (lc_of_f<F>(g.lpy)) {
#define C(L) case L: if constexpr (lc_compiled<F>(L)) k_yz<T, F, PZ, L><<<g.C, threads_yz<T>(g), smem_yz_t<T>(g), s>>>(g, P); break;
        MM_LC_CASES(C)
#undef C
    }
    return cudaGetLastError();
}

template <typename T, typename F>
cudaError_t launch_yz_any(const Geom &g, const FieldPtrs<T, F> &P, cudaStream_t s)
{
    switch (g.Pz) {
    case 1: return launch_yz<T, F, 1>(g, P, s);
    case 4: return launch_yz<T, F, 4>(g, P, s);
    case 8: return launch_yz<T, F, 8>(g, P, s);
    default: return cudaErrorInvalidValue;  // Pz = 2 does not occur (nz = 1 gives 1, nz = 2 gives 4)
    }
}

// the bulk layout's passes exist for double and float (double-word problems
// are film-layout only: the planner refuses bulk grids for them)
template <typename T, typename F>
constexpr bool has_bulk = std::is_same<T, F>::value && !std::is_same<F, dfloat>::value;

// the y-z stage: the film kernel, or the three passes of the bulk layout
template <typename T, typename F>
cudaError_t launch_conv(const Geom &g, const FieldPtrs<T, F> &P, cudaStream_t s)
{
    if constexpr (has_bulk<T, F>) {
        if (g.bulk) return mm_bulk_conv(g, P, s, -1);
    }
    return launch_yz_any<T, F>(g, P, s);
}

// the bytes a launch needs must fit the common cap, which every kernel is given
template <typename K> cudaError_t smem_attr(K *f, size_t bytes)
{
    if (bytes > (size_t)MM_SMEM_CAP) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, MM_SMEM_CAP);
}

// dynamic shared memory limits of the instances this geometry launches
template <typename T, typename F> cudaError_t configure_t(const Geom &g, size_t sxf, size_t sx, size_t syz)
{
    cudaError_t e = cudaSuccess;
    switch (lc_of_f<F>(g.lhx)) {
#define C(L)                                                                                     \
    case L:                                                                                      \
        if constexpr (lc_compiled<F>(L)) {                                                       \
            if ((e = smem_attr(k_xfwd<T, F, false, L>, sxf)) || (e = smem_attr(k_xfwd<T, F, true, L>, sxf)) || \
                (e = smem_attr(k_xinv<T, F, MODE_HEFF, L>, sx)) || (e = smem_attr(k_xinv<T, F, MODE_ENERGY, L>, sx)) || \
                (e = smem_attr(k_xinv<T, F, MODE_MIN, L>, sx)))                                     \
                return e;                                                                        \
        }                                                                                        \
        break;
        MM_LC_CASES(C)
#undef C
    }
    if (g.bulk) return cudaSuccess;
    switch (lc_of_f<F>(g.lpy)) {
#define C(L)                                                                                     \
    case L:                                                                                      \
        if constexpr (lc_compiled<F>(L)) {                                                       \
            if (g.Pz == 1) return smem_attr(k_yz<T, F, 1, L>, syz);                              \
            if (g.Pz == 4) return smem_attr(k_yz<T, F, 4, L>, syz);                              \
            if (g.Pz == 8) return smem_attr(k_yz<T, F, 8, L>, syz);                              \
        }                                                                                        \
        return cudaErrorInvalidValue;
        MM_LC_CASES(C)
#undef C
    }
    return cudaErrorInvalidValue;
}

// Launch-shape autotuner: time every admissible rows-per-tile of the
// x-forward kernel and, separately, of the x-inverse kernel (the two are
// independent: the spectrum layout does not depend on the tile), and every
// rows-per-batch RB of the y-z kernel, on this problem's own buffers
// (MM_TUNE_REPS repetitions, best taken: candidates within a few percent of
// each other otherwise swap places from run to run); keep the fastest of each.
// The kernels run in their minimiser modes on the zeroed state of a fresh
// problem.
#define MM_TUNE_REPS 5
template <typename T, typename F> cudaError_t autotune_t(mm_problem *p, const int *tys, int nty, const int *rbs, int nrb,
                                             cudaStream_t s)
{
    Geom g = p->g;
    typedef typename io_of<T>::type IO;
    FieldPtrs<T, F> P = make_ptrs<T, F>(p);
    P.m_src = (const IO *)p->mbuf[0];
    P.H_out = (IO *)p->gbuf[0];
    cudaEvent_t a, b;
    cudaError_t e;
    // a minimiser state past its first iteration, so that the step and the
    // step-size sums are part of what is timed (the zeroed buffers make it
    // arithmetic on zeros and NaNs, which costs the same)
    MinState ms;
    memset(&ms, 0, sizeof ms);
    ms.k = 1;
    ms.tau = ms.tau0 = 1e-9;
    ms.tauf = 1e-9f;
    ms.tauw = dfloat(1e-9);
    ms.max_iter = 1L << 40;
    ms.status = MMS_RUNNING;
    if ((e = cudaMemcpyAsync(p->st, &ms, sizeof ms, cudaMemcpyHostToDevice, s)) || (e = cudaStreamSynchronize(s)))
        return e;
    if ((e = cudaEventCreate(&a))) return e;
    if ((e = cudaEventCreate(&b))) { cudaEventDestroy(a); return e; }
    for (int which = 0; which < 2 && !e; ++which) {
        float best = 1e30f;
        int bty = tys[0];
        for (int i = 0; i < nty && !e; ++i) {
            if (which == 0) { g.TYF = tys[i]; g.ltyf = mm_ilog2(g.TYF); }
            else { g.TY = tys[i]; g.lty = mm_ilog2(g.TY); }
            float tmin = 1e30f;
            for (int r = 0; r < MM_TUNE_REPS && !e; ++r) {
                cudaEventRecord(a, s);
                if (which == 0) launch_xfwd<T, F, true>(g, P, s);
                else launch_xinv<T, F, MODE_MIN>(g, P, s, nullptr, 0, 0);
                cudaEventRecord(b, s);
                if ((e = cudaGetLastError()) || (e = cudaEventSynchronize(b))) break;
                float t = 0;
                cudaEventElapsedTime(&t, a, b);
                if (t < tmin) tmin = t;
            }
            if (tmin < best) { best = tmin; bty = tys[i]; }
        }
        if (which == 0) { g.TYF = bty; g.ltyf = mm_ilog2(bty); }
        else { g.TY = bty; g.lty = mm_ilog2(bty); }
    }
    float best = 1e30f;
    int brb = rbs[0];
    for (int i = 0; i < nrb && !e && !g.bulk; ++i) {
        g.RB = rbs[i];
        float tmin = 1e30f;
        for (int r = 0; r < MM_TUNE_REPS && !e; ++r) {
            cudaEventRecord(a, s);
            e = launch_yz_any<T, F>(g, P, s);
            cudaEventRecord(b, s);
            if (e || (e = cudaEventSynchronize(b))) break;
            float t = 0;
            cudaEventElapsedTime(&t, a, b);
            if (t < tmin) tmin = t;
        }
        if (tmin < best) { best = tmin; brb = rbs[i]; }
    }
    g.RB = brb;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (!e) e = cudaMemsetAsync(p->st, 0, sizeof(MinState), s);
    if (!e) e = cudaMemsetAsync(p->counter, 0, 64, s);
    if (!e) p->g = g;
    return e;
}

// Field chain for MODE_HEFF / MODE_ENERGY on caller-provided m (and H).
template <typename T, typename F>
cudaError_t heff_chain_t(mm_problem *p, const void *m, void *H, const double *hext, int mode, cudaStream_t s,
                         double hscale)
{
    const Geom &g = p->g;
    typedef typename io_of<T>::type IO;
    FieldPtrs<T, F> P = make_ptrs<T, F>(p);
    P.m_src = (const IO *)m;
    P.H_out = (IO *)H;
    P.hscale = hscale;
    cudaError_t e = launch_xfwd<T, F, false>(g, P, s);
    if (e) return e;
    if ((e = launch_conv<T, F>(g, P, s))) return e;
    if (mode == MODE_HEFF) return launch_xinv<T, F, MODE_HEFF>(g, P, s, hext, 0, 0);
    return launch_xinv<T, F, MODE_ENERGY>(g, P, s, hext, 0, 0);
}

template <typename T, typename F>
cudaError_t min_body_t(mm_problem *p, cudaGraphConditionalHandle h, cudaStream_t s, int use_cond)
{
    const Geom &g = p->g;
    FieldPtrs<T, F> P = make_ptrs<T, F>(p);
    cudaError_t e = launch_xfwd<T, F, true>(g, P, s);
    if (e) return e;
    if ((e = launch_conv<T, F>(g, P, s))) return e;
    return launch_xinv<T, F, MODE_MIN>(g, P, s, nullptr, h, use_cond);
}

template <typename T, typename F>
cudaError_t stage_times_t(mm_problem *p, int reps, double *ms, cudaStream_t s)
{
    const Geom &g = p->g;
    FieldPtrs<T, F> P = make_ptrs<T, F>(p);
    const int nst = g.bulk ? 5 : 3;
    cudaEvent_t ev[6];
    for (int i = 0; i <= nst; ++i)
        if (cudaEventCreate(&ev[i])) return cudaGetLastError();
    double acc[5] = {0, 0, 0, 0, 0};
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps && !e; ++r) {
        int i = 0;
        cudaEventRecord(ev[i++], s);
        launch_xfwd<T, F, true>(g, P, s);
        cudaEventRecord(ev[i++], s);
        if (g.bulk) {
            if constexpr (has_bulk<T, F>) {
                for (int pass = 0; pass < 3; ++pass) {
                    mm_bulk_conv(g, P, s, pass);
                    cudaEventRecord(ev[i++], s);
                }
            }
        } else {
            launch_yz_any<T, F>(g, P, s);
            cudaEventRecord(ev[i++], s);
        }
        launch_xinv<T, F, MODE_MIN>(g, P, s, nullptr, 0, 0);
        cudaEventRecord(ev[i++], s);
        if ((e = cudaGetLastError())) break;
        if ((e = cudaEventSynchronize(ev[nst]))) break;
        for (int k = 0; k < nst; ++k) {
            float t = 0;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            acc[k] += t;
        }
    }
    for (int i = 0; i <= nst; ++i) cudaEventDestroy(ev[i]);
    for (int i = 0; i < nst; ++i) ms[i] = acc[i] / (reps > 0 ? reps : 1);
    return e;
}

} // namespace

// Entry points of one precision, defined by its translation unit with
// MM_DEFINE_FIELD_ENTRIES(suffix, T, F).
#define MM_DEFINE_FIELD_ENTRIES(SFX, T, F)                                                                     \
    cudaError_t mm_fields_configure_##SFX(const Geom &g, size_t sxf, size_t sx, size_t syz)                   \
    {                                                                                                          \
        return configure_t<T, F>(g, sxf, sx, syz);                                                             \
    }                                                                                                          \
    cudaError_t mm_fields_autotune_##SFX(mm_problem *p, const int *tys, int nty, const int *rbs, int nrb,       \
                                         cudaStream_t s)                                                       \
    {                                                                                                          \
        return autotune_t<T, F>(p, tys, nty, rbs, nrb, s);                                                     \
    }                                                                                                          \
    cudaError_t mm_fields_chain_##SFX(mm_problem *p, const void *m, void *H, const double *hext, int mode,     \
                                      cudaStream_t s, double hscale)                                          \
    {                                                                                                          \
        return heff_chain_t<T, F>(p, m, H, hext, mode, s, hscale);                                             \
    }                                                                                                          \
    cudaError_t mm_fields_min_body_##SFX(mm_problem *p, cudaGraphConditionalHandle h, cudaStream_t s,          \
                                         int use_cond)                                                         \
    {                                                                                                          \
        return min_body_t<T, F>(p, h, s, use_cond);                                                            \
    }                                                                                                          \
    cudaError_t mm_fields_stage_times_##SFX(mm_problem *p, int reps, double *ms, cudaStream_t s)              \
    {                                                                                                          \
        return stage_times_t<T, F>(p, reps, ms, s);                                                            \
    }
