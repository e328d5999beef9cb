// Batched hysteresis sweeps (an extension; the paper runs one sample at a
// time): many independent problems, of uneven grid sizes and each with the
// launch shapes its own setup autotuner picked, swept together.
//
// Every problem keeps its own CUDA graph (the device-side minimiser loop with
// a conditional WHILE node).  The batch gives each problem a stream of its
// own and, for every field value, issues init -> graph launch -> record on
// all streams in turn; the streams are independent, so the problems'
// minimisations run concurrently and small films fill the GPU together.
// The caller's stream is joined to all of them at the start and the end.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

struct mm_batch {
    std::vector<mm_problem *> probs;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t start_ev = nullptr;
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

} // namespace

extern "C" MM_API int mm_batch_create(mm_problem *const *probs, int n, mm_batch **out)
{
    if (!probs || n < 1 || !out) return MM_ERR_ARG;
    // a problem listed twice would run on two streams over one set of buffers
    std::vector<mm_problem *> sorted(probs, probs + n);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return MM_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!probs[i] || !probs[i]->graph_ready) return MM_ERR_ARG;
    mm_batch *b = new (std::nothrow) mm_batch;
    if (!b) return MM_ERR_OOM;
    b->probs.assign(probs, probs + n);
    int rc = MM_OK;
    if (cudaEventCreateWithFlags(&b->start_ev, cudaEventDisableTiming)) rc = MM_ERR_CUDA;
    for (int i = 0; i < n && rc == MM_OK; ++i) {
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) { rc = MM_ERR_CUDA; break; }
        b->streams.push_back(st);
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) { rc = MM_ERR_CUDA; break; }
        b->done.push_back(ev);
    }
    if (rc) {
        mm_set_cuda_error(cudaGetLastError(), "mm_batch_create");
        for (auto st : b->streams) cudaStreamDestroy(st);
        for (auto ev : b->done) cudaEventDestroy(ev);
        if (b->start_ev) cudaEventDestroy(b->start_ev);
        delete b;
        return rc;
    }
    *out = b;
    return MM_OK;
}

extern "C" MM_API int mm_batch_destroy(mm_batch *b)
{
    if (!b) return MM_OK;
    for (auto st : b->streams) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
    for (auto ev : b->done) cudaEventDestroy(ev);
    if (b->start_ev) cudaEventDestroy(b->start_ev);
    delete b;
    return MM_OK;
}

extern "C" MM_API int mm_batch_sweep(mm_batch *b, void *const *m_list, const double *H_list, int n, int start,
                                     const mm_min_opts *opts, double *mavg, mm_min_result *per_step, void *stream)
{
    if (!b || !m_list || !H_list || !mavg || n < 1 || start < 0 || start >= n || !opts) return MM_ERR_ARG;
    if (!mm_opts_ok(opts))
        return MM_ERR_ARG;
    for (int j = 0; j < 3 * n; ++j)
        if (!std::isfinite(H_list[j])) return MM_ERR_ARG;
    const size_t P = b->probs.size();
    for (size_t i = 0; i < P; ++i)
        if (!m_list[i]) return MM_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int rc;
    for (size_t i = 0; i < P; ++i)
        if ((rc = ensure_records(b->probs[i], n))) return rc;
    // fork: every problem stream waits for the caller's stream
    cudaError_t e = cudaEventRecord(b->start_ev, s);
    for (size_t i = 0; i < P && !e; ++i) e = cudaStreamWaitEvent(b->streams[i], b->start_ev, 0);
    if (e) { mm_set_cuda_error(e, "mm_batch_sweep"); return MM_ERR_CUDA; }
    // issue everything; on a failure stop issuing, but still join every
    // problem stream to the caller's stream so that no work is left unordered
    rc = MM_OK;
    for (size_t i = 0; i < P && rc == MM_OK; ++i) {
        mm_problem *p = b->probs[i];
        const size_t F = 3 * (size_t)p->g.N * p->esz;
        rc = mm_copy_user(p->mbuf[0], m_list[i], F, true, mm_is_device_ptr(m_list[i]), b->streams[i]);
    }
    for (int j = start; j < n && rc == MM_OK; ++j)
        for (size_t i = 0; i < P && rc == MM_OK; ++i) {
            mm_problem *p = b->probs[i];
            cudaStream_t si = b->streams[i];
            if ((rc = mm_launch_init_state(p, H_list + 3 * j, opts, j == start, si))) break;
            e = cudaGraphLaunch(p->gexec, si);
            if (e) { mm_set_cuda_error(e, "cudaGraphLaunch(batch)"); rc = MM_ERR_CUDA; break; }
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
    if (rc != MM_OK) {
        cudaStreamSynchronize(s);
        return rc;
    }
    std::vector<StepRecord> rec((size_t)n);
    int first_bad = MM_OK;
    for (size_t i = 0; i < P; ++i) {
        e = cudaMemcpyAsync(rec.data() + start, b->probs[i]->rec_dev + start, sizeof(StepRecord) * (size_t)(n - start),
                            cudaMemcpyDeviceToHost, s);
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
                o.kernel_launches = r.launches + 1 + (j == n - 1 ? 1 : 0);
            }
        }
    }
    return first_bad;
}
