// Serving form: a request loop around SMP-PCA (Algorithm 1) with continuous batching.
//
// Every admitted job owns a context (its resident sketch state, Omega and scratch) on a stream of its own. Row
// blocks of many jobs arrive interleaved; each smp_serve_block enqueues the sketch of one block on its job's
// stream, so the blocks of different jobs run concurrently on the device. When a job's last block has been
// pushed (smp_serve_close) the job joins a queue that a pool of host worker threads drains: finalize, sample,
// estimate and WAltMin run on the job's stream while other jobs keep sketching. Admission is gated by a device
// memory budget: a job is admitted only if the bytes its context can hold (smp_serve_job_bytes) fit in what is
// left; otherwise SMP_EBUSY and the caller retries once running jobs have been collected. Latency is measured on
// the host from smp_serve_close to the end of the job's WAltMin.
//
// Results do not depend on the interleaving: a job's kernels touch only its own context, and every reduction in
// them has a fixed order, so a job computes the same bits alone or in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum class JobState { Streaming, Queued, Solving, Done, Failed, Cancelled };

struct Job {
    smp_job_params jp{};
    smp_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    int64_t bytes = 0;
    JobState state = JobState::Streaming;
    double* U = nullptr;   // n1 x r, S r, V n2 x r (device, binary64, one allocation)
    double* S = nullptr;
    double* V = nullptr;
    int64_t nnz = 0;
    Clock::time_point t_close, t_done;
    smp_status status = SMP_OK;
    std::string err;
};

int64_t round_up64(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

struct smp_server {
    smp_server_params p{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> ready;
    std::unordered_map<int64_t, std::unique_ptr<Job>> jobs;
    int64_t next_id = 1;
    int64_t used = 0;
    bool stopping = false;
    std::vector<std::thread> workers;
};

namespace {

// The solve chain of one closed job, on its stream (the context's calls synchronise where they need to).
void solve_job(Job* j) {
    smp_ctx* c = j->ctx;
    smp_status s = smp_sketch_finalize(c);
    int64_t nnz = 0;
    if (s == SMP_OK) s = smp_sample(c, j->jp.m, j->jp.sample_seed, &nnz);
    void* vals = nullptr;
    const size_t vbytes = (size_t)std::max<int64_t>(nnz, 1) * (c->acc_bytes == 8 ? 8 : 4);
    if (s == SMP_OK && smp::dev_malloc(&vals, vbytes, j->stream) != cudaSuccess) s = SMP_ENOMEM;
    if (s == SMP_OK) s = smp_estimate(c, vals);
    if (s == SMP_OK)
        s = smp_waltmin(c, vals, j->jp.r, j->jp.T, j->jp.flags, j->jp.walt_seed, nullptr, j->U, j->S, j->V);
    if (cudaStreamSynchronize(j->stream) != cudaSuccess && s == SMP_OK) s = SMP_ECUDA;
    smp::free_idle(vals);
    j->nnz = nnz;
    j->status = s;
    if (s != SMP_OK) j->err = smp_last_error(c);
}

void worker_loop(smp_server* sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        Job* j = nullptr;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_work.wait(lk, [&] { return sv->stopping || !sv->ready.empty(); });
            if (sv->ready.empty()) return;   // stopping and nothing left
            const int64_t id = sv->ready.front();
            sv->ready.pop_front();
            auto it = sv->jobs.find(id);
            if (it == sv->jobs.end() || it->second->state != JobState::Queued) continue;
            j = it->second.get();
            j->state = JobState::Solving;
        }
        solve_job(j);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            j->t_done = Clock::now();
            j->state = j->status == SMP_OK ? JobState::Done : JobState::Failed;
        }
        sv->cv_done.notify_all();
    }
}

void release_job(smp_server* sv, int64_t id) {   // caller holds sv->mu; the job is not running anywhere
    auto it = sv->jobs.find(id);
    if (it == sv->jobs.end()) return;
    Job* j = it->second.get();
    if (j->stream) cudaStreamSynchronize(j->stream);
    if (j->ctx) smp_destroy(j->ctx);
    smp::free_idle(j->U);   // the job's stream was synchronised above
    if (j->stream) cudaStreamDestroy(j->stream);
    sv->used -= j->bytes;
    sv->jobs.erase(it);
}

}  // namespace

extern "C" {

smp_status smp_serve_job_bytes(const smp_job_params* jp, int64_t* bytes) {
    if (!jp || !bytes) return SMP_EINVAL;
    const smp_params& p = jp->sketch;
    if (p.n1 < 1 || p.n2 < 1 || p.k < 1 || jp->r < 1 || !(jp->m > 0.0)) return SMP_EINVAL;
    const int64_t n1 = p.n1, n2 = p.n2, ntot = p.same_ab ? n1 : n1 + n2, nmax = std::max(n1, n2);
    const int64_t ldk = round_up64(p.k, 4), acc = p.dtype == SMP_F64 ? 8 : 4;
    const int64_t rows = p.max_rows ? p.max_rows : 65536;
    const int64_t r = jp->r, b = std::min<int64_t>(2 * r + 8, 72);
    // |Omega| <= sum of min(1, q) <= m (Bernoulli); capacity nnz + nnz / 8 + 1024
    const int64_t cap = (int64_t)std::ceil(jp->m) + (int64_t)std::ceil(jp->m) / 8 + 1024;
    int64_t t = 0;
    t += 9 * ntot * ldk * acc;                                  // 8 row-split partials + the finalized sketch
    t += 12 * ntot * 8 + (n1 + n2 + 2) * 8 * 3 + (n1 + n2) * 8; // norms, rescale, CSR / CSC offsets, alpha, beta
    t += n1 * round_up64(n2, 32) / 32 * 8;                      // coin words and their prefix
    t += cap * (4 + 4 + 8 + 4 + 8);                             // col, erow, qhat, csc_row, csc_pos
    t += 2 * round_up64(round_up64(p.k, 16), 256) * round_up64(rows, 64) * 4;   // tensor-core Pi buffers
    // WAltMin scratch (largest arena) and the estimate's values
    t += cap * (1 + 2 * acc + 4 + acc) + (n1 + n2) * b * acc * 2 + (nmax / 64 + 1) * 72 * 72 * 8;
    t += (2 * n1 + n2) * r * 8 + (n1 + n2) * r * acc + cap / 32 * 8 * 4 + nmax * (r * (r + 1) / 2 + r) * 8;
    t += (n1 + n2 + 1) * r * 8;                                 // result factors
    *bytes = t + (1 << 20);
    return SMP_OK;
}

smp_status smp_serve_create(const smp_server_params* params, smp_server** out) {
    if (!params || !out) return SMP_EINVAL;
    *out = nullptr;
    if (params->hbm_budget_bytes <= 0 || params->solve_workers < 1 || params->solve_workers > 64) return SMP_EINVAL;
    smp_server* sv = new (std::nothrow) smp_server();
    if (!sv) return SMP_ENOMEM;
    sv->p = *params;
    if (cudaGetDevice(&sv->device) != cudaSuccess) {
        delete sv;
        return SMP_ECUDA;
    }
    for (int i = 0; i < params->solve_workers; ++i) sv->workers.emplace_back(worker_loop, sv);
    *out = sv;
    return SMP_OK;
}

smp_status smp_serve_admit(smp_server* sv, const smp_job_params* jp, int64_t* job_id) {
    if (!sv || !jp || !job_id) return SMP_EINVAL;
    int64_t need = 0;
    smp_status s = smp_serve_job_bytes(jp, &need);
    if (s != SMP_OK) return s;
    if (jp->r > 32 || jp->r > jp->sketch.n1 || jp->r > jp->sketch.n2 || jp->T < 0 || jp->T > 127) return SMP_EINVAL;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stopping) return SMP_ESTATE;
        if (sv->used + need > sv->p.hbm_budget_bytes) return SMP_EBUSY;
        sv->used += need;   // reserved before the allocations so that concurrent admissions see it
    }
    std::unique_ptr<Job> j(new (std::nothrow) Job());
    auto unreserve = [&] {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->used -= need;
    };
    if (!j) {
        unreserve();
        return SMP_ENOMEM;
    }
    j->jp = *jp;
    j->bytes = need;
    const int64_t n1 = jp->sketch.n1, n2 = jp->sketch.n2, r = jp->r;
    if (cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking) != cudaSuccess) {
        unreserve();
        return SMP_ECUDA;
    }
    s = smp_sketch_begin(&jp->sketch, j->stream, &j->ctx);
    if (s == SMP_OK && smp::dev_malloc((void**)&j->U, (size_t)(n1 + n2 + 1) * r * 8, j->stream) != cudaSuccess)
        s = SMP_ENOMEM;
    if (s != SMP_OK) {
        if (j->ctx) smp_destroy(j->ctx);
        cudaStreamDestroy(j->stream);
        unreserve();
        return s;
    }
    j->S = j->U + n1 * r;
    j->V = j->S + r;
    std::lock_guard<std::mutex> lk(sv->mu);
    const int64_t id = sv->next_id++;
    sv->jobs.emplace(id, std::move(j));
    *job_id = id;
    return SMP_OK;
}

smp_status smp_serve_block(smp_server* sv, int64_t job_id, const void* A_blk, int64_t lda, const void* B_blk,
                           int64_t ldb, int64_t row0, int64_t nrows) {
    if (!sv) return SMP_EINVAL;
    Job* j = nullptr;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->jobs.find(job_id);
        if (it == sv->jobs.end()) return SMP_EINVAL;
        if (it->second->state != JobState::Streaming) return SMP_ESTATE;
        j = it->second.get();
    }
    // only the caller's thread touches a streaming job
    return smp_sketch_accumulate(j->ctx, A_blk, lda, B_blk, ldb, row0, nrows);
}

smp_status smp_serve_close(smp_server* sv, int64_t job_id) {
    if (!sv) return SMP_EINVAL;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->jobs.find(job_id);
        if (it == sv->jobs.end()) return SMP_EINVAL;
        Job* j = it->second.get();
        if (j->state != JobState::Streaming) return SMP_ESTATE;
        j->state = JobState::Queued;
        j->t_close = Clock::now();
        sv->ready.push_back(job_id);
    }
    sv->cv_work.notify_one();
    return SMP_OK;
}

smp_status smp_serve_poll(smp_server* sv, int64_t job_id, int32_t* done) {
    if (!sv || !done) return SMP_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(job_id);
    if (it == sv->jobs.end()) return SMP_EINVAL;
    const JobState st = it->second->state;
    *done = (st == JobState::Done || st == JobState::Failed) ? 1 : 0;
    return SMP_OK;
}

smp_status smp_serve_collect(smp_server* sv, int64_t job_id, double timeout_s, double* U_dev, double* S_dev,
                             double* V_dev, int64_t* nnz, double* latency_ms) {
    if (!sv) return SMP_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(job_id);
    if (it == sv->jobs.end()) return SMP_EINVAL;
    Job* j = it->second.get();
    if (j->state == JobState::Streaming) return SMP_ESTATE;
    const auto pred = [&] { return j->state == JobState::Done || j->state == JobState::Failed; };
    if (timeout_s < 0.0) {
        sv->cv_done.wait(lk, pred);
    } else if (!sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
        return SMP_ETIMEOUT;
    }
    smp_status s = j->status;
    if (s == SMP_OK) {
        const int64_t n1 = j->jp.sketch.n1, n2 = j->jp.sketch.n2, r = j->jp.r;
        cudaError_t e = cudaSuccess;
        if (U_dev) e = cudaMemcpyAsync(U_dev, j->U, (size_t)n1 * r * 8, cudaMemcpyDeviceToDevice, j->stream);
        if (e == cudaSuccess && S_dev)
            e = cudaMemcpyAsync(S_dev, j->S, (size_t)r * 8, cudaMemcpyDeviceToDevice, j->stream);
        if (e == cudaSuccess && V_dev)
            e = cudaMemcpyAsync(V_dev, j->V, (size_t)n2 * r * 8, cudaMemcpyDeviceToDevice, j->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(j->stream);
        if (e != cudaSuccess) s = SMP_ECUDA;
        if (nnz) *nnz = j->nnz;
        if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(j->t_done - j->t_close).count();
    }
    release_job(sv, job_id);
    return s;
}

smp_status smp_serve_cancel(smp_server* sv, int64_t job_id) {
    if (!sv) return SMP_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(job_id);
    if (it == sv->jobs.end()) return SMP_EINVAL;
    Job* j = it->second.get();
    if (j->state == JobState::Solving) {   // let the worker finish, then drop the result
        sv->cv_done.wait(lk, [&] { return j->state != JobState::Solving; });
    }
    release_job(sv, job_id);   // a queued job is skipped by the workers once it is gone
    return SMP_OK;
}

smp_status smp_serve_stats(smp_server* sv, int64_t* used_bytes, int32_t* live_jobs) {
    if (!sv) return SMP_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (used_bytes) *used_bytes = sv->used;
    if (live_jobs) *live_jobs = (int32_t)sv->jobs.size();
    return SMP_OK;
}

smp_status smp_serve_destroy(smp_server* sv) {
    if (!sv) return SMP_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
        sv->ready.clear();
    }
    sv->cv_work.notify_all();
    for (auto& t : sv->workers) t.join();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        std::vector<int64_t> ids;
        for (auto& kv : sv->jobs) ids.push_back(kv.first);
        for (int64_t id : ids) release_job(sv, id);
    }
    delete sv;
    return SMP_OK;
}

}  // extern "C"
