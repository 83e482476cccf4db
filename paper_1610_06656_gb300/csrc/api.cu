// libsmp C ABI: argument checks, context lifecycle, call ordering and error reporting. Every compute step runs in
// the kernels of sketch*.cu, sample.cu, estimate.cu and waltmin.cu; this file only validates and dispatches.
#include <cuda_runtime.h>

#include <mutex>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace {
thread_local std::string g_begin_error;
}

namespace smp {

std::atomic<uint64_t> g_launches{0};
std::atomic<int32_t> g_fail_allocs{0};
std::atomic<int64_t> g_tc_wait_ns{0};
std::atomic<int32_t> g_tc_skip_stage{-1};

cudaStream_t release_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        streams[dev] = nullptr;
    }
    return streams[dev];
}

void free_idle(void* p) {
    if (p) cudaFreeAsync(p, release_stream());
}

void release_after(cudaStream_t st) {
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
        if (cudaEventRecord(ev, st) != cudaSuccess || cudaStreamWaitEvent(release_stream(), ev, 0) != cudaSuccess)
            cudaStreamSynchronize(st);   // cannot order the release stream: wait for st instead
        cudaEventDestroy(ev);
    } else {
        cudaStreamSynchronize(st);
    }
}

void free_after(void* p, cudaStream_t st) {
    if (!p) return;
    release_after(st);
    free_idle(p);
}

smp_status fail(smp_ctx* c, smp_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_begin_error = msg;
    return s;
}

smp_status check_cuda(smp_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SMP_OK;
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? SMP_ENOMEM : SMP_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

smp_status read_device_error(smp_ctx* c) {
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return check_cuda(c, e, "reading the device error word");
    if (h == 0) return SMP_OK;
    cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream);
    char word[32];
    snprintf(word, sizeof(word), " (error word 0x%x)", h);
    if (h & DEVERR_TIMEOUT) return fail(c, SMP_ETIMEOUT, std::string("a bounded device-side wait gave up") + word);
    if (h & DEVERR_NUMERIC) return fail(c, SMP_ENUMERIC, "a Cholesky pivot was not positive");
    return fail(c, SMP_ECUDA, "a kernel index check failed");
}

}  // namespace smp

using namespace smp;

namespace {

void release_host_stage(smp_ctx* c) {
    if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
    release_after(c->stream);
    for (int b = 0; b < 2; ++b) {
        free_idle(c->host_stage[b]);
        if (c->host_copied[b]) cudaEventDestroy(c->host_copied[b]);
        if (c->host_consumed[b]) cudaEventDestroy(c->host_consumed[b]);
        c->host_stage[b] = nullptr;
        c->host_copied[b] = c->host_consumed[b] = nullptr;
    }
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    c->copy_stream = nullptr;
    c->host_stage_bytes = 0;
}

void free_ctx(smp_ctx* c) {
    release_host_stage(c);
    release_tc(c);
    void* ptrs[] = {c->part,   c->nsq,    c->sk,      c->s_all,   c->D_all,   c->F,     c->row_ptr, c->col_ptr,
                    c->col,    c->qhat,   c->csc_row, c->csc_pos, c->alpha,   c->beta,  c->mask,    c->wpre,
                    c->erow,   c->srht_y, c->srht_nsq, c->srht_rows, c->mn_S,   c->mn_bcum, c->mn_btot, c->mn_rows, c->mn_off, c->mn_draw, c->mn_count,
                    c->row_cnt, c->col_cnt, c->ex_part, c->ex_at, c->dev_err};
    // stream-ordered frees behind the context's queued work, on the shared release stream: no device-wide
    // synchronisation, so other contexts' work keeps running
    release_after(c->stream);
    for (void* p : ptrs) free_idle(p);
    delete c;
}

// Context memory comes from the device's default stream-ordered pool; keep what contexts free cached there for the
// next ones instead of returning it to the driver at every synchronisation (a process-local pool setting).
void keep_pool_memory(int device) {
    static std::once_flag once;
    std::call_once(once, [device] {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    });
}

bool elem_size(int dtype, size_t* sz) {
    switch (dtype) {
        case SMP_F32: *sz = 4; return true;
        case SMP_BF16: *sz = 2; return true;
        case SMP_F64: *sz = 8; return true;
    }
    return false;
}

// Record rows [row0, row0 + nrows) as accumulated in v; a range that overlaps rows already there is rejected (a
// duplicated row block would be summed twice).
smp_status track_rows_in(smp_ctx* c, std::vector<std::pair<int64_t, int64_t>>& v, int64_t row0, int64_t nrows) {
    const int64_t a = row0, b = row0 + nrows;
    auto it = std::upper_bound(v.begin(), v.end(), a,
                               [](int64_t x, const std::pair<int64_t, int64_t>& r) { return x < r.second; });
    if (it != v.end() && it->first < b) {
        char msg[160];
        snprintf(msg, sizeof msg, "rows [%lld, %lld) overlap rows [%lld, %lld) already accumulated", (long long)a,
                 (long long)b, (long long)it->first, (long long)it->second);
        return fail(c, SMP_EINVAL, msg);
    }
    it = v.insert(it, {a, b});
    if (it + 1 != v.end() && (it + 1)->first == b) {   // merge with the range that starts where this one ends
        it->second = (it + 1)->second;
        v.erase(it + 1);
    }
    if (it != v.begin() && (it - 1)->second == a) {    // and with the one that ends where it starts
        (it - 1)->second = it->second;
        v.erase(it);
    }
    return SMP_OK;
}

// Rows of the single pass (sketch or norms), since the last reset.
smp_status track_rows(smp_ctx* c, int64_t row0, int64_t nrows) { return track_rows_in(c, c->seen, row0, nrows); }

// A single pass accumulates either the sketch (with the norms) or the norms alone (LELA's first pass), not both.
smp_status claim_pass(smp_ctx* c, int kind) {
    if (c->pass_kind != 0 && c->pass_kind != kind)
        return fail(c, SMP_ESTATE, kind == 1 ? "sketch rows after norms-only rows in the same pass"
                                             : "norms-only rows after sketch rows in the same pass");
    c->pass_kind = kind;
    return SMP_OK;
}

// A new Omega invalidates the exact entries accumulated for the previous one.
void omega_changed(smp_ctx* c) {
    c->ex_ready = false;
    c->seen_exact.clear();
}

smp_status coverage_of(const std::vector<std::pair<int64_t, int64_t>>& v, int64_t* rows, int64_t* first_missing,
                       int64_t* ranges) {
    int64_t total = 0;
    for (const auto& r : v) total += r.second - r.first;
    if (rows) *rows = total;
    if (first_missing) *first_missing = (!v.empty() && v.front().first == 0) ? v.front().second : 0;
    if (ranges) *ranges = (int64_t)v.size();
    return SMP_OK;
}

smp_status check_block(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t nrows) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    if (c->finalized) return fail(c, SMP_ESTATE, "accumulate after finalize");
    if (nrows < 0 || nrows > c->max_rows) return fail(c, SMP_EINVAL, "nrows out of [0, max_rows]");
    if (nrows == 0) return SMP_OK;
    if (!A || lda < c->p.n1) return fail(c, SMP_EINVAL, "A_blk is null or lda < n1");
    if (!c->p.same_ab && (!B || ldb < c->p.n2)) return fail(c, SMP_EINVAL, "B_blk is null or ldb < n2");
    return SMP_OK;
}

}  // namespace

extern "C" {

smp_status smp_sketch_begin(const smp_params* params, void* stream, smp_ctx** out) {
    if (!params || !out) return fail(nullptr, SMP_EINVAL, "null params or out");
    *out = nullptr;
    const smp_params& p = *params;
    size_t esz = 0;
    if (!elem_size(p.dtype, &esz)) return fail(nullptr, SMP_EINVAL, "unknown dtype");
    if (p.n1 < 1 || p.n2 < 1 || p.n1 > (int64_t)1 << 30 || p.n2 > (int64_t)1 << 30)
        return fail(nullptr, SMP_EINVAL, "n1, n2 must be in [1, 2^30]");
    if (p.same_ab && p.n1 != p.n2) return fail(nullptr, SMP_EINVAL, "same_ab needs n1 == n2");
    if (p.k < 1 || p.k > 4096) return fail(nullptr, SMP_EINVAL, "k must be in [1, 4096]");
    if (p.engine < SMP_ENGINE_AUTO || p.engine > SMP_ENGINE_TC_BF16) return fail(nullptr, SMP_EINVAL, "unknown engine");
    if (p.engine == SMP_ENGINE_TC_BF16 && p.dtype != SMP_F32)
        return fail(nullptr, SMP_EUNSUPPORTED, "SMP_ENGINE_TC_BF16 takes SMP_F32 row blocks");
    if (p.engine == SMP_ENGINE_SRHT) {
        if (p.dtype != SMP_F32) return fail(nullptr, SMP_EUNSUPPORTED, "SMP_ENGINE_SRHT takes SMP_F32 row blocks");
        const int64_t R = p.max_rows ? p.max_rows : 65536;
        if (R < 256 || R > 65536 || (R & (R - 1)) != 0)
            return fail(nullptr, SMP_EINVAL, "SMP_ENGINE_SRHT needs max_rows a power of two in [256, 65536]");
    }
    if (p.engine == SMP_ENGINE_TC_FP8 && p.dtype != SMP_BF16)
        return fail(nullptr, SMP_EUNSUPPORTED, "SMP_ENGINE_TC_FP8 takes SMP_BF16 row blocks");
    if (p.max_rows < 0) return fail(nullptr, SMP_EINVAL, "max_rows < 0");
    smp_ctx* c = new (std::nothrow) smp_ctx();
    if (!c) return fail(nullptr, SMP_ENOMEM, "host allocation");
    c->p = p;
    c->stream = (cudaStream_t)stream;
    c->max_rows = p.max_rows ? p.max_rows : 65536;
    c->acc_bytes = p.dtype == SMP_F64 ? 8 : 4;
    c->ntot = p.same_ab ? p.n1 : p.n1 + p.n2;
    c->ldk = round_up(p.k, 4);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        smp_status s = check_cuda(nullptr, e, "smp_sketch_begin: device query");
        delete c;
        return s;
    }
    c->splits = 8;
    keep_pool_memory(c->device);
    const size_t acc = (size_t)c->acc_bytes;
    const int64_t n1 = p.n1, n2 = p.n2;
    bool ok = true;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (!ok) return;
        if (smp::dev_malloc(ptr, std::max<size_t>(bytes, 16), c->stream) != cudaSuccess) ok = false;
    };
    alloc(&c->part, (size_t)c->splits * c->ntot * c->ldk * acc);
    alloc((void**)&c->nsq, (size_t)c->splits * c->ntot * 8);
    alloc(&c->sk, (size_t)c->ntot * c->ldk * acc);
    alloc((void**)&c->s_all, (size_t)c->ntot * 8);
    alloc((void**)&c->D_all, (size_t)c->ntot * 8);
    alloc((void**)&c->F, 16);
    alloc((void**)&c->row_ptr, (size_t)(n1 + 1) * 8);
    alloc((void**)&c->col_ptr, (size_t)(n2 + 1) * 8);
    alloc((void**)&c->alpha, (size_t)n1 * 8);
    alloc((void**)&c->beta, (size_t)n2 * 8);
    alloc((void**)&c->row_cnt, (size_t)n1 * 4);
    alloc((void**)&c->col_cnt, (size_t)n2 * 4);
    alloc((void**)&c->dev_err, sizeof(int));
    if (!ok) {
        cudaGetLastError();
        free_ctx(c);
        return fail(nullptr, SMP_ENOMEM, "smp_sketch_begin: device allocation failed");
    }
    cudaStream_t st = c->stream;
    e = cudaMemsetAsync(c->part, 0, (size_t)c->splits * c->ntot * c->ldk * acc, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->nsq, 0, (size_t)c->splits * c->ntot * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dev_err, 0, sizeof(int), st);
    if (e != cudaSuccess) {
        smp_status s = check_cuda(nullptr, e, "smp_sketch_begin: clearing accumulators");
        free_ctx(c);
        return s;
    }
    *out = c;
    return SMP_OK;
}

smp_status smp_sketch_accumulate(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                                 int64_t nrows) {
    smp_status s = check_block(c, A, lda, B, ldb, nrows);
    if (s != SMP_OK || nrows == 0) return s;
    if (row0 < 0) return fail(c, SMP_EINVAL, "row0 < 0");
    if ((s = claim_pass(c, 1)) != SMP_OK) return s;
    if (c->p.engine == SMP_ENGINE_TC_FP8) {
        if (!fp8_block_ok(c, A, lda, B, ldb))
            return fail(c, SMP_EUNSUPPORTED, "the FP8 sketch needs k <= 1024, 16-byte aligned blocks, lda, ldb % 8 == 0");
        if ((s = track_rows(c, row0, nrows)) != SMP_OK) return s;
        return check_cuda(c, launch_sketch_fp8(c, A, lda, B, ldb, row0, nrows, nullptr, 0), "smp_sketch_accumulate");
    }
    if (c->p.engine == SMP_ENGINE_SRHT) {
        if (!srht_block_ok(c, row0, nrows))
            return fail(c, SMP_EINVAL, "the SRHT sketch takes whole blocks: row0 % max_rows == 0");
        if ((s = track_rows(c, row0, nrows)) != SMP_OK) return s;
        return check_cuda(c, launch_sketch_srht(c, A, lda, B, ldb, row0, nrows), "smp_sketch_accumulate");
    }
    const bool bf16 = c->p.dtype == SMP_BF16;
    const bool tc_ok = bf16 ? bf16_block_ok(c, A, lda, B, ldb) : tc_block_ok(c, A, lda, B, ldb);
    const bool tc_engine = c->p.engine == SMP_ENGINE_TC || c->p.engine == SMP_ENGINE_TC_BF16;
    if (tc_engine && !tc_ok)
        return fail(c, SMP_EUNSUPPORTED,
                    "the tensor-core sketch needs SMP_F32 with k <= 512 and lda, ldb % 4 == 0, or SMP_BF16 with "
                    "k <= 1024 and lda, ldb % 8 == 0, and 16-byte aligned blocks");
    const bool want_tc = tc_engine || (c->p.engine == SMP_ENGINE_AUTO && tc_ok);
    if ((s = track_rows(c, row0, nrows)) != SMP_OK) return s;
    cudaError_t e = !want_tc ? launch_sketch_simt(c, A, lda, B, ldb, row0, nrows, nullptr, 0)
                             : bf16 ? launch_sketch_bf16(c, A, lda, B, ldb, row0, nrows, nullptr, 0)
                                    : launch_sketch_tc(c, A, lda, B, ldb, row0, nrows);
    return check_cuda(c, e, "smp_sketch_accumulate");
}

smp_status smp_sketch_accumulate_host(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb,
                                      int64_t row0, int64_t nrows) {
    smp_status s = check_block(c, A, lda, B, ldb, nrows);
    if (s != SMP_OK || nrows == 0) return s;
    if (row0 < 0) return fail(c, SMP_EINVAL, "row0 < 0");
    size_t esz = 0;
    elem_size(c->p.dtype, &esz);
    // staging rows padded to 16 bytes, so every engine's alignment rule holds for the device copy
    const int64_t pitch_a = round_up(c->p.n1, (int64_t)(16 / esz));
    const int64_t pitch_b = c->p.same_ab ? 0 : round_up(c->p.n2, (int64_t)(16 / esz));
    const size_t bytes = (size_t)c->max_rows * (size_t)(pitch_a + pitch_b) * esz;
    cudaError_t e = cudaSuccess;
    if (!c->copy_stream) {
        e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaEventCreateWithFlags(&c->host_copied[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->host_consumed[b], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return check_cuda(c, e, "smp_sketch_accumulate_host: copy stream");
    }
    if (c->host_stage_bytes < bytes) {
        for (int b = 0; b < 2; ++b) {
            free_after(c->host_stage[b], c->stream);
            c->host_stage[b] = nullptr;
        }
        c->host_stage_bytes = 0;
        for (int b = 0; b < 2; ++b) {
            if (smp::dev_malloc(&c->host_stage[b], bytes, c->stream) != cudaSuccess) {
                cudaGetLastError();
                return fail(c, SMP_ENOMEM, "smp_sketch_accumulate_host: staging buffers");
            }
            if ((e = cudaEventRecord(c->host_consumed[b], c->stream)) != cudaSuccess)
                return check_cuda(c, e, "smp_sketch_accumulate_host");
        }
        c->host_stage_bytes = bytes;
    }
    const int b = c->host_next;
    char* dA = (char*)c->host_stage[b];
    char* dB = dA + (size_t)c->max_rows * pitch_a * esz;
    // a block whose rows are already packed at the staging pitch goes in one linear copy (a 2-D copy of 65,536
    // short rows costs the copy engine per row and ran at a quarter of the link's rate)
    auto copy_rows = [&](void* dst, int64_t dpitch, const void* src, int64_t spitch, int64_t width) {
        if (spitch == dpitch && width == dpitch)
            return cudaMemcpyAsync(dst, src, (size_t)nrows * dpitch * esz, cudaMemcpyHostToDevice, c->copy_stream);
        return cudaMemcpy2DAsync(dst, dpitch * esz, src, spitch * esz, width * esz, nrows, cudaMemcpyHostToDevice,
                                 c->copy_stream);
    };
    e = cudaStreamWaitEvent(c->copy_stream, c->host_consumed[b], 0);   // the sketch that last read buffer b ended
    if (e == cudaSuccess) e = copy_rows(dA, pitch_a, A, lda, c->p.n1);
    if (e == cudaSuccess && !c->p.same_ab) e = copy_rows(dB, pitch_b, B, ldb, c->p.n2);
    if (e == cudaSuccess) e = cudaEventRecord(c->host_copied[b], c->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->host_copied[b], 0);
    if (e != cudaSuccess) return check_cuda(c, e, "smp_sketch_accumulate_host: host-to-device copy");
    s = smp_sketch_accumulate(c, dA, pitch_a, c->p.same_ab ? nullptr : dB, pitch_b, row0, nrows);
    e = cudaEventRecord(c->host_consumed[b], c->stream);
    c->host_next = 1 - b;
    if (s != SMP_OK) return s;
    return check_cuda(c, e, "smp_sketch_accumulate_host");
}

smp_status smp_sketch_accumulate_pi(smp_ctx* c, const void* Pi, int64_t ldp, const void* A, int64_t lda,
                                    const void* B, int64_t ldb, int64_t row0, int64_t nrows) {
    smp_status s = check_block(c, A, lda, B, ldb, nrows);
    if (s != SMP_OK || nrows == 0) return s;
    if (!Pi || ldp < nrows) return fail(c, SMP_EINVAL, "Pi_blk is null or ldp < nrows");
    if (c->p.engine == SMP_ENGINE_SRHT) return fail(c, SMP_EUNSUPPORTED, "the SRHT engine generates its own Pi");
    if (row0 < 0) return fail(c, SMP_EINVAL, "row0 < 0");
    if ((s = claim_pass(c, 1)) != SMP_OK) return s;
    if (c->p.engine == SMP_ENGINE_TC_FP8) {
        if (!fp8_block_ok(c, A, lda, B, ldb))
            return fail(c, SMP_EUNSUPPORTED, "the FP8 sketch needs k <= 1024, 16-byte aligned blocks, lda, ldb % 8 == 0");
        if ((s = track_rows(c, row0, nrows)) != SMP_OK) return s;
        return check_cuda(c, launch_sketch_fp8(c, A, lda, B, ldb, row0, nrows, (const float*)Pi, ldp),
                          "smp_sketch_accumulate_pi");
    }
    const bool bf16 = c->p.dtype == SMP_BF16;
    const bool tc_ok = bf16 ? bf16_block_ok(c, A, lda, B, ldb)
                            : tc_block_ok(c, A, lda, B, ldb) && ((uintptr_t)Pi % 16 == 0) && (ldp % 4 == 0);
    const bool tc_engine = c->p.engine == SMP_ENGINE_TC || c->p.engine == SMP_ENGINE_TC_BF16;
    if (tc_engine && !tc_ok)
        return fail(c, SMP_EUNSUPPORTED, "the tensor-core sketch needs 16-byte aligned Pi and ldp % 4 == 0");
    if ((s = track_rows(c, row0, nrows)) != SMP_OK) return s;
    if (tc_engine || (c->p.engine == SMP_ENGINE_AUTO && tc_ok))
        return check_cuda(c,
                          bf16 ? launch_sketch_bf16(c, A, lda, B, ldb, row0, nrows, (const float*)Pi, ldp)
                               : launch_sketch_tc_pi(c, A, lda, B, ldb, row0, nrows, (const float*)Pi, ldp),
                          "smp_sketch_accumulate_pi");
    return check_cuda(c, launch_sketch_simt(c, A, lda, B, ldb, row0, nrows, Pi, ldp), "smp_sketch_accumulate_pi");
}

smp_status smp_sketch_reset(smp_ctx* c) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    cudaError_t e = cudaMemsetAsync(c->part, 0, (size_t)c->splits * c->ntot * c->ldk * c->acc_bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->nsq, 0, (size_t)c->splits * c->ntot * 8, c->stream);
    if (e == cudaSuccess) e = tc_speculate_first_block(c);   // the next solve most likely starts at row 0
    if (e != cudaSuccess) return check_cuda(c, e, "smp_sketch_reset");
    c->finalized = false;
    c->sampled = false;
    c->nnz = 0;
    c->seen.clear();
    c->pass_kind = 0;
    omega_changed(c);
    return SMP_OK;
}

smp_status smp_sketch_finalize(smp_ctx* c) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    if (c->finalized) return fail(c, SMP_ESTATE, "finalize called twice");
    smp_status s = check_cuda(c, launch_finalize(c), "smp_sketch_finalize");
    if (s == SMP_OK) c->finalized = true;
    return s;
}

smp_status smp_sketch_view(smp_ctx* c, const void** At, const void** Bt, int64_t* ldk, const double** sA,
                           const double** sB, double* F_host) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    if (!c->finalized) return fail(c, SMP_ESTATE, "sketch not finalized");
    const char* base = (const char*)c->sk;
    if (At) *At = base;
    if (Bt) *Bt = c->p.same_ab ? base : base + (size_t)c->p.n1 * c->ldk * c->acc_bytes;
    if (ldk) *ldk = c->ldk;
    if (sA) *sA = c->s_all;
    if (sB) *sB = c->p.same_ab ? c->s_all : c->s_all + c->p.n1;
    if (F_host) {
        cudaError_t e = cudaMemcpyAsync(F_host, c->F, 16, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return check_cuda(c, e, "smp_sketch_view");
    }
    return SMP_OK;
}

smp_status smp_sketch_import(smp_ctx* c, const void* At, const void* Bt, const double* sA, const double* sB) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    if (!At || !sA || (!c->p.same_ab && (!Bt || !sB))) return fail(c, SMP_EINVAL, "null sketch or norms");
    smp_status s = check_cuda(c, launch_import(c, At, Bt, sA, sB), "smp_sketch_import");
    if (s == SMP_OK) {
        c->finalized = true;
        c->pass_kind = 1;
    }
    return s;
}

smp_status smp_sample(smp_ctx* c, double m, uint64_t seed, int64_t* nnz_out) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    if (!c->finalized) return fail(c, SMP_ESTATE, "smp_sample before finalize");
    if (!(m > 0.0)) return fail(c, SMP_EINVAL, "m must be > 0");
    double F[2];
    cudaError_t e = cudaMemcpyAsync(F, c->F, 16, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return check_cuda(c, e, "smp_sample");
    if (!(F[0] > 0.0) && !(F[1] > 0.0)) return fail(c, SMP_EINVAL, "both Frobenius norms are zero");
    omega_changed(c);
    return run_sample(c, m, seed, nnz_out);
}

smp_status smp_sample_multinomial(smp_ctx* c, double m, uint64_t seed, int64_t* nnz_out) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    if (!c->finalized) return fail(c, SMP_ESTATE, "smp_sample_multinomial before finalize");
    if (!(m > 0.0)) return fail(c, SMP_EINVAL, "m must be > 0");
    double F[2];
    cudaError_t e = cudaMemcpyAsync(F, c->F, 16, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return check_cuda(c, e, "smp_sample_multinomial");
    if (!(F[0] > 0.0) && !(F[1] > 0.0)) return fail(c, SMP_EINVAL, "both Frobenius norms are zero");
    omega_changed(c);
    return run_sample(c, m, seed, nnz_out, true);
}

smp_status smp_sample_from_norms(smp_ctx* c, const double* sA, const double* sB, double m, uint64_t seed,
                                 int64_t* nnz_out) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    if (!sA || (!c->p.same_ab && !sB)) return fail(c, SMP_EINVAL, "null norms");
    if (!(m > 0.0)) return fail(c, SMP_EINVAL, "m must be > 0");
    cudaError_t e = cudaMemcpyAsync(c->s_all, sA, (size_t)c->p.n1 * 8, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && !c->p.same_ab)
        e = cudaMemcpyAsync(c->s_all + c->p.n1, sB, (size_t)c->p.n2 * 8, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = launch_frobenius(c);
    double F[2];
    if (e == cudaSuccess) e = cudaMemcpyAsync(F, c->F, 16, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return check_cuda(c, e, "smp_sample_from_norms");
    if (!(F[0] > 0.0) && !(F[1] > 0.0)) return fail(c, SMP_EINVAL, "both Frobenius norms are zero");
    omega_changed(c);
    return run_sample(c, m, seed, nnz_out);
}

smp_status smp_omega_view(const smp_ctx* c, int64_t* nnz, const int64_t** row_ptr, const int32_t** col,
                          const double** qhat, const int64_t** col_ptr, const int32_t** csc_row,
                          const int64_t** csc_pos) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    if (!c->sampled) return fail(const_cast<smp_ctx*>(c), SMP_ESTATE, "Omega not drawn yet");
    if (nnz) *nnz = c->nnz;
    if (row_ptr) *row_ptr = c->row_ptr;
    if (col) *col = c->col;
    if (qhat) *qhat = c->qhat;
    if (col_ptr) *col_ptr = c->col_ptr;
    if (csc_row) *csc_row = c->csc_row;
    if (csc_pos) *csc_pos = c->csc_pos;
    return SMP_OK;
}

smp_status smp_estimate(smp_ctx* c, void* vals) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    if (!c->sampled || !c->finalized) return fail(c, SMP_ESTATE, "smp_estimate needs a finalized sketch and Omega");
    if (!vals && c->nnz > 0) return fail(c, SMP_EINVAL, "null vals");
    if (c->pass_kind == 2) return fail(c, SMP_ESTATE, "smp_estimate: the pass accumulated norms only (no sketch)");
    return check_cuda(c, launch_estimate(c, vals), "smp_estimate");
}

smp_status smp_waltmin(smp_ctx* c, const void* vals, int32_t r, int32_t T, uint32_t flags, uint64_t seed,
                       const double* U_init, double* U, double* S, double* V) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    if (!c->sampled) return fail(c, SMP_ESTATE, "smp_waltmin before smp_sample");
    if (r < 1 || r > 32 || r > c->p.n1 || r > c->p.n2) return fail(c, SMP_EINVAL, "r out of [1, min(32, n1, n2)]");
    if (T < 0 || T > 127) return fail(c, SMP_EINVAL, "T out of [0, 127]");
    if (flags & ~(SMP_SPLIT_OMEGA | SMP_NO_TRIM | SMP_INIT_GIVEN | SMP_FP64_ALS))
        return fail(c, SMP_EINVAL, "unknown flag");
    if ((flags & SMP_INIT_GIVEN) && !U_init) return fail(c, SMP_EINVAL, "SMP_INIT_GIVEN without U_init");
    if (!U || !S || !V || (!vals && c->nnz > 0)) return fail(c, SMP_EINVAL, "null output or vals");
    return run_waltmin(c, vals, r, T, flags, seed, U_init, U, S, V);
}

smp_status smp_sketch_svd(smp_ctx* c, int32_t r, uint64_t seed, double* U, double* S, double* V) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    if (!c->finalized) return fail(c, SMP_ESTATE, "smp_sketch_svd before finalize");
    if (r < 1 || r > 32 || r > c->p.n1 || r > c->p.n2 || r > c->p.k)
        return fail(c, SMP_EINVAL, "r out of [1, min(32, n1, n2, k)]");
    if (!U || !S || !V) return fail(c, SMP_EINVAL, "null output");
    if (c->pass_kind == 2) return fail(c, SMP_ESTATE, "smp_sketch_svd: the pass accumulated norms only (no sketch)");
    return run_sketch_svd(c, r, seed, U, S, V);
}

smp_status smp_norms_accumulate(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                                int64_t nrows) {
    smp_status s = check_block(c, A, lda, B, ldb, nrows);
    if (s != SMP_OK || nrows == 0) return s;
    if (row0 < 0) return fail(c, SMP_EINVAL, "row0 < 0");
    if ((s = claim_pass(c, 2)) != SMP_OK) return s;
    if ((s = track_rows(c, row0, nrows)) != SMP_OK) return s;
    return check_cuda(c, launch_norms(c, A, lda, B, ldb, nrows), "smp_norms_accumulate");
}

smp_status smp_exact_accumulate(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                                int64_t nrows) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    if (!c->sampled) return fail(c, SMP_ESTATE, "smp_exact_accumulate before smp_sample");
    if (nrows < 0 || nrows > c->max_rows) return fail(c, SMP_EINVAL, "nrows out of [0, max_rows]");
    if (nrows == 0) return SMP_OK;
    if (row0 < 0) return fail(c, SMP_EINVAL, "row0 < 0");
    if (!A || lda < c->p.n1) return fail(c, SMP_EINVAL, "A_blk is null or lda < n1");
    if (!c->p.same_ab && (!B || ldb < c->p.n2)) return fail(c, SMP_EINVAL, "B_blk is null or ldb < n2");
    const bool tc_ok = exact_tc_ok(c, A, lda, B, ldb);
    if (c->p.engine == SMP_ENGINE_TC && !tc_ok)
        return fail(c, SMP_EUNSUPPORTED,
                    "the tensor-core exact pass needs SMP_F32 and 16-byte aligned blocks with lda, ldb % 4 == 0");
    const bool use_tc = tc_ok && c->p.engine != SMP_ENGINE_SIMT;
    if ((use_tc ? (c->p.n1 + 511) / 512 : (c->p.n1 + 31) / 32) > 65535)
        return fail(c, SMP_EUNSUPPORTED, "smp_exact_accumulate: n1 too large for one launch grid");
    smp_status s = track_rows_in(c, c->seen_exact, row0, nrows);
    if (s != SMP_OK) return s;
    return check_cuda(c, launch_exact(c, A, lda, B, ldb, nrows, use_tc), "smp_exact_accumulate");
}

smp_status smp_exact_values(smp_ctx* c, void* vals) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    if (!c->sampled) return fail(c, SMP_ESTATE, "smp_exact_values before smp_sample");
    if (c->seen_exact.empty()) return fail(c, SMP_ESTATE, "smp_exact_values before smp_exact_accumulate");
    if (!vals && c->nnz > 0) return fail(c, SMP_EINVAL, "null vals");
    return check_cuda(c, launch_exact_values(c, vals), "smp_exact_values");
}

smp_status smp_exact_coverage(const smp_ctx* c, int64_t* rows, int64_t* first_missing, int64_t* ranges) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    return coverage_of(c->seen_exact, rows, first_missing, ranges);
}

smp_status smp_sync(smp_ctx* c) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    smp_status s = check_cuda(c, cudaStreamSynchronize(c->stream), "smp_sync");
    if (s != SMP_OK) return s;
    return read_device_error(c);
}

smp_status smp_destroy(smp_ctx* c) {
    if (!c) return SMP_OK;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
    return SMP_OK;
}

const char* smp_last_error(const smp_ctx* c) { return c ? c->err.c_str() : g_begin_error.c_str(); }

const char* smp_status_string(smp_status s) {
    switch (s) {
        case SMP_OK: return "SMP_OK";
        case SMP_EINVAL: return "SMP_EINVAL";
        case SMP_ENOMEM: return "SMP_ENOMEM";
        case SMP_ECUDA: return "SMP_ECUDA";
        case SMP_ESTATE: return "SMP_ESTATE";
        case SMP_ETIMEOUT: return "SMP_ETIMEOUT";
        case SMP_ENUMERIC: return "SMP_ENUMERIC";
        case SMP_EUNSUPPORTED: return "SMP_EUNSUPPORTED";
        case SMP_EBUSY: return "SMP_EBUSY";
    }
    return "SMP_UNKNOWN";
}

int32_t smp_version(void) { return 100; }

int64_t smp_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }

void smp_debug_fail_allocs(int32_t n) { g_fail_allocs.store(n > 0 ? n : 0, std::memory_order_relaxed); }

void smp_debug_tc_wait(int64_t wait_ns, int32_t skip_stage) {
    g_tc_wait_ns.store(wait_ns > 0 ? wait_ns : 0, std::memory_order_relaxed);
    g_tc_skip_stage.store(skip_stage >= 0 ? skip_stage : -1, std::memory_order_relaxed);
}

smp_status smp_sketch_coverage(const smp_ctx* c, int64_t* rows, int64_t* first_missing, int64_t* ranges) {
    if (!c) return fail(nullptr, SMP_EINVAL, "null context");
    return coverage_of(c->seen, rows, first_missing, ranges);
}

}  // extern "C"
