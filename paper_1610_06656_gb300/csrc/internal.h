// Host-side internals of libsmp: the context object and the kernel launchers each translation unit exports.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/smp.h"

struct smp_ctx {
    smp_params p{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 0;
    int acc_bytes = 4;              // 4: float sketch state, 8: double (SMP_F64)
    bool finalized = false;
    bool sampled = false;
    int64_t ntot = 0;               // n1 + n2 (n1 when same_ab)
    int64_t ldk = 0;                // k rounded up to a multiple of 4
    int64_t max_rows = 0;
    int splits = 1;                 // row splits of the sketch partials
    void* part = nullptr;           // [splits][ntot][ldk] partial sketches (acc type)
    double* nsq = nullptr;          // [splits][ntot] partial column sums of squares
    void* sk = nullptr;             // [ntot][ldk] finalized sketch (row c = sketch column c)
    double* s_all = nullptr;        // [ntot] column sums of squares (A columns, then B columns)
    double* D_all = nullptr;        // [ntot] rescale factors ||X_c|| / ||Xt_c||
    double* F = nullptr;            // [2] Frobenius squares (device)
    // Omega
    int64_t nnz = 0, cap = 0;
    int64_t* row_ptr = nullptr;     // [n1 + 1]
    int64_t* col_ptr = nullptr;     // [n2 + 1]
    int32_t* col = nullptr;         // [cap]
    int32_t* erow = nullptr;        // [cap] row of each CSR entry
    double* qhat = nullptr;         // [cap]
    int32_t* csc_row = nullptr;     // [cap]
    int64_t* csc_pos = nullptr;     // [cap]
    double* alpha = nullptr;        // [n1]
    double* beta = nullptr;         // [n2]
    uint32_t* mask = nullptr;       // [n1][W] keep bits, W = ceil(n2 / 32)
    int32_t* wpre = nullptr;        // [n1][W] set bits of the row before each word
    int32_t* row_cnt = nullptr;     // [n1]
    int32_t* col_cnt = nullptr;     // [n2]
    int64_t mask_words = 0;
    // row-wise multinomial sampling (allocated on first use)
    double* mn_S = nullptr;         // [n1] row totals S_i
    double* mn_bcum = nullptr;      // [n2] blocked prefix sums of beta
    double* mn_btot = nullptr;      // [ceil(n2 / 1024)] block totals, then block offsets
    int32_t* mn_rows = nullptr;     // [n1] draws per row c_i
    int64_t* mn_off = nullptr;      // [n1 + 1] first draw of each row
    int32_t* mn_draw = nullptr;     // [mn_draw_cap] drawn column of every draw
    int64_t mn_draw_cap = 0;
    int32_t* mn_count = nullptr;    // [mn_count_cap] draws of each Omega entry (CSR order)
    // block SRHT sketch (allocated on first use)
    float* srht_y = nullptr;        // [max_rows][256] chunk transforms of one column group
    double* srht_nsq = nullptr;     // [max_rows / 256][256] chunk column sums of squares
    int32_t* srht_rows = nullptr;   // bucket offsets [257], bucketed sketch rows [1024], s >> 8 per row [1024]
    int64_t mn_count_cap = 0;
    int* dev_err = nullptr;         // device error word
    // tensor-core engine: two Pi buffers filled on a side stream; while one row block is sketched, Pi of the next
    // one (row0 + nrows, same size) is generated speculatively into the other buffer
    void* pi_buf[2] = {nullptr, nullptr};
    size_t pi_buf_bytes = 0;
    int64_t pi_row0[2] = {-1, -1};  // rows of Pi each buffer holds (or will hold once pi_ready fires)
    int64_t pi_nrows[2] = {0, 0};
    cudaStream_t gen_stream = nullptr;
    cudaEvent_t pi_ready[2] = {nullptr, nullptr};   // recorded on gen_stream after a buffer's generation
    cudaEvent_t pi_free[2] = {nullptr, nullptr};    // recorded on stream after the sketch that read a buffer
    void* fp8_ws = nullptr;          // FP8 engine: block maxima, scales, completion counter
    int pi_last = -1;                // buffer the last tensor-core sketch read
    int64_t pi_last_rows = 0;        // largest row block sketched so far
    std::vector<std::pair<int64_t, int64_t>> seen;   // disjoint sorted [begin, end) row ranges accumulated
    int pass_kind = 0;               // rows accumulated since the last reset: 0 none, 1 sketch, 2 norms only
    // LELA's second pass (allocated on first use): exact entries of A^T B over Omega
    double* ex_part = nullptr;       // [EXACT_SPLITS][ex_cap] row-split partials, CSC order
    int64_t ex_cap = 0;
    bool ex_ready = false;           // ex_part cleared for the current Omega
    float* ex_at = nullptr;          // [n1][max_rows rounded up to 4] TF32 A^T of the current row block
    size_t ex_at_bytes = 0;
    std::vector<std::pair<int64_t, int64_t>> seen_exact;   // row ranges of the second pass since Omega was drawn
    // host-resident row blocks (smp_sketch_accumulate_host, allocated on first use): two device staging buffers
    // filled on a copy stream, so the copy of block i + 1 overlaps the sketch of block i
    void* host_stage[2] = {nullptr, nullptr};
    size_t host_stage_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t host_copied[2] = {nullptr, nullptr};     // recorded on copy_stream after a buffer's copy
    cudaEvent_t host_consumed[2] = {nullptr, nullptr};   // recorded on stream after the sketch that read a buffer
    int host_next = 0;
    std::string err;
};

namespace smp {

// Kernel launches made by this library since it was loaded (process-wide), for launch-count reporting.
extern std::atomic<uint64_t> g_launches;
template <typename G>
inline G counted(G grid) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return grid;
}

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Device allocations of the library (stream-ordered). smp_debug_fail_allocs(n) makes the next n of them fail with
// cudaErrorMemoryAllocation: host-side fault injection for the SMP_ENOMEM paths.
extern std::atomic<int32_t> g_fail_allocs;
// Test hooks of the tensor-core sketch engines' bounded waits (smp_debug_tc_wait): the wait limit in ns (0: the
// 2 s default) and a stage whose data loads the next launch does not issue (-1: none; consumed by that launch).
extern std::atomic<int64_t> g_tc_wait_ns;
extern std::atomic<int32_t> g_tc_skip_stage;
template <typename T>
inline cudaError_t dev_malloc(T** p, size_t bytes, cudaStream_t st) {
    int32_t left = g_fail_allocs.load(std::memory_order_relaxed);
    while (left > 0) {
        if (g_fail_allocs.compare_exchange_weak(left, left - 1)) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMallocAsync((void**)p, bytes, st);
}

// Stream-ordered frees all go to one long-lived stream per device: when frees are spread over the many short-lived
// streams of contexts and jobs, the device memory pool's later allocations slow down several-fold.
cudaStream_t release_stream();
// Free memory that no queued work uses any more.
void free_idle(void* p);
// Order the release stream behind the work queued so far on st (then free_idle frees after that work).
void release_after(cudaStream_t st);
// release_after(st) + free_idle(p): for memory that work queued on st may still read.
void free_after(void* p, cudaStream_t st);

// sketch.cu
cudaError_t launch_sketch_simt(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                               int64_t nrows, const void* Pi, int64_t ldp);
cudaError_t launch_finalize(smp_ctx* c);
cudaError_t launch_frobenius(smp_ctx* c);   // F[0], F[1] from s_all (left-to-right sums)
cudaError_t launch_import(smp_ctx* c, const void* At, const void* Bt, const double* sA, const double* sB);
// Row splits the SIMT engine uses for a row range of nrows rows when at most `splits` partials are available: the
// `splits` argument launch_sketch_simt_into needs to touch exactly the partials it writes.
int simt_into_splits(int64_t ntot, int k, int64_t nrows, int splits, int sm_count);
cudaError_t launch_sketch_simt_into(int dtype, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n1,
                                    int64_t n2, int k, uint64_t seed, int64_t row0, int64_t nrows, float* part,
                                    double* nsq, int splits, int sm_count, float* At, float* Bt, double* sA,
                                    double* sB, cudaStream_t st);

// sketch_tc.cu
bool tc_supported(const smp_ctx* c);
void release_tc(smp_ctx* c);   // waits for the side stream, frees the Pi buffers, stream and events
cudaError_t tc_speculate_first_block(smp_ctx* c);   // after a reset: Pi of rows [0, last block size) ahead of time
// Generated Pi of the tensor-core engines: kpad rows (round_up(k, 16) up to 256 for binary32 contexts, else a
// multiple of 256; zero beyond k) x ld columns (row stride),
// esize bytes per element (4: TF32 in binary32 containers, 2: BF16, 1: E4M3).
struct PiGeom {
    int kpad;
    int64_t ld;
    int esize;
};
PiGeom pi_geom(const smp_ctx* c);
// Buffer holding Pi of rows [row0, row0 + nrows) (generated now on the side stream if no buffer has it); the
// context's stream waits for it.
cudaError_t pi_acquire(smp_ctx* c, int64_t row0, int64_t nrows, int* buf);
// After the sketch that reads buffer b is enqueued: mark b free at its end and generate Pi of the next row block
// into the other buffer.
cudaError_t pi_release(smp_ctx* c, int b, int64_t row0, int64_t nrows);
// A caller's Pi (k x nrows binary32, row stride ldp) rounded into a Pi buffer (BF16 contexts); the buffer is then
// released with pi_release like a generated one.
cudaError_t pi_import(smp_ctx* c, const float* Pi, int64_t ldp, int64_t nrows, int* buf);

// sketch_srht.cu
bool srht_block_ok(const smp_ctx* c, int64_t row0, int64_t nrows);
cudaError_t launch_sketch_srht(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                               int64_t nrows);

// sketch_fp8.cu
bool fp8_block_ok(const smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb);
cudaError_t launch_sketch_fp8(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                              int64_t nrows, const float* Pi, int64_t ldp);

// sketch_bf16.cu
bool bf16_tc_supported(const smp_ctx* c);
bool bf16_block_ok(const smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb);
cudaError_t launch_sketch_bf16(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                               int64_t nrows, const float* Pi, int64_t ldp);
bool tc_block_ok(const smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb);
cudaError_t launch_sketch_tc(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                             int64_t nrows);
cudaError_t launch_sketch_tc_pi(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                                int64_t nrows, const float* Pi, int64_t ldp);

// sample.cu
smp_status run_sample(smp_ctx* c, double m, uint64_t seed, int64_t* nnz_out, bool multinomial = false);

// estimate.cu
cudaError_t launch_estimate(smp_ctx* c, void* vals);

// exact.cu (LELA's two passes)
constexpr int EXACT_SPLITS = 4;   // row splits of the exact-entry partials
cudaError_t launch_norms(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t nrows);
bool exact_tc_ok(const smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb);
cudaError_t launch_exact(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t nrows,
                         bool tensor_cores);
cudaError_t launch_exact_values(smp_ctx* c, void* vals);

// waltmin.cu
smp_status run_sketch_svd(smp_ctx* c, int r, uint64_t seed, double* U, double* S, double* V);
smp_status run_waltmin(smp_ctx* c, const void* vals, int r, int T, uint32_t flags, uint64_t seed,
                       const double* U_init, double* U, double* S, double* V);

// api.cu
smp_status fail(smp_ctx* c, smp_status s, const std::string& msg);
smp_status check_cuda(smp_ctx* c, cudaError_t e, const char* what);
smp_status read_device_error(smp_ctx* c);

}  // namespace smp
