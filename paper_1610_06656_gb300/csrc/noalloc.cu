// smp_sketch_noalloc: the single-pass sketch of one row range written straight into caller buffers, with every
// byte of scratch taken from a fixed array compiled into this library instead of from cudaMalloc.
//
// Who needs it: code that is handed device memory but may not allocate any. Examples are a plug-in running inside
// a host framework that owns the whole device-memory budget through its own pool (a stray cudaMalloc can push the
// process over that budget or fragment the pool), and latency-critical loops where cudaMalloc / cudaFree would
// synchronise the device and stall work queued on other streams.
//
// The scratch (row-split partial sketches and partial column sums) lives in g_noalloc_scratch, a __device__ array
// of SMP_NOALLOC_SCRATCH_BYTES at file scope (internal linkage). Every GPU that loads this library holds that much
// memory until the process exits. Host code cannot pass the array's name to a kernel (in host code it is only a
// host-side stand-in for the symbol), so the first call in each CUDA context looks up the array's device address
// with cudaGetSymbolAddress and caches it under the context's unique id: a device reset or a second context on the
// same device gets a lookup of its own instead of a stale address.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)SMP_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxSplits = 8;
constexpr int64_t kMaxColumns = (int64_t)1 << 30;   // the same bound smp_sketch_begin puts on n1 and n2

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

std::mutex g_scratch_mu;
std::vector<std::pair<unsigned long long, void*>> g_scratch_addr;   // (context id, device address of the array)

template <typename F>
F driver_entry(const char* name) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return (F)p;
}

// Device address of g_noalloc_scratch in the current context (looked up on the first call in that context).
smp_status scratch_address(void** out) {
    static const CtxGetCurrentFn get_current = driver_entry<CtxGetCurrentFn>("cuCtxGetCurrent");
    static const CtxGetIdFn get_id = driver_entry<CtxGetIdFn>("cuCtxGetId");
    if (!get_current || !get_id)
        return smp::fail(nullptr, SMP_ECUDA, "smp_sketch_noalloc: driver entry points cuCtxGetCurrent / cuCtxGetId");
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) {
        // no context current yet: let the runtime set up the current device's primary context
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return smp::check_cuda(nullptr, e, "smp_sketch_noalloc: cudaGetSymbolAddress");
        if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr)
            return smp::fail(nullptr, SMP_ECUDA, "smp_sketch_noalloc: no current CUDA context");
    }
    unsigned long long id = 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return smp::fail(nullptr, SMP_ECUDA, "smp_sketch_noalloc: cuCtxGetId");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    for (const auto& kv : g_scratch_addr)
        if (kv.first == id) {
            *out = kv.second;
            return SMP_OK;
        }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
        return smp::check_cuda(nullptr, e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                               "smp_sketch_noalloc: cudaGetSymbolAddress of the scratch array");
    g_scratch_addr.emplace_back(id, p);
    *out = p;
    return SMP_OK;
}

}  // namespace

extern "C" smp_status smp_sketch_noalloc(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n1,
                                         int64_t n2, int32_t k, int32_t dtype, uint64_t seed, int64_t row0,
                                         int64_t nrows, float* At, float* Bt, double* sA, double* sB,
                                         void* stream) {
    using smp::fail;
    if (dtype != SMP_F32 && dtype != SMP_BF16)
        return fail(nullptr, SMP_EUNSUPPORTED, "smp_sketch_noalloc: dtype must be SMP_F32 or SMP_BF16");
    if (n1 < 1 || n2 < 1 || n1 > kMaxColumns || n2 > kMaxColumns || k < 1 || k > 1024 || nrows < 0 || row0 < 0 ||
        nrows > INT64_MAX - row0)
        return fail(nullptr, SMP_EINVAL,
                    "smp_sketch_noalloc: need 1 <= n1, n2 <= 2^30, 1 <= k <= 1024, nrows, row0 >= 0, row0 + nrows "
                    "representable");
    if (!At || !Bt || !sA || !sB) return fail(nullptr, SMP_EINVAL, "smp_sketch_noalloc: null output");
    if (nrows > 0 && (!A || !B || lda < n1 || ldb < n2))
        return fail(nullptr, SMP_EINVAL, "smp_sketch_noalloc: null input or leading dimension too small");
    const int64_t ntot = n1 + n2;
    const int64_t ldk = smp::round_up(k, 4);
    // one split needs ntot * ldk floats of partial sketch and ntot doubles of partial column sums
    const size_t part_split = (size_t)ntot * (size_t)ldk * 4;
    const size_t nsq_split = (size_t)ntot * 8;
    const size_t per_split = smp::round_up((int64_t)part_split, 256) + smp::round_up((int64_t)nsq_split, 256);
    if (per_split > kScratchBytes)
        return fail(nullptr, SMP_EINVAL,
                    "smp_sketch_noalloc: (n1 + n2) x k = " + std::to_string(ntot) + " x " + std::to_string(k) +
                        " needs " + std::to_string(per_split) + " bytes of scratch, more than the fixed " +
                        std::to_string(kScratchBytes) + "; use smp_sketch_begin for this size");
    const int splits = (int)std::min<size_t>(kMaxSplits, kScratchBytes / per_split);
    void* base = nullptr;
    smp_status s = scratch_address(&base);
    if (s != SMP_OK) return s;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return smp::check_cuda(nullptr, e, "smp_sketch_noalloc: device query");
    cudaStream_t st = (cudaStream_t)stream;
    // the row splits the kernel will write: only their partials are cleared and reduced
    const int used = smp::simt_into_splits(ntot, k, nrows, splits, sms);
    const size_t part_bytes = smp::round_up((int64_t)(part_split * used), 256);
    float* part = (float*)base;
    double* nsq = (double*)((char*)base + part_bytes);
    // the array keeps the previous call's partials: clear what this call accumulates into
    e = cudaMemsetAsync(base, 0, part_bytes + nsq_split * used, st);
    if (e != cudaSuccess) return smp::check_cuda(nullptr, e, "smp_sketch_noalloc: clearing scratch");
    e = smp::launch_sketch_simt_into(dtype, A, lda, B, ldb, n1, n2, k, seed, row0, nrows, part, nsq, used, sms, At,
                                     Bt, sA, sB, st);
    return smp::check_cuda(nullptr, e, "smp_sketch_noalloc: kernel launch");
}
