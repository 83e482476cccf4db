// smp_sketch_noalloc: the single-pass sketch of one row range written straight into caller buffers, with every
// byte of scratch taken from a fixed array compiled into this library instead of from cudaMalloc.
//
// Who needs it: code that is handed device memory but may not allocate any. Examples are a plug-in running inside
// a host framework that owns the whole device-memory budget through its own pool (a stray cudaMalloc can push the
// process over that budget or fragment the pool), and latency-critical loops where cudaMalloc / cudaFree would
// synchronise the device and stall work queued on other streams.
//
// The scratch (row-split partial sketches and partial column sums) lives in g_noalloc_scratch, a file-scope
// __device__ array of SMP_NOALLOC_SCRATCH_BYTES. Every GPU that loads this library holds that much memory until
// the process exits. Host code cannot pass the array's name to a kernel (in host code it is only a host-side
// stand-in for the symbol), so the first call on each device, with that device current, looks up its device
// address once with cudaGetSymbolAddress and caches it per device.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)SMP_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
constexpr int kMaxSplits = 8;

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up on the first call for that device).
smp_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return smp::check_cuda(nullptr, e, "smp_sketch_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return smp::fail(nullptr, SMP_EUNSUPPORTED, "smp_sketch_noalloc: device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return smp::check_cuda(nullptr, e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                   "smp_sketch_noalloc: cudaGetSymbolAddress of the scratch array");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
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
    if (n1 < 1 || n2 < 1 || k < 1 || k > 1024 || nrows < 0 || row0 < 0)
        return fail(nullptr, SMP_EINVAL, "smp_sketch_noalloc: need n1, n2 >= 1, 1 <= k <= 1024, nrows, row0 >= 0");
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
    int splits = (int)std::min<size_t>(kMaxSplits, kScratchBytes / per_split);
    void* base = nullptr;
    smp_status s = scratch_address(&base);
    if (s != SMP_OK) return s;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return smp::check_cuda(nullptr, e, "smp_sketch_noalloc: device query");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t part_bytes = smp::round_up((int64_t)(part_split * splits), 256);
    float* part = (float*)base;
    double* nsq = (double*)((char*)base + part_bytes);
    // the array keeps the previous call's partials: clear what this call accumulates into
    e = cudaMemsetAsync(base, 0, part_bytes + nsq_split * splits, st);
    if (e != cudaSuccess) return smp::check_cuda(nullptr, e, "smp_sketch_noalloc: clearing scratch");
    e = smp::launch_sketch_simt_into(dtype, A, lda, B, ldb, n1, n2, k, seed, row0, nrows, part, nsq, splits, sms, At,
                                     Bt, sA, sB, st);
    return smp::check_cuda(nullptr, e, "smp_sketch_noalloc: kernel launch");
}
