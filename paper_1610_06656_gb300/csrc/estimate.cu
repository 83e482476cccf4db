// Rescaled JL estimate over Omega (Algorithm 1, step 4; Eq. (2)), as a sampled dense-dense product (SDDMM):
// M~(i, j) = D_A,i D_B,j <At_i, Bt_j>, the compact form D_A At^T Bt D_B with (D_X)_cc = ||X_c|| / ||Xt_c||
// (Appendix B).
//
// Work is split by CSR position, not by row: rows of heavy columns keep every entry (q^ = 1 across the row) and
// would otherwise serialise on one warp. Each warp takes CHUNK consecutive entries; it keeps At_i in registers
// while the row index stays the same (rows are contiguous in CSR order), reads each Bt_j (k contiguous values)
// with coalesced lane-strided loads from L2, reduces with warp shuffles, and scales in binary64.
#include "common.cuh"
#include "internal.h"

namespace smp {
namespace {

constexpr int CHUNK = 8;

template <typename T, int NPL>
__global__ void __launch_bounds__(256) estimate_kernel(const T* __restrict__ At, const T* __restrict__ Bt,
                                                       int64_t ldk, int k, const double* __restrict__ DA,
                                                       const double* __restrict__ DB,
                                                       const int32_t* __restrict__ erow,
                                                       const int32_t* __restrict__ col, int64_t nnz, T* vals) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t p0 = warp * CHUNK;
    if (p0 >= nnz) return;
    const int64_t p1 = min(nnz, p0 + CHUNK);
    int64_t cur = -1;
    double da = 0.0;
    T a[NPL];
    for (int64_t p = p0; p < p1; ++p) {
        const int64_t i = erow[p];
        if (i != cur) {
            cur = i;
            da = DA[i];
            const T* ai = At + i * ldk;
#pragma unroll
            for (int q = 0; q < NPL; ++q) {
                const int idx = lane + 32 * q;
                a[q] = idx < k ? ai[idx] : T(0);
            }
        }
        const int64_t j = col[p];
        const T* bj = Bt + j * ldk;
        T s = T(0);
#pragma unroll
        for (int q = 0; q < NPL; ++q) {
            const int idx = lane + 32 * q;
            if (idx < k) s = fma(a[q], bj[idx], s);
        }
        s = warp_sum(s);
        if (lane == 0) vals[p] = (T)(da * DB[j] * (double)s);
    }
}

// k > 1024: the same sums without caching At_i in registers (lanes stride over the sketch rows).
template <typename T>
__global__ void __launch_bounds__(256) estimate_long_kernel(const T* __restrict__ At, const T* __restrict__ Bt,
                                                            int64_t ldk, int k, const double* __restrict__ DA,
                                                            const double* __restrict__ DB,
                                                            const int32_t* __restrict__ erow,
                                                            const int32_t* __restrict__ col, int64_t nnz, T* vals) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= nnz) return;
    const int64_t i = erow[p], j = col[p];
    const T* ai = At + i * ldk;
    const T* bj = Bt + j * ldk;
    T s = T(0);
    for (int idx = lane; idx < k; idx += 32) s = fma(ai[idx], bj[idx], s);
    s = warp_sum(s);
    if (lane == 0) vals[p] = (T)(DA[i] * DB[j] * (double)s);
}

template <typename T, int NPL>
void launch_npl(smp_ctx* c, void* vals) {
    const T* At = (const T*)c->sk;
    const T* Bt = c->p.same_ab ? At : At + c->p.n1 * c->ldk;
    const double* DA = c->D_all;
    const double* DB = c->p.same_ab ? c->D_all : c->D_all + c->p.n1;
    const int64_t warps = (c->nnz + CHUNK - 1) / CHUNK;
    const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    estimate_kernel<T, NPL><<<smp::counted(blocks), 256, 0, c->stream>>>(At, Bt, c->ldk, c->p.k, DA, DB, c->erow,
                                                                         c->col, c->nnz, (T*)vals);
}

template <typename T>
void launch_typed(smp_ctx* c, void* vals) {
    const int k = c->p.k;
    if (k <= 128) launch_npl<T, 4>(c, vals);
    else if (k <= 256) launch_npl<T, 8>(c, vals);
    else if (k <= 512) launch_npl<T, 16>(c, vals);
    else if (k <= 1024) launch_npl<T, 32>(c, vals);
    else {
        const T* At = (const T*)c->sk;
        const T* Bt = c->p.same_ab ? At : At + c->p.n1 * c->ldk;
        const double* DB = c->p.same_ab ? c->D_all : c->D_all + c->p.n1;
        estimate_long_kernel<T><<<smp::counted((unsigned)((c->nnz * 32 + 255) / 256)), 256, 0, c->stream>>>(
            At, Bt, c->ldk, k, c->D_all, DB, c->erow, c->col, c->nnz, (T*)vals);
    }
}

}  // namespace

cudaError_t launch_estimate(smp_ctx* c, void* vals) {
    if (c->nnz == 0) return cudaSuccess;
    if (c->acc_bytes == 8) launch_typed<double>(c, vals);
    else launch_typed<float>(c, vals);
    return cudaGetLastError();
}

}  // namespace smp
