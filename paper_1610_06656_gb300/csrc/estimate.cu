// Rescaled JL estimate over Omega (Algorithm 1, step 4; Eq. (2)), as a sampled dense-dense product (SDDMM):
// M~(i, j) = D_A,i D_B,j <At_i, Bt_j>, the compact form D_A At^T Bt D_B with (D_X)_cc = ||X_c|| / ||Xt_c||
// (Appendix B). One warp per CSR row i keeps At_i in registers and walks the row's columns; each Bt_j (k
// contiguous values) is read with coalesced lane-strided loads from L2 and reduced with warp shuffles.
#include "common.cuh"
#include "internal.h"

namespace smp {
namespace {

template <typename T, int NPL>
__global__ void __launch_bounds__(256) estimate_kernel(const T* __restrict__ At, const T* __restrict__ Bt,
                                                       int64_t ldk, int k, const double* __restrict__ DA,
                                                       const double* __restrict__ DB,
                                                       const int64_t* __restrict__ row_ptr,
                                                       const int32_t* __restrict__ col, int64_t n1, T* vals) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n1) return;
    const int64_t i = warp;
    T a[NPL];
    const T* ai = At + i * ldk;
#pragma unroll
    for (int q = 0; q < NPL; ++q) {
        const int idx = lane + 32 * q;
        a[q] = idx < k ? ai[idx] : T(0);
    }
    const double da = DA[i];
    const int64_t p0 = row_ptr[i], p1 = row_ptr[i + 1];
    int64_t p = p0;
    // two columns per iteration for memory-level parallelism
    for (; p + 1 < p1; p += 2) {
        const int64_t j0 = col[p], j1 = col[p + 1];
        const T* b0 = Bt + j0 * ldk;
        const T* b1 = Bt + j1 * ldk;
        T s0 = T(0), s1 = T(0);
#pragma unroll
        for (int q = 0; q < NPL; ++q) {
            const int idx = lane + 32 * q;
            if (idx < k) {
                s0 = fma(a[q], b0[idx], s0);
                s1 = fma(a[q], b1[idx], s1);
            }
        }
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
        if (lane == 0) {
            vals[p] = (T)(da * DB[j0] * (double)s0);
            vals[p + 1] = (T)(da * DB[j1] * (double)s1);
        }
    }
    if (p < p1) {
        const int64_t j0 = col[p];
        const T* b0 = Bt + j0 * ldk;
        T s0 = T(0);
#pragma unroll
        for (int q = 0; q < NPL; ++q) {
            const int idx = lane + 32 * q;
            if (idx < k) s0 = fma(a[q], b0[idx], s0);
        }
        s0 = warp_sum(s0);
        if (lane == 0) vals[p] = (T)(da * DB[j0] * (double)s0);
    }
}

template <typename T, int NPL>
void launch_npl(smp_ctx* c, void* vals) {
    const T* At = (const T*)c->sk;
    const T* Bt = c->p.same_ab ? At : At + c->p.n1 * c->ldk;
    const double* DA = c->D_all;
    const double* DB = c->p.same_ab ? c->D_all : c->D_all + c->p.n1;
    const int64_t warps = c->p.n1;
    const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    estimate_kernel<T, NPL><<<smp::counted(blocks), 256, 0, c->stream>>>(At, Bt, c->ldk, c->p.k, DA, DB, c->row_ptr, c->col,
                                                           c->p.n1, (T*)vals);
}

template <typename T>
void launch_typed(smp_ctx* c, void* vals) {
    const int k = c->p.k;
    if (k <= 128) launch_npl<T, 4>(c, vals);
    else if (k <= 256) launch_npl<T, 8>(c, vals);
    else if (k <= 512) launch_npl<T, 16>(c, vals);
    else launch_npl<T, 32>(c, vals);
}

}  // namespace

cudaError_t launch_estimate(smp_ctx* c, void* vals) {
    if (c->nnz == 0) return cudaSuccess;
    if (c->acc_bytes == 8) launch_typed<double>(c, vals);
    else launch_typed<float>(c, vals);
    return cudaGetLastError();
}

}  // namespace smp
