// Single-pass sketch on CUDA cores (Algorithm 1, step 2; Section 2.1 "Step 1") and the finalize step.
//
// sketch_simt_kernel: one CTA owns a 64-column x 64-sketch-row output tile over one row split. Per 32-row step it
// stages the data tile in shared memory, generates the matching 64 x 32 tile of Pi from Philox (or reads the
// caller's Pi in the explicit-Pi test mode), and accumulates Pi_tile * X_tile with FMAs; the CTAs of the first
// sketch-row chunk also fold the squares of the data tile into compensated column sums (Ogita-Rump-Oishi
// TwoSum with the exact FMA residual of each square). Partials go to [split][column][row] and are reduced in a
// fixed order by finalize, so the result is bitwise reproducible.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace smp {
namespace {

constexpr int TN = 64;   // data columns per CTA
constexpr int TK = 64;   // sketch rows per CTA
constexpr int TR = 32;   // data rows per step

template <typename T>
struct Arith;
template <>
struct Arith<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
};
template <>
struct Arith<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
};

// Compensated sum of squares: x^2 = p + e exactly (FMA residual), p is added with TwoSum, both errors go to lo.
template <typename T>
__device__ __forceinline__ void add_square(T x, T& hi, T& lo) {
    using A = Arith<T>;
    const T p = A::mul(x, x);
    const T e = A::fma(x, x, -p);
    const T s = A::add(hi, p);
    const T bp = A::sub(s, hi);
    const T err = A::add(A::sub(hi, A::sub(s, bp)), A::sub(p, bp));
    hi = s;
    lo = A::add(lo, A::add(err, e));
}

__device__ __forceinline__ float load_elem(const float* p, float) { return *p; }
__device__ __forceinline__ float load_elem(const __nv_bfloat16* p, float) { return __bfloat162float(*p); }
__device__ __forceinline__ double load_elem(const double* p, double) { return *p; }

template <typename TAcc>
__device__ __forceinline__ void gauss4(uint64_t t, int g, uint32_t k0, uint32_t k1, TAcc scale, TAcc z[4]);
template <>
__device__ __forceinline__ void gauss4<float>(uint64_t t, int g, uint32_t k0, uint32_t k1, float scale,
                                              float z[4]) {
    const U32x4 x = philox4x32_10((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)g, TAG_PI, k0, k1);
    box_muller_f32(x.x, x.y, z[0], z[1]);
    box_muller_f32(x.z, x.w, z[2], z[3]);
#pragma unroll
    for (int q = 0; q < 4; ++q) z[q] *= scale;
}
template <>
__device__ __forceinline__ void gauss4<double>(uint64_t t, int g, uint32_t k0, uint32_t k1, double scale,
                                               double z[4]) {
    const U32x4 x = philox4x32_10((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)g, TAG_PI, k0, k1);
    box_muller_f64(x.x, x.y, z[0], z[1]);
    box_muller_f64(x.z, x.w, z[2], z[3]);
#pragma unroll
    for (int q = 0; q < 4; ++q) z[q] *= scale;
}

template <typename TIn, typename TAcc>
struct SketchArgs {
    const TIn* A;
    const TIn* B;
    const TAcc* Pi;     // explicit Pi (k x nrows, ld = ldp) or null
    int64_t lda, ldb, ldp;
    int64_t n1, ntot;
    int64_t row0, nrows, rows_per_split;
    int k;
    int64_t ldk;
    uint32_t key0, key1;
    TAcc scale;         // 1 / sqrt(k)
    TAcc* part;         // [splits][ntot][ldk]
    double* nsq;        // [splits][ntot]
};

template <typename TIn, typename TAcc>
__global__ void __launch_bounds__(256) sketch_simt_kernel(const SketchArgs<TIn, TAcc> a) {
    __shared__ __align__(16) TAcc xs[TR][TN + 4];
    __shared__ __align__(16) TAcc ps[TR][TK + 4];
    __shared__ double nred[4][TN];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t c0 = (int64_t)blockIdx.x * TN;
    const int a0 = blockIdx.y * TK;
    const int s = blockIdx.z;
    const int64_t rs = (int64_t)s * a.rows_per_split;
    const int64_t re = min(a.nrows, rs + a.rows_per_split);
    const bool do_norm = blockIdx.y == 0;
    const int ncol = tid & 63, nq = tid >> 6;

    TAcc acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = TAcc(0);
    TAcc nhi = TAcc(0), nlo = TAcc(0);

    for (int64_t t0 = rs; t0 < re; t0 += TR) {
        {   // data tile: thread -> one row, 8 consecutive columns
            const int lr = tid >> 3, cs = (tid & 7) * 8;
            const int64_t row = t0 + lr;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int64_t c = c0 + cs + e;
                TAcc v = TAcc(0);
                if (row < re && c < a.ntot) {
                    const TIn* src = c < a.n1 ? a.A + row * a.lda + c : a.B + row * a.ldb + (c - a.n1);
                    v = load_elem(src, TAcc(0));
                }
                xs[lr][cs + e] = v;
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {   // Pi tile: thread -> one data row, one Philox group of 4 sketch rows
            const int rr = (tid >> 4) + 16 * h, g = tid & 15;
            const int arow = a0 + 4 * g;
            const int64_t row = t0 + rr;
            TAcc z[4] = {TAcc(0), TAcc(0), TAcc(0), TAcc(0)};
            if (row < re && arow < a.k) {
                if (a.Pi) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (arow + q < a.k) z[q] = a.Pi[(int64_t)(arow + q) * a.ldp + row];
                } else {
                    gauss4<TAcc>((uint64_t)(a.row0 + row), arow >> 2, a.key0, a.key1, a.scale, z);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (arow + q >= a.k) z[q] = TAcc(0);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) ps[rr][4 * g + q] = z[q];
        }
        __syncthreads();
#pragma unroll 8
        for (int tt = 0; tt < TR; ++tt) {
            TAcc pa[4], xc[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                pa[q] = ps[tt][ty * 4 + q];
                xc[q] = xs[tt][tx * 4 + q];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(pa[i], xc[j], acc[i][j]);
        }
        if (do_norm) {
#pragma unroll
            for (int rr = 0; rr < TR / 4; ++rr) add_square<TAcc>(xs[nq * (TR / 4) + rr][ncol], nhi, nlo);
        }
        __syncthreads();
    }

    const int64_t pbase = (int64_t)s * a.ntot;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t c = c0 + tx * 4 + j;
        if (c >= a.ntot) continue;
        TAcc* dst = a.part + (pbase + c) * a.ldk + a0 + ty * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (a0 + ty * 4 + i < a.ldk) dst[i] += acc[i][j];
    }
    if (do_norm) {
        nred[nq][ncol] = (double)nhi + (double)nlo;
        __syncthreads();
        if (tid < TN && c0 + tid < a.ntot) {
            double v = nred[0][tid];
            v += nred[1][tid];
            v += nred[2][tid];
            v += nred[3][tid];
            a.nsq[pbase + c0 + tid] += v;
        }
    }
}

template <typename TIn, typename TAcc>
cudaError_t launch_simt_typed(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                              int64_t nrows, const void* Pi, int64_t ldp) {
    SketchArgs<TIn, TAcc> a;
    a.A = (const TIn*)A;
    a.B = (const TIn*)(c->p.same_ab ? A : B);
    a.Pi = (const TAcc*)Pi;
    a.lda = lda;
    a.ldb = c->p.same_ab ? lda : ldb;
    a.ldp = ldp;
    a.n1 = c->p.n1;
    a.ntot = c->ntot;
    a.row0 = row0;
    a.nrows = nrows;
    const int64_t steps = (nrows + TR - 1) / TR;
    const int64_t tiles = ((c->ntot + TN - 1) / TN) * ((c->p.k + TK - 1) / TK);
    int splits = (int)std::min<int64_t>(c->splits, std::max<int64_t>(1, (2 * c->sm_count + tiles - 1) / tiles));
    splits = (int)std::min<int64_t>(splits, std::max<int64_t>(1, steps));
    a.rows_per_split = ((steps + splits - 1) / splits) * TR;
    a.k = c->p.k;
    a.ldk = c->ldk;
    a.key0 = (uint32_t)c->p.seed;
    a.key1 = (uint32_t)(c->p.seed >> 32);
    a.scale = (TAcc)(1.0 / sqrt((double)c->p.k));
    a.part = (TAcc*)c->part;
    a.nsq = c->nsq;
    dim3 grid((unsigned)((c->ntot + TN - 1) / TN), (unsigned)((c->p.k + TK - 1) / TK), (unsigned)splits);
    sketch_simt_kernel<TIn, TAcc><<<smp::counted(grid), 256, 0, c->stream>>>(a);
    return cudaGetLastError();
}

// Finalize: fixed-order reduction of the split partials; ||Xt_c||^2 by a fixed-shape block tree in double;
// s_c = sum over splits (fixed order); D_c = sqrt(s_c) / ||Xt_c|| (0 when the sketch column is zero).
template <typename TAcc>
__global__ void __launch_bounds__(256) finalize_kernel(const TAcc* __restrict__ part, const double* __restrict__ nsq,
                                                       int splits, int64_t ntot, int k, int64_t ldk, TAcc* sk,
                                                       double* s_all, double* D_all) {
    __shared__ double red[8];
    const int64_t c = blockIdx.x;
    double ss = 0.0;
    for (int a = threadIdx.x; a < ldk; a += blockDim.x) {
        TAcc v = TAcc(0);
        for (int s = 0; s < splits; ++s) v += part[((int64_t)s * ntot + c) * ldk + a];
        if (a >= k) v = TAcc(0);
        sk[c * ldk + a] = v;
        ss += (double)v * (double)v;
    }
    ss = warp_sum(ss);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double n2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) n2 += red[w];
        double sc = 0.0;
        for (int s = 0; s < splits; ++s) sc += nsq[(int64_t)s * ntot + c];
        s_all[c] = sc;
        D_all[c] = n2 > 0.0 ? sqrt(sc) / sqrt(n2) : 0.0;
    }
}

// ||X||_F^2 summed strictly left to right: the order the sampler's reading fixes. ||A||_F^2 on thread 0 and
// ||B||_F^2 on thread 32 (two warps, so the two dependent chains run side by side).
__global__ void frobenius_kernel(const double* s_all, int64_t n1, int64_t n2, int same_ab, double* F) {
    if (blockIdx.x != 0) return;
    if (threadIdx.x == 0) {
        double fa = 0.0;
        for (int64_t i = 0; i < n1; ++i) fa = __dadd_rn(fa, s_all[i]);
        F[0] = fa;
        if (same_ab) F[1] = fa;
    } else if (threadIdx.x == 32 && !same_ab) {
        double fb = 0.0;
        for (int64_t j = 0; j < n2; ++j) fb = __dadd_rn(fb, s_all[n1 + j]);
        F[1] = fb;
    }
}

// Import: copy caller sketch columns (n x k, dense) into the padded layout and recompute D.
template <typename TAcc>
__global__ void __launch_bounds__(256) import_kernel(const TAcc* __restrict__ At, const TAcc* __restrict__ Bt,
                                                     int64_t n1, int64_t ntot, int k, int64_t ldk, TAcc* sk,
                                                     const double* sA, const double* sB, double* s_all,
                                                     double* D_all) {
    __shared__ double red[8];
    const int64_t c = blockIdx.x;
    const TAcc* src = c < n1 ? At + c * k : Bt + (c - n1) * k;
    double ss = 0.0;
    for (int a = threadIdx.x; a < ldk; a += blockDim.x) {
        const TAcc v = a < k ? src[a] : TAcc(0);
        sk[c * ldk + a] = v;
        ss += (double)v * (double)v;
    }
    ss = warp_sum(ss);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double n2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) n2 += red[w];
        const double sc = c < n1 ? sA[c] : sB[c - n1];
        s_all[c] = sc;
        D_all[c] = n2 > 0.0 ? sqrt(sc) / sqrt(n2) : 0.0;
    }
}

}  // namespace

cudaError_t launch_sketch_simt(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                               int64_t nrows, const void* Pi, int64_t ldp) {
    switch (c->p.dtype) {
        case SMP_F32: return launch_simt_typed<float, float>(c, A, lda, B, ldb, row0, nrows, Pi, ldp);
        case SMP_BF16: return launch_simt_typed<__nv_bfloat16, float>(c, A, lda, B, ldb, row0, nrows, Pi, ldp);
        case SMP_F64: return launch_simt_typed<double, double>(c, A, lda, B, ldb, row0, nrows, Pi, ldp);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_frobenius(smp_ctx* c) {
    frobenius_kernel<<<smp::counted(1), 64, 0, c->stream>>>(c->s_all, c->p.n1, c->p.n2, c->p.same_ab, c->F);
    return cudaGetLastError();
}

cudaError_t launch_finalize(smp_ctx* c) {
    const unsigned nb = (unsigned)c->ntot;
    if (c->acc_bytes == 8)
        finalize_kernel<double><<<smp::counted(nb), 256, 0, c->stream>>>((const double*)c->part, c->nsq, c->splits, c->ntot,
                                                          c->p.k, c->ldk, (double*)c->sk, c->s_all, c->D_all);
    else
        finalize_kernel<float><<<smp::counted(nb), 256, 0, c->stream>>>((const float*)c->part, c->nsq, c->splits, c->ntot,
                                                         c->p.k, c->ldk, (float*)c->sk, c->s_all, c->D_all);
    frobenius_kernel<<<smp::counted(1), 64, 0, c->stream>>>(c->s_all, c->p.n1, c->p.n2, c->p.same_ab, c->F);
    return cudaGetLastError();
}

cudaError_t launch_import(smp_ctx* c, const void* At, const void* Bt, const double* sA, const double* sB) {
    const unsigned nb = (unsigned)c->ntot;
    const void* bt = c->p.same_ab ? At : Bt;
    const double* sb = c->p.same_ab ? sA : sB;
    if (c->acc_bytes == 8)
        import_kernel<double><<<smp::counted(nb), 256, 0, c->stream>>>((const double*)At, (const double*)bt, c->p.n1, c->ntot,
                                                        c->p.k, c->ldk, (double*)c->sk, sA, sb, c->s_all,
                                                        c->D_all);
    else
        import_kernel<float><<<smp::counted(nb), 256, 0, c->stream>>>((const float*)At, (const float*)bt, c->p.n1, c->ntot,
                                                       c->p.k, c->ldk, (float*)c->sk, sA, sb, c->s_all, c->D_all);
    frobenius_kernel<<<smp::counted(1), 64, 0, c->stream>>>(c->s_all, c->p.n1, c->p.n2, c->p.same_ab, c->F);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------------------------
// The same SIMT sketch over one row range with caller-supplied split partials, and the fixed-order reduction of
// those partials into dense caller outputs. Used only by the allocation-free entry point in noalloc.cu.
// ---------------------------------------------------------------------------------------------------------------
namespace {

__global__ void __launch_bounds__(256) reduce_into_kernel(const float* __restrict__ part,
                                                          const double* __restrict__ nsq, int splits, int64_t n1,
                                                          int64_t ntot, int k, int64_t ldk, float* At, float* Bt,
                                                          double* sA, double* sB) {
    const int64_t c = blockIdx.x;
    float* dst = c < n1 ? At + c * k : Bt + (c - n1) * k;
    for (int a = threadIdx.x; a < k; a += blockDim.x) {
        float v = 0.0f;
        for (int s = 0; s < splits; ++s) v += part[((int64_t)s * ntot + c) * ldk + a];
        dst[a] = v;
    }
    if (threadIdx.x == 0) {
        double sc = 0.0;
        for (int s = 0; s < splits; ++s) sc += nsq[(int64_t)s * ntot + c];
        if (c < n1) sA[c] = sc;
        else sB[c - n1] = sc;
    }
}

template <typename TIn>
cudaError_t sketch_into_typed(const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n1, int64_t n2, int k,
                              uint64_t seed, int64_t row0, int64_t nrows, float* part, double* nsq, int splits,
                              int sm_count, cudaStream_t st) {
    SketchArgs<TIn, float> a;
    a.A = (const TIn*)A;
    a.B = (const TIn*)B;
    a.Pi = nullptr;
    a.lda = lda;
    a.ldb = ldb;
    a.ldp = 0;
    a.n1 = n1;
    a.ntot = n1 + n2;
    a.row0 = row0;
    a.nrows = nrows;
    const int64_t steps = (nrows + TR - 1) / TR;
    const int used = simt_into_splits(a.ntot, k, nrows, splits, sm_count);
    a.rows_per_split = ((steps + used - 1) / used) * TR;
    a.k = k;
    a.ldk = round_up(k, 4);
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.scale = (float)(1.0 / sqrt((double)k));
    a.part = part;
    a.nsq = nsq;
    dim3 grid((unsigned)((a.ntot + TN - 1) / TN), (unsigned)((k + TK - 1) / TK), (unsigned)used);
    if (nrows > 0) sketch_simt_kernel<TIn, float><<<smp::counted(grid), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

int simt_into_splits(int64_t ntot, int k, int64_t nrows, int splits, int sm_count) {
    const int64_t steps = (nrows + TR - 1) / TR;
    const int64_t tiles = ((ntot + TN - 1) / TN) * ((k + TK - 1) / TK);
    int used = (int)std::min<int64_t>(splits, std::max<int64_t>(1, (2 * sm_count + tiles - 1) / tiles));
    return (int)std::min<int64_t>(used, std::max<int64_t>(1, steps));
}

cudaError_t launch_sketch_simt_into(int dtype, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t n1,
                                    int64_t n2, int k, uint64_t seed, int64_t row0, int64_t nrows, float* part,
                                    double* nsq, int splits, int sm_count, float* At, float* Bt, double* sA,
                                    double* sB, cudaStream_t st) {
    cudaError_t e = dtype == SMP_BF16
                        ? sketch_into_typed<__nv_bfloat16>(A, lda, B, ldb, n1, n2, k, seed, row0, nrows, part, nsq,
                                                           splits, sm_count, st)
                        : sketch_into_typed<float>(A, lda, B, ldb, n1, n2, k, seed, row0, nrows, part, nsq, splits,
                                                   sm_count, st);
    if (e != cudaSuccess) return e;
    reduce_into_kernel<<<smp::counted((unsigned)(n1 + n2)), 256, 0, st>>>(part, nsq, splits, n1, n1 + n2, k,
                                                                          round_up(k, 4), At, Bt, sA, sB);
    return cudaGetLastError();
}

}  // namespace smp
