// WAltMin (Algorithm 2, Appendix A) and the canonical form of its output.
//
//  * weights w = 1/q^ (step 2); optional split of Omega into 2T+1 subsets by the split coin (step 3);
//  * U0: top-r left singular subspace of R_Omega0(M~) = w .* P_Omega0(M~) (steps 4-5) by block subspace iteration
//    with b = min(2r + 8, 72, n1, n2) columns: Y <- orth(R (R^T Y)) with entry-parallel CSR / CSC products and a
//    Cholesky-QR (twice) whose factorisation runs in binary64, then a Rayleigh-Ritz step on Z = R^T Y; trim (6);
//  * T rounds of the two weighted least-squares half-steps (steps 8 and 9). Each output row's samples are cut into
//    segments of at most SEG entries; one warp per segment accumulates the partial Gram G = sum w f f^T and
//    b = sum w M~ f (lane l owns column l of G); one thread per output row then sums its segments in binary64, adds
//    the ridge 1e-10 tr(G)/r and solves by its own binary64 Cholesky;
//  * canonical form: Cholesky-QR (twice) of U^ and V^, the SVD of the r x r core Ru Rv^T via the symmetric
//    eigenproblem of [[0, K], [K^T, 0]], and the sign rule (largest-magnitude entry of each U column positive).
//
// Binary64 is used where the method needs it (the r x r and b x b factorisations, the canonical form); the
// per-sample arithmetic stays in binary32 unless SMP_FP64_ALS asks otherwise, because binary64 throughput on this
// part is about 1/40 of binary32.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "dense_small.cuh"
#include "internal.h"

namespace smp {
namespace {

constexpr int SEG = 64;          // samples per LS segment
constexpr int LS_WARPS = 4;      // segments per CTA in the Gram kernel
constexpr int CHECK_EVERY = 4;   // subspace-iteration steps between convergence checks

// ---------------------------------------------------------------------------------------------------------------
// weights, split, values of R_Omega(M~)
// ---------------------------------------------------------------------------------------------------------------
__global__ void split_kernel(const int32_t* __restrict__ erow, const int32_t* __restrict__ col, int64_t nnz, int T,
                             uint32_t k0, uint32_t k1, uint8_t* sub) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const double u = coin((uint32_t)erow[e], (uint32_t)col[e], TAG_SPLIT, k0, k1);
    const double f = floor(__dmul_rn(u, (double)(2 * T + 1)));
    sub[e] = (uint8_t)min((int)f, 2 * T);
}

// rv[e] = w_e M~_e for entries of subset sid (0 elsewhere), in CSR order; rv_csc = the same values in CSC order.
template <typename TV, typename TR>
__global__ void rvals_kernel(const TV* __restrict__ vals, const double* __restrict__ qhat,
                             const uint8_t* __restrict__ sub, int sid, const int64_t* __restrict__ csc_pos,
                             int64_t nnz, TR* rv, TR* rv_csc) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    auto value = [&](int64_t p) {
        const double q = qhat[p];
        const double w = q > 0.0 ? 1.0 / q : 0.0;
        const bool in = sub == nullptr || sub[p] == sid;
        return in ? (TR)(w * (double)vals[p]) : TR(0);
    };
    rv[e] = value(e);
    rv_csc[e] = value(csc_pos[e]);
}

// ---------------------------------------------------------------------------------------------------------------
// initial subspace (block subspace iteration)
// ---------------------------------------------------------------------------------------------------------------
template <typename TY>
__global__ void start_block_kernel(int64_t n1, int b, uint32_t k0, uint32_t k1, TY* Y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t groups = (b + 3) / 4;
    if (e >= n1 * groups) return;
    const int64_t i = e / groups;
    const int g = (int)(e - i * groups);
    const U32x4 x = philox4x32_10((uint32_t)i, 0u, (uint32_t)g, TAG_INIT, k0, k1);
    float z[4];
    box_muller_f32(x.x, x.y, z[0], z[1]);
    box_muller_f32(x.z, x.w, z[2], z[3]);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (4 * g + q < b) Y[i * b + 4 * g + q] = (TY)z[q];
}

// Partial sparse product of one segment: Yp[s] = sum over the segment's entries p of val[p] X[idx[p]] (lanes over
// the b columns, BCH chunks of 32; the segment's indices and values are loaded once per 32 entries and broadcast).
template <typename TY, int BCH>
__global__ void __launch_bounds__(256) spmm_seg_kernel(const int64_t* __restrict__ seg_b,
                                                       const int64_t* __restrict__ seg_e, int64_t nseg,
                                                       const int32_t* __restrict__ idx, const TY* __restrict__ val,
                                                       const TY* __restrict__ X, int b, TY* Yp) {
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= nseg) return;
    TY acc[BCH];
#pragma unroll
    for (int h = 0; h < BCH; ++h) acc[h] = TY(0);
    const int64_t p0 = seg_b[s], p1 = seg_e[s];
    for (int64_t base = p0; base < p1; base += 32) {
        const int64_t p = base + lane;
        const int32_t in = p < p1 ? idx[p] : 0;
        const TY v = p < p1 ? val[p] : TY(0);
        const int cnt = (int)(p1 - base < 32 ? p1 - base : 32);
#pragma unroll 4
        for (int t = 0; t < cnt; ++t) {
            const int32_t in_t = __shfl_sync(0xffffffffu, in, t);
            const TY v_t = __shfl_sync(0xffffffffu, v, t);
            const TY* x = X + (int64_t)in_t * b;
#pragma unroll
            for (int h = 0; h < BCH; ++h)
                if (h * 32 + lane < b) acc[h] = fma(v_t, x[h * 32 + lane], acc[h]);
        }
    }
#pragma unroll
    for (int h = 0; h < BCH; ++h)
        if (h * 32 + lane < b) Yp[s * b + h * 32 + lane] = acc[h];
}

// Y[o][c] = sum of the segment partials of row o, in segment order.
template <typename TY>
__global__ void spmm_reduce_kernel(const int64_t* __restrict__ seg_start, const TY* __restrict__ Yp, int64_t n_out,
                                   int b, TY* Y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_out * b) return;
    const int64_t o = e / b;
    const int c = (int)(e - o * b);
    TY acc = TY(0);
    for (int64_t s = seg_start[o]; s < seg_start[o + 1]; ++s) acc += Yp[s * b + c];
    Y[e] = acc;
}

// U0[i][c] = sum_l Y[i][l] E[l][c] for the top-r Ritz vectors (E: b x b, eigenvectors in columns, sorted).
template <typename TY>
__global__ void ritz_kernel(const TY* __restrict__ Y, const double* __restrict__ E, int64_t n1, int b, int r,
                            double* U0) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n1 * r) return;
    const int64_t i = e / r;
    const int c = (int)(e - i * r);
    double s = 0.0;
    for (int l = 0; l < b; ++l) s = fma((double)Y[i * b + l], E[l * b + c], s);
    U0[e] = s;
}

// Rayleigh-Ritz rotation of the whole block: Yout = Y E (n1 x b times b x b), so the iteration continues in the
// Ritz basis and the next check's b x b matrix is nearly diagonal (its Jacobi sweeps converge at once).
template <typename TY>
__global__ void rotate_kernel(const TY* __restrict__ Y, const double* __restrict__ E, int64_t n1, int b, TY* Yout) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n1 * b) return;
    const int64_t i = e / b;
    const int c = (int)(e - i * b);
    TY s = TY(0);
    for (int l = 0; l < b; ++l) s = fma(Y[i * b + l], (TY)E[l * b + c], s);
    Yout[e] = s;
}

// Trim (step 6): zero row i when ||U0^i|| > 8 sqrt(r) ||A_i|| / ||A||_F.
__global__ void trim_kernel(double* U0, int64_t n1, int r, const double* __restrict__ sA,
                            const double* __restrict__ F) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n1) return;
    const double fa = F[0];
    double rn = 0.0;
    for (int c = 0; c < r; ++c) rn += U0[i * r + c] * U0[i * r + c];
    rn = sqrt(rn);
    const double thr = fa > 0.0 ? 8.0 * sqrt((double)r) * sqrt(sA[i]) / sqrt(fa) : 0.0;
    if (rn > thr)
        for (int c = 0; c < r; ++c) U0[i * r + c] = 0.0;
}

template <typename TA, typename TB>
__global__ void convert_kernel(const TA* __restrict__ a, int64_t n, TB* b) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] = (TB)a[e];
}

// ---------------------------------------------------------------------------------------------------------------
// weighted least-squares half-step
// ---------------------------------------------------------------------------------------------------------------
// Segments: each output row o is cut into max(1, ceil(len / SEG)) pieces of at most SEG consecutive entries.
__global__ void seg_count_kernel(const int64_t* __restrict__ ptr, int64_t n, int32_t* cnt) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int64_t len = ptr[o + 1] - ptr[o];
    cnt[o] = (int32_t)(len > SEG ? (len + SEG - 1) / SEG : 1);
}

// Exclusive scan of n int32 counts into int64 offsets (out has n + 1 entries). One CTA, chunked, fixed order.
__global__ void scan_kernel(const int32_t* __restrict__ cnt, int64_t n, int64_t* out) {
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < n; base += blockDim.x) {
        const int64_t idx = base + threadIdx.x;
        const int64_t c = idx < n ? (int64_t)cnt[idx] : 0;
        int64_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int64_t v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            wsum[lane] = v;
        }
        __syncthreads();
        const int64_t excl = x - c + (wid ? wsum[wid - 1] : 0) + carry;
        if (idx < n) out[idx] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + c;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
}

// Segment bounds: [seg_b, seg_e) for every segment of every output row.
__global__ void seg_fill_kernel(const int64_t* __restrict__ ptr, const int64_t* __restrict__ seg_start, int64_t n,
                                int64_t* seg_b, int64_t* seg_e) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int64_t s0 = seg_start[o], s1 = seg_start[o + 1];
    for (int64_t s = s0; s < s1; ++s) {
        const int64_t b0 = ptr[o] + (s - s0) * SEG;
        seg_b[s] = b0;
        seg_e[s] = min(ptr[o + 1], b0 + SEG);
    }
}

// Partial Gram of one segment: lane l accumulates column l of G; each sample's factor row is loaded once
// (lane c <- F[c]) and broadcast. part[s] = G (r x r, full) followed by b (r).
template <typename TF, typename TG, typename TV, int RMAX>
__global__ void __launch_bounds__(32 * LS_WARPS) seg_gram_kernel(
    const int64_t* __restrict__ seg_b, const int64_t* __restrict__ seg_e, int64_t nseg,
    const int32_t* __restrict__ idx, const int64_t* __restrict__ pos, const TV* __restrict__ vals,
    const double* __restrict__ qhat, const uint8_t* __restrict__ sub, int sid, const TF* __restrict__ Fin, int r,
    TG* part) {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * LS_WARPS + wid;
    if (s >= nseg) return;
    TG g[RMAX];
#pragma unroll
    for (int a = 0; a < RMAX; ++a) g[a] = TG(0);
    TG bl = TG(0);
    const int64_t p0 = seg_b[s], p1 = seg_e[s];
    for (int64_t base = p0; base < p1; base += 32) {
        const int64_t p = base + lane;
        int32_t in = 0;
        TG wv = TG(0), mv = TG(0);
        if (p < p1) {
            const int64_t e = pos ? pos[p] : p;
            in = idx[p];
            const bool use = sub == nullptr || sub[e] == sid;
            const double q = qhat[e];
            wv = (use && q > 0.0) ? (TG)(1.0 / q) : TG(0);
            mv = (TG)vals[e];
        }
        const int cnt = (int)(p1 - base < 32 ? p1 - base : 32);
        for (int t = 0; t < cnt; ++t) {
            const int32_t in_t = __shfl_sync(0xffffffffu, in, t);
            const TG w_t = __shfl_sync(0xffffffffu, wv, t);
            const TG m_t = __shfl_sync(0xffffffffu, mv, t);
            const TG f = lane < r ? (TG)Fin[(int64_t)in_t * r + lane] : TG(0);
            const TG wf = w_t * f;
#pragma unroll
            for (int a = 0; a < RMAX; ++a) g[a] = fma(wf, __shfl_sync(0xffffffffu, f, a), g[a]);
            bl = fma(wf, m_t, bl);
        }
    }
    TG* dst = part + s * (int64_t)(r * r + r);
    if (lane < r) {
#pragma unroll
        for (int a = 0; a < RMAX; ++a)
            if (a < r) dst[a * r + lane] = g[a];
        dst[r * r + lane] = bl;
    }
}

// Gc[o] (binary64) = sum of the segment partials of output row o, in segment order and in the partials' type (binary32
// partials summed in binary32, as the lane path for r <= 12 does: binary64 arithmetic, conversions included, issues
// about one warp instruction per 64 cycles per SM sub-partition here, and summing binary32 partials in it took
// 70 us at n = 1,504, r = 20): the packed lower triangle of G (r (r + 1) / 2 values) followed by b (r values). One
// warp per row; lanes over the r^2 + r partial values (every segment read with coalesced loads).
template <typename TG, int RMAX>
__global__ void __launch_bounds__(256) seg_reduce_kernel(const int64_t* __restrict__ seg_start,
                                                         const TG* __restrict__ part, int r, int64_t n_out,
                                                         double* Gc) {
    constexpr int Q = (RMAX * RMAX + RMAX + 31) / 32;
    const int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (o >= n_out) return;
    const int stride = r * r + r;
    const int nt = r * (r + 1) / 2;
    double* dst = Gc + o * (int64_t)(nt + r);
    TG acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = TG(0);
    // four segments' values are loaded before they are added (in segment order): rows with many samples (the
    // large-norm rows get most of them) have dozens of segments, and a round trip per segment made them the tail
    const int64_t s0 = seg_start[o], s1 = seg_start[o + 1];
    for (int64_t sg = s0; sg < s1; sg += 4) {
        TG v[4][Q];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const TG* ps = part + (sg + u) * (int64_t)stride;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int e = q * 32 + lane;
                v[u][q] = (sg + u < s1 && e < stride) ? ps[e] : TG(0);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < Q; ++q)
                if (sg + u < s1) acc[q] += v[u][q];
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int e = q * 32 + lane;
        if (e < r * r) {
            const int i = e / r, j = e - i * r;
            if (j <= i) dst[i * (i + 1) / 2 + j] = (double)acc[q];
        } else if (e < stride) {
            dst[nt + (e - r * r)] = (double)acc[q];
        }
    }
}

// Ridge, Cholesky and solve of each output row's compact binary64 system with one warp per row (r <= 32), for the
// orders where one thread per row is too long a binary64 chain: binary64 issues about one warp instruction per 64
// cycles per SM sub-partition, so a row per thread puts r^3 / 6 dependent instructions on one warp of every 32 rows
// (47 warps for n = 1,504 at r = 20: 0.18 ms), while a warp per row spreads the factorisation over every
// sub-partition. The factorisation is
// right-looking: lane 0 takes the pivot, the lanes scale the column below it and then share the trailing update's
// (i, k) pairs; the substitutions keep y[i] in lane i and broadcast each solved entry. Eight rows per CTA, each with
// its packed triangle in shared memory.
template <typename TF>
__global__ void __launch_bounds__(256) solve_warp_kernel(const double* __restrict__ Gc, int r, int64_t n_out,
                                                         TF* Xout, int* err) {
    constexpr int W = 8;
    __shared__ double Lsm[W][32 * 33 / 2];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t o = (int64_t)blockIdx.x * W + w;
    if (o >= n_out) return;   // warp-uniform
    double* L = Lsm[w];
    auto T = [](int i) { return i * (i + 1) / 2; };
    const int nt = T(r);
    const double* src = Gc + o * (int64_t)(nt + r);
    for (int e = lane; e < nt; e += 32) L[e] = src[e];
    double y = lane < r ? src[nt + lane] : 0.0;
    __syncwarp();
    double tr = lane < r ? L[T(lane) + lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, off);
    if (!(tr > 0.0)) {
        if (lane < r) Xout[o * r + lane] = TF(0);
        return;
    }
    const double lam = 1e-10 * tr / (double)r;
    if (lane < r) L[T(lane) + lane] += lam;
    __syncwarp();
    double rj_mine = 0.0;   // lane j keeps 1 / L[j][j]
    for (int j = 0; j < r; ++j) {
        const double d = L[T(j) + j];   // the same value in every lane: the branch below is warp-uniform
        if (!(d > 0.0)) {
            if (lane == 0) set_error(err, DEVERR_NUMERIC);
            if (lane < r) Xout[o * r + lane] = TF(0);
            return;
        }
        const double rj = rsqrt_refined(d);
        if (lane == j) rj_mine = rj;
        __syncwarp();
        if (lane == 0) L[T(j) + j] = d * rj;
        for (int i = j + 1 + lane; i < r; i += 32) L[T(i) + j] *= rj;
        __syncwarp();
        // pairs (i, k), j < k <= i < r, numbered p = a (a + 1) / 2 + c with i = j + 1 + a, k = j + 1 + c
        const int m = r - j - 1;
        const int np = T(m);
        for (int p = lane; p < np; p += 32) {
            int a = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
            if (T(a + 1) <= p) ++a;
            if (T(a) > p) --a;
            const int i = j + 1 + a, k = j + 1 + (p - T(a));
            L[T(i) + k] = fma(-L[T(i) + j], L[T(k) + j], L[T(i) + k]);
        }
        __syncwarp();
    }
    for (int j = 0; j < r; ++j) {   // L z = y
        const double zj = __shfl_sync(0xffffffffu, y, j) * __shfl_sync(0xffffffffu, rj_mine, j);
        if (lane == j) y = zj;
        else if (lane > j && lane < r) y = fma(-L[T(lane) + j], zj, y);
    }
    for (int j = r - 1; j >= 0; --j) {   // L^T x = z
        const double xj = __shfl_sync(0xffffffffu, y, j) * __shfl_sync(0xffffffffu, rj_mine, j);
        if (lane == j) y = xj;
        else if (lane < j) y = fma(-L[T(j) + lane], xj, y);
    }
    if (lane < r) Xout[o * r + lane] = (TF)y;
}

// The same ridge + Cholesky solve with each row's system held in registers (r <= R: R (R + 1) / 2 + 2 R doubles).
// Binary64 on this part issues about one warp instruction per 64 cycles per SM sub-partition whatever the number of
// active lanes, so a warp's binary64 instruction count sets the time; registers remove a shared-memory round trip
// for every operand. Every index is a template constant (the loops are generated by
// recursion, so no array is indexed at run time and nothing goes to local memory); r only enters warp-uniform guards.
template <int R>
struct RegChol {
    __host__ __device__ static constexpr int T(int i) { return i * (i + 1) / 2; }   // row i of the packed triangle
    // acc -= sum_{k < N} L[a + k] L[b + k]
    template <int N, int A, int B>
    static __device__ __forceinline__ void dot(const double (&L)[R * (R + 1) / 2], double& acc) {
        if constexpr (N > 0) {
            dot<N - 1, A, B>(L, acc);
            acc = fma(-L[A + N - 1], L[B + N - 1], acc);
        }
    }
    // rows I.. of column J below the pivot: L[I][J] = (L[I][J] - sum_k L[I][k] L[J][k]) / L[J][J]
    template <int J, int I>
    static __device__ __forceinline__ void below(double (&L)[R * (R + 1) / 2], double rj, int r) {
        if constexpr (I < R) {
            if (I < r) {
                double v = L[T(I) + J];
                dot<J, T(I), T(J)>(L, v);
                L[T(I) + J] = v * rj;
            }
            below<J, I + 1>(L, rj, r);
        }
    }
    template <int J>
    static __device__ __forceinline__ void factor(double (&L)[R * (R + 1) / 2], double (&ri)[R], int r, bool& bad) {
        if constexpr (J < R) {
            if (J < r) {
                double d = L[T(J) + J];
                dot<J, T(J), T(J)>(L, d);
                // a pivot that is not a positive normal number marks the system (2^-1022 is far below the ridge)
                const bool ok = d >= 2.2250738585072014e-308 && d <= 1.7976931348623157e308;
                bad = bad || !ok;
                const double rj = ok ? rsqrt_scaled(d) : 0.0;
                ri[J] = rj;
                L[T(J) + J] = d * rj;
                below<J, J + 1>(L, rj, r);
            }
            factor<J + 1>(L, ri, r, bad);
        }
    }
    // y[I] = (y[I] - sum_{k < I} L[I][k] y[k]) ri[I], I = 0, 1, ...
    template <int N, int A>
    static __device__ __forceinline__ void doty(const double (&L)[R * (R + 1) / 2], const double (&y)[R], double& acc) {
        if constexpr (N > 0) {
            doty<N - 1, A>(L, y, acc);
            acc = fma(-L[A + N - 1], y[N - 1], acc);
        }
    }
    template <int I>
    static __device__ __forceinline__ void forward(const double (&L)[R * (R + 1) / 2], const double (&ri)[R],
                                                   double (&y)[R], int r) {
        if constexpr (I < R) {
            if (I < r) {
                double v = y[I];
                doty<I, T(I)>(L, y, v);
                y[I] = v * ri[I];
            }
            forward<I + 1>(L, ri, y, r);
        }
    }
    // y[I] = (y[I] - sum_{k > I, k < r} L[k][I] y[k]) ri[I], I = R - 1, ..., 0
    template <int I, int K>
    static __device__ __forceinline__ void colsum(const double (&L)[R * (R + 1) / 2], const double (&y)[R], int r,
                                                  double& acc) {
        if constexpr (K < R) {
            if (K < r) acc = fma(-L[T(K) + I], y[K], acc);
            colsum<I, K + 1>(L, y, r, acc);
        }
    }
    template <int I>
    static __device__ __forceinline__ void backward(const double (&L)[R * (R + 1) / 2], const double (&ri)[R],
                                                    double (&y)[R], int r) {
        if constexpr (I >= 0) {
            if (I < r) {
                double v = y[I];
                colsum<I, I + 1>(L, y, r, v);
                y[I] = v * ri[I];
            }
            backward<I - 1>(L, ri, y, r);
        }
    }
};

template <typename TF, int R>
__global__ void __launch_bounds__(32) solve_reg_kernel(const double* __restrict__ Gc, int r, int64_t n_out, TF* Xout,
                                                       int* err) {
    using C = RegChol<R>;
    const int64_t o = (int64_t)blockIdx.x * 32 + threadIdx.x;
    if (o >= n_out) return;
    const int nt = r * (r + 1) / 2;
    const double* src = Gc + o * (int64_t)(nt + r);
    double L[R * (R + 1) / 2], y[R], ri[R];
#pragma unroll
    for (int e = 0; e < R * (R + 1) / 2; ++e) L[e] = e < nt ? src[e] : 0.0;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        y[i] = i < r ? src[nt + i] : 0.0;
        ri[i] = 0.0;
    }
    double tr = 0.0;
#pragma unroll
    for (int i = 0; i < R; ++i)
        if (i < r) tr += L[C::T(i) + i];
    const bool empty = !(tr > 0.0);
    const double lam = 1e-10 * tr / (double)r;
#pragma unroll
    for (int i = 0; i < R; ++i)
        if (i < r) L[C::T(i) + i] += lam;
    bool bad = false;   // not positive definite: the factorisation runs on, the row gets x = 0
    C::template factor<0>(L, ri, r, bad);
    if (empty || bad) {
        if (bad && !empty) set_error(err, DEVERR_NUMERIC);
        for (int i = 0; i < r; ++i) Xout[o * r + i] = TF(0);
        return;
    }
    C::template forward<0>(L, ri, y, r);
    C::template backward<R - 1>(L, ri, y, r);
#pragma unroll
    for (int i = 0; i < R; ++i)
        if (i < r) Xout[o * r + i] = (TF)y[i];
}

// ---------------------------------------------------------------------------------------------------------------
// canonical form
// ---------------------------------------------------------------------------------------------------------------
// K = Ru Rv^T (r x r), the core whose SVD gives the canonical form.
__global__ void core_kernel(const double* __restrict__ Ru, const double* __restrict__ Rv, int r, double* K) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= r * r) return;
    const int i = e / r, j = e - i * r;
    double v = 0.0;
    for (int l = 0; l < r; ++l) v = fma(Ru[i * r + l], Rv[j * r + l], v);
    K[e] = v;
}

// X_out (n x r) = Q (n x r) * Wc (r x r)
__global__ void small_right_mul_kernel(const double* __restrict__ Q, const double* __restrict__ Wc, int64_t n,
                                       int r, double* Xout) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * r) return;
    const int64_t i = e / r;
    const int c = (int)(e - i * r);
    double s = 0.0;
    for (int l = 0; l < r; ++l) s = fma(Q[i * r + l], Wc[l * r + c], s);
    Xout[e] = s;
}

// Sign rule: one CTA per column c of U; find the largest |U_ic| (lowest i on ties); flip U and V columns if < 0.
__global__ void sign_kernel(double* U, int64_t n1, double* V, int64_t n2, int r) {
    __shared__ double bv[256];
    __shared__ int64_t bi[256];
    const int c = blockIdx.x;
    double best = -1.0;
    int64_t besti = 0;
    for (int64_t i = threadIdx.x; i < n1; i += blockDim.x) {
        const double a = fabs(U[i * r + c]);
        if (a > best) {
            best = a;
            besti = i;
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = besti;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double o = bv[threadIdx.x + s];
            const int64_t oi = bi[threadIdx.x + s];
            if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = o;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const bool flip = U[bi[0] * r + c] < 0.0;
    __syncthreads();
    if (!flip) return;
    for (int64_t i = threadIdx.x; i < n1; i += blockDim.x) U[i * r + c] = -U[i * r + c];
    for (int64_t i = threadIdx.x; i < n2; i += blockDim.x) V[i * r + c] = -V[i * r + c];
}

__global__ void upper_mul_kernel(const double* __restrict__ R2, const double* __restrict__ R1, int b, double* R) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b * b) return;
    const int i = e / b, j = e - i * b;
    double s = 0.0;
    for (int l = i; l <= j; ++l) s += R2[i * b + l] * R1[l * b + j];
    R[e] = j >= i ? s : 0.0;
}

// ---------------------------------------------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------------------------------------------
struct Arena {
    char* base = nullptr;
    size_t used = 0, cap = 0;
    template <typename T>
    T* take(int64_t n) {
        used = (used + 255) & ~size_t(255);
        T* p = (T*)(base + used);
        used += (size_t)std::max<int64_t>(n, 1) * sizeof(T);
        return p;
    }
};

unsigned nblocks(int64_t n, int threads) { return (unsigned)std::max<int64_t>(1, (n + threads - 1) / threads); }

// Gram of X (n x a) with Y (n x b) into G (a x b), fixed-order reduction.
template <typename TX, typename TY>
void gram(const TX* X, const TY* Y, int64_t n, int a, int b, double* part, double* G, cudaStream_t st) {
    const int nblk = (int)std::max<int64_t>(1, (n + GRAM_ROWS_PER_BLOCK - 1) / GRAM_ROWS_PER_BLOCK);
    gram_partial_kernel<TX, TY><<<smp::counted(nblk), 256, 0, st>>>(X, Y, n, a, b, part);
    gram_reduce_kernel<<<smp::counted(nblocks(a * b * 32, 256)), 256, 0, st>>>(part, nblk, a * b, G);
}

// Cholesky-QR twice: Q = X R^-1 with X = Q R; Rout = R2 R1 (upper). Q may alias X. The Gram matrices and the
// factorisations are binary64; the substitutions run in TC.
// Upper Cholesky factor R of the Gram matrix X^T X (X: n x b): partial Gram blocks, their fixed-order reduction,
// then the register Cholesky (b <= 32) or the shared-memory one.
template <typename TX>
void gram_chol(const TX* X, int64_t n, int b, double* part, double* G, double* R, cudaStream_t st) {
    const int nblk = (int)std::max<int64_t>(1, (n + GRAM_ROWS_PER_BLOCK - 1) / GRAM_ROWS_PER_BLOCK);
    gram_partial_kernel<TX, TX><<<smp::counted(nblk), 256, 0, st>>>(X, X, n, b, b, part);
    gram_reduce_kernel<<<smp::counted(nblocks(b * b * 32, 256)), 256, 0, st>>>(part, nblk, b * b, G);
    if (b <= 32)
        chol32_kernel<<<smp::counted(1), 128, 0, st>>>(G, b, R, 1e-28);
    else
        chol_par_kernel<<<smp::counted(1), 128, 0, st>>>(G, b, R, 1e-28);
}

// Xout = Xin R^-1 (the row in registers; instantiations for b <= 32, 48 and MAX_SMALL).
template <typename TIn, typename TOut, typename TC>
void apply_rinv(const TIn* Xin, int64_t n, int b, const double* R, TOut* Xout, cudaStream_t st) {
    const unsigned g = smp::counted(nblocks(n, 128));
    if (b <= 32)
        apply_rinv_kernel<TIn, TOut, TC, 32><<<g, 128, 0, st>>>(Xin, n, b, R, Xout);
    else if (b <= 48)
        apply_rinv_kernel<TIn, TOut, TC, 48><<<g, 128, 0, st>>>(Xin, n, b, R, Xout);
    else
        apply_rinv_kernel<TIn, TOut, TC, MAX_SMALL><<<g, 128, 0, st>>>(Xin, n, b, R, Xout);
}

template <typename TX, typename TQ, typename TC>
void cholqr2(const TX* X, int64_t n, int b, TQ* Q, double* part, double* G, double* R1, double* R2, double* Rout,
             cudaStream_t st) {
    gram_chol<TX>(X, n, b, part, G, R1, st);
    apply_rinv<TX, TQ, TC>(X, n, b, R1, Q, st);
    gram_chol<TQ>(Q, n, b, part, G, R2, st);
    apply_rinv<TQ, TQ, TC>(Q, n, b, R2, Q, st);
    if (Rout) upper_mul_kernel<<<smp::counted(nblocks(b * b, 256)), 256, 0, st>>>(R2, R1, b, Rout);
}

// The Jacobi eigen kernel takes up to 2 MAX_SMALL (MAX_SMALL + 1) elements of dynamic shared memory.
void jacobi_smem_attr() {
    static std::atomic<bool> done{false};
    if (done) return;
    cudaFuncSetAttribute(jacobi_eig_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * MAX_SMALL * (MAX_SMALL + 1) * 8);
    cudaFuncSetAttribute(jacobi_eig_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * MAX_SMALL * (MAX_SMALL + 1) * 4);
    done = true;
}

struct Segments {
    int64_t* start = nullptr;   // [n_out + 1]
    int64_t* b = nullptr;       // [nseg]
    int64_t* e = nullptr;       // [nseg]
    int64_t nseg = 0;
};

// Y (n_out x b) = sum over each output row's entries of val * X[idx]; Yp: scratch of nseg x b partials.
template <typename TY>
void spmm(const Segments& sg, const int32_t* idx, const TY* val, const TY* X, int64_t n_out, int b, TY* Yp, TY* Y,
          cudaStream_t st) {
    const unsigned g = nblocks(sg.nseg * 32, 256);
    if (b <= 32) spmm_seg_kernel<TY, 1><<<smp::counted(g), 256, 0, st>>>(sg.b, sg.e, sg.nseg, idx, val, X, b, Yp);
    else if (b <= 64) spmm_seg_kernel<TY, 2><<<smp::counted(g), 256, 0, st>>>(sg.b, sg.e, sg.nseg, idx, val, X, b, Yp);
    else spmm_seg_kernel<TY, 3><<<smp::counted(g), 256, 0, st>>>(sg.b, sg.e, sg.nseg, idx, val, X, b, Yp);
    spmm_reduce_kernel<TY><<<smp::counted(nblocks(n_out * b, 256)), 256, 0, st>>>(sg.start, Yp, n_out, b, Y);
}

// ---------------------------------------------------------------------------------------------------------------
// binary32 Gram path for r <= LANE_R: one sample per lane
// ---------------------------------------------------------------------------------------------------------------
constexpr int LANE_R = 12;
constexpr int LANE_NT = LANE_R * (LANE_R + 1) / 2;
constexpr int LANE_PS = (LANE_NT + LANE_R + 3) / 4 * 4;   // floats per segment partial (packed G, then b)
constexpr int LANE2_PS = (20 * 21 / 2 + 20 + 3) / 4 * 4;  // the same for the two-pass lane path (r <= 20)

// w_e = 1 / q^_e for every sample of Omega (binary32), once per WAltMin call.
__global__ void weights_kernel(const double* __restrict__ qhat, int64_t nnz, float* wt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const double q = qhat[e];
    wt[e] = q > 0.0 ? (float)(1.0 / q) : 0.f;
}

// Weighted Gram partials of one segment (<= 64 samples of one output row), one warp per segment, lane t taking
// samples t, t + 32: every lane accumulates w f f^T (packed lower triangle, rows < r) and w m f of its own samples
// in registers, then a butterfly transpose-sum over the lanes gives each value's segment total (fixed order).
// Layout of a partial: LANE_PS floats, G(a, c) at a (a + 1) / 2 + c, b(a) at LANE_NT + a, zeros beyond r.
template <typename TF, typename TV>
__global__ void __launch_bounds__(32 * LS_WARPS) seg_gram_lane_kernel(
    const int64_t* __restrict__ seg_b, const int64_t* __restrict__ seg_e, int64_t nseg,
    const int32_t* __restrict__ idx, const int64_t* __restrict__ pos, const TV* __restrict__ vals,
    const float* __restrict__ wt, const uint8_t* __restrict__ sub, int sid, const TF* __restrict__ Fin, int r,
    float* part) {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * LS_WARPS + wid;
    if (s >= nseg) return;
    float g[LANE_PS];
#pragma unroll
    for (int e = 0; e < LANE_PS; ++e) g[e] = 0.f;
    const int64_t p1 = seg_e[s];
    for (int64_t p = seg_b[s] + lane; p < p1; p += 32) {
        const int64_t e = pos ? pos[p] : p;
        if (sub != nullptr && sub[e] != sid) continue;
        const float w = wt[e];
        const float wm = w * (float)vals[e];
        const TF* fr = Fin + (int64_t)idx[p] * r;
        float f[LANE_R];
#pragma unroll
        for (int a = 0; a < LANE_R; ++a) f[a] = a < r ? (float)fr[a] : 0.f;
#pragma unroll
        for (int a = 0; a < LANE_R; ++a) {
            if (a < r) {
                const float wf = w * f[a];
#pragma unroll
                for (int c = 0; c <= a; ++c) g[a * (a + 1) / 2 + c] = fmaf(wf, f[c], g[a * (a + 1) / 2 + c]);
                g[LANE_NT + a] = fmaf(wm, f[a], g[LANE_NT + a]);
            }
        }
    }
    float* dst = part + s * (int64_t)LANE_PS;
#pragma unroll
    for (int c0 = 0; c0 < LANE_PS; c0 += 32) {
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = c0 + i < LANE_PS ? g[c0 + i] : 0.f;
        const float tot = transpose_sum32(v, lane);
        if (c0 + lane < LANE_PS) dst[c0 + lane] = tot;
    }
}

// The lane Gram path for 12 < r <= R (R = 20): one sample per lane as in seg_gram_lane_kernel, the packed triangle
// split over two passes over the segment's samples so each pass's accumulators fit in registers (pass 0: rows
// [0, RS); pass 1: rows [RS, R) and b). Against one warp per segment broadcasting each sample's factor row with
// shuffles (RMAX shuffles and FMAs per sample and lane), about a fifth of the instructions. Layout of a partial:
// G(a, c) at a (a + 1) / 2 + c, b(a) at R (R + 1) / 2 + a, zeros beyond r.
template <typename TF, typename TV, int R, int RS>
__global__ void __launch_bounds__(32 * LS_WARPS) seg_gram_lane2_kernel(
    const int64_t* __restrict__ seg_b, const int64_t* __restrict__ seg_e, int64_t nseg,
    const int32_t* __restrict__ idx, const int64_t* __restrict__ pos, const TV* __restrict__ vals,
    const float* __restrict__ wt, const uint8_t* __restrict__ sub, int sid, const TF* __restrict__ Fin, int r,
    float* part) {
    constexpr int NT = R * (R + 1) / 2;
    constexpr int PS = (NT + R + 3) / 4 * 4;
    constexpr int N0 = RS * (RS + 1) / 2;      // pass 0 values
    constexpr int N1 = NT - N0 + R;            // pass 1 values (rows RS.. of G, then b)
    constexpr int NA = N0 > N1 ? N0 : N1;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * LS_WARPS + wid;
    if (s >= nseg) return;
    const int64_t p1 = seg_e[s];
    float* dst = part + s * (int64_t)PS;
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        float g[NA];
#pragma unroll
        for (int e = 0; e < NA; ++e) g[e] = 0.f;
        for (int64_t p = seg_b[s] + lane; p < p1; p += 32) {
            const int64_t e = pos ? pos[p] : p;
            if (sub != nullptr && sub[e] != sid) continue;
            const float w = wt[e];
            const TF* fr = Fin + (int64_t)idx[p] * r;
            float f[R];
#pragma unroll
            for (int a = 0; a < R; ++a) f[a] = a < r ? (float)fr[a] : 0.f;
            if (pass == 0) {
#pragma unroll
                for (int a = 0; a < RS; ++a) {
                    const float wf = w * f[a];
#pragma unroll
                    for (int c = 0; c <= a; ++c) g[a * (a + 1) / 2 + c] = fmaf(wf, f[c], g[a * (a + 1) / 2 + c]);
                }
            } else {
                const float wm = w * (float)vals[e];
#pragma unroll
                for (int a = RS; a < R; ++a) {
                    const float wf = w * f[a];
#pragma unroll
                    for (int c = 0; c <= a; ++c)
                        g[a * (a + 1) / 2 - N0 + c] = fmaf(wf, f[c], g[a * (a + 1) / 2 - N0 + c]);
                }
#pragma unroll
                for (int a = 0; a < R; ++a) g[NT - N0 + a] = fmaf(wm, f[a], g[NT - N0 + a]);
            }
        }
        const int nv = pass == 0 ? N0 : N1, off = pass == 0 ? 0 : N0;
#pragma unroll
        for (int c0 = 0; c0 < NA; c0 += 32) {
            if (c0 < nv) {
                float v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = (c0 + i < NA && c0 + i < nv) ? g[c0 + i] : 0.f;
                const float tot = transpose_sum32(v, lane);
                if (c0 + lane < nv) dst[off + c0 + lane] = tot;
            }
        }
    }
    static_assert(R != 20 || PS == LANE2_PS, "partial size");
    if (lane < PS - NT - R) dst[NT + R + lane] = 0.f;   // padding
}

// Gc[o] (binary64, the layout the solves read: packed G of rows < r, then b) = sum of the row's segment partials
// of the lane Gram paths (R = LANE_R or 20), in segment order, in binary32. One warp per row, lanes over the
// partial's values.
template <int R>
__global__ void __launch_bounds__(256) seg_reduce_lane_kernel(const int64_t* __restrict__ seg_start,
                                                              const float* __restrict__ part, int r, int64_t n_out,
                                                              double* Gc) {
    constexpr int NTR = R * (R + 1) / 2;
    constexpr int PSR = (NTR + R + 3) / 4 * 4;
    const int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (o >= n_out) return;
    const int nt = r * (r + 1) / 2;
    double* dst = Gc + o * (int64_t)(nt + r);
    const int64_t s0 = seg_start[o], s1 = seg_start[o + 1];
    constexpr int Q = (PSR + 31) / 32;
    float acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = 0.f;
    for (int64_t s = s0; s < s1; s += 4) {   // four segments' loads in flight, added in segment order
        float v[4][Q];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int e = q * 32 + lane;
                v[u][q] = (s + u < s1 && e < PSR) ? part[(s + u) * (int64_t)PSR + e] : 0.f;
            }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < Q; ++q)
                if (s + u < s1) acc[q] += v[u][q];
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int e = q * 32 + lane;
        if (e < nt) dst[e] = (double)acc[q];
        else if (e >= NTR && e < NTR + r) dst[nt + (e - NTR)] = (double)acc[q];
    }
}

template <typename TF, typename TG, typename TV>
void launch_ls(int r, const Segments& sg, const int32_t* idx, const int64_t* pos, const TV* vals,
               const double* qhat, const float* wt, const uint8_t* sub, int sid, const TF* Fin, int64_t n_out,
               TG* part, double* Gc, TF* Xout, int* err, cudaStream_t st) {
    const unsigned g = nblocks(sg.nseg, LS_WARPS);
    const unsigned gr = nblocks(n_out * 32, 256);
    const unsigned gs = nblocks(n_out, 32);
    const unsigned gw = nblocks(n_out, 8);
    if (sizeof(TG) == 4 && r <= LANE_R) {
        seg_gram_lane_kernel<TF, TV><<<smp::counted(g), 32 * LS_WARPS, 0, st>>>(sg.b, sg.e, sg.nseg, idx, pos, vals,
                                                                                wt, sub, sid, Fin, r, (float*)part);
        seg_reduce_lane_kernel<LANE_R><<<smp::counted(gr), 256, 0, st>>>(sg.start, (const float*)part, r, n_out, Gc);
        solve_reg_kernel<TF, 12><<<smp::counted(gs), 32, 0, st>>>(Gc, r, n_out, Xout, err);
    } else if (sizeof(TG) == 4 && r <= 20) {
        seg_gram_lane2_kernel<TF, TV, 20, 14><<<smp::counted(g), 32 * LS_WARPS, 0, st>>>(
            sg.b, sg.e, sg.nseg, idx, pos, vals, wt, sub, sid, Fin, r, (float*)part);
        seg_reduce_lane_kernel<20><<<smp::counted(gr), 256, 0, st>>>(sg.start, (const float*)part, r, n_out, Gc);
        solve_warp_kernel<TF><<<smp::counted(gw), 256, 0, st>>>(Gc, r, n_out, Xout, err);
    } else if (r <= 8) {
        seg_gram_kernel<TF, TG, TV, 8><<<smp::counted(g), 32 * LS_WARPS, 0, st>>>(sg.b, sg.e, sg.nseg, idx, pos,
                                                                                  vals, qhat, sub, sid, Fin, r, part);
        seg_reduce_kernel<TG, 8><<<smp::counted(gr), 256, 0, st>>>(sg.start, part, r, n_out, Gc);
        solve_reg_kernel<TF, 12><<<smp::counted(gs), 32, 0, st>>>(Gc, r, n_out, Xout, err);
    } else if (r <= 16) {
        seg_gram_kernel<TF, TG, TV, 16><<<smp::counted(g), 32 * LS_WARPS, 0, st>>>(sg.b, sg.e, sg.nseg, idx, pos,
                                                                                   vals, qhat, sub, sid, Fin, r, part);
        seg_reduce_kernel<TG, 16><<<smp::counted(gr), 256, 0, st>>>(sg.start, part, r, n_out, Gc);
        if (r <= 12)
            solve_reg_kernel<TF, 12><<<smp::counted(gs), 32, 0, st>>>(Gc, r, n_out, Xout, err);
        else
            solve_warp_kernel<TF><<<smp::counted(gw), 256, 0, st>>>(Gc, r, n_out, Xout, err);
    } else if (r <= 20) {
        seg_gram_kernel<TF, TG, TV, 20><<<smp::counted(g), 32 * LS_WARPS, 0, st>>>(sg.b, sg.e, sg.nseg, idx, pos,
                                                                                   vals, qhat, sub, sid, Fin, r, part);
        seg_reduce_kernel<TG, 20><<<smp::counted(gr), 256, 0, st>>>(sg.start, part, r, n_out, Gc);
        solve_warp_kernel<TF><<<smp::counted(gw), 256, 0, st>>>(Gc, r, n_out, Xout, err);
    } else {
        seg_gram_kernel<TF, TG, TV, 32><<<smp::counted(g), 32 * LS_WARPS, 0, st>>>(sg.b, sg.e, sg.nseg, idx, pos,
                                                                                   vals, qhat, sub, sid, Fin, r, part);
        seg_reduce_kernel<TG, 32><<<smp::counted(gr), 256, 0, st>>>(sg.start, part, r, n_out, Gc);
        solve_warp_kernel<TF><<<smp::counted(gw), 256, 0, st>>>(Gc, r, n_out, Xout, err);
    }
}

template <typename TV, typename TF, typename TG, typename TY>
smp_status waltmin_typed(smp_ctx* c, const TV* vals, int r, int T, uint32_t flags, uint64_t seed,
                         const double* U_init, double* U, double* S, double* V) {
    const int64_t n1 = c->p.n1, n2 = c->p.n2, nnz = c->nnz;
    cudaStream_t st = c->stream;
    const int b = (int)std::min<int64_t>(std::min<int64_t>(2 * r + 8, MAX_SMALL), std::min(n1, n2));
    const bool split = (flags & SMP_SPLIT_OMEGA) != 0;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);

    // segments of the CSR rows and the CSC columns: an upper bound on their count sizes the scratch
    const int64_t nseg_max = nnz / SEG + n1 + n2 + 2;
    const int64_t nmax = std::max(n1, n2);
    const int64_t gblk = std::max<int64_t>(1, (nmax + GRAM_ROWS_PER_BLOCK - 1) / GRAM_ROWS_PER_BLOCK);
    size_t need = 0;
    auto add = [&](int64_t n, size_t sz) { need += ((size_t)std::max<int64_t>(n, 1) * sz + 511) & ~size_t(255); };
    add(nnz, 1);                             // sub
    add(2 * nnz, sizeof(TY));                // rv, rv_csc
    add(n1 * b, sizeof(TY));                 // Y
    add(n2 * b, sizeof(TY));                 // Z
    add(n1 * b, sizeof(TY));                 // Ytmp
    add(gblk * MAX_SMALL * MAX_SMALL, 8);    // gram partials
    add(5 * b * b + 4 * b, 8);               // G, R1, R2, E, evals
    add(2 * n1 * r, 8);                      // U0, U0prev
    add(n1 * r, sizeof(TF));                 // Uf
    add(n2 * r, sizeof(TF));                 // Vf
    add(n1 * r, 8);                          // Qu
    add(n2 * r, 8);                          // Qv
    add(12 * r * r + 8 * r, 8);              // Ru, Rv, K, W, Z, ...
    add(n1 + n2 + 2, 4);                     // segment counts
    add(n1 + n2 + 4, 8);                     // segment starts
    add(4 * nseg_max, 8);                    // segment begins / ends
    add(nseg_max * (int64_t)std::max(r * r + r, std::max(LANE_PS, LANE2_PS)), sizeof(TG));   // LS partials
    add(nnz, 4);                                        // binary32 weights 1 / q^
    add(nseg_max * (int64_t)b, sizeof(TY));             // SpMM segment partials
    add(nmax * (int64_t)(r * (r + 1) / 2 + r), 8);      // compact per-row systems
    void* ws = nullptr;
    if (dev_malloc(&ws, need, st) != cudaSuccess) return fail(c, SMP_ENOMEM, "smp_waltmin: scratch");
    Arena ar{(char*)ws, 0, need};
    uint8_t* sub = ar.take<uint8_t>(nnz);
    TY* rv = ar.take<TY>(nnz);
    TY* rv_csc = ar.take<TY>(nnz);
    TY* Y = ar.take<TY>(n1 * b);
    TY* Z = ar.take<TY>(n2 * b);
    TY* Yt = ar.take<TY>(n1 * b);
    double* part = ar.take<double>(gblk * MAX_SMALL * MAX_SMALL);
    double* G = ar.take<double>(b * b);
    double* R1 = ar.take<double>(b * b);
    double* R2 = ar.take<double>(b * b);
    double* E = ar.take<double>(b * b);
    double* ev = ar.take<double>(4 * b);
    double* U0 = ar.take<double>(n1 * r);
    double* U0p = ar.take<double>(n1 * r);
    TF* Uf = ar.take<TF>(n1 * r);
    TF* Vf = ar.take<TF>(n2 * r);
    double* Qu = ar.take<double>(n1 * r);
    double* Qv = ar.take<double>(n2 * r);
    double* Ru = ar.take<double>(r * r);
    double* Rv = ar.take<double>(r * r);
    double* H = ar.take<double>(4 * r * r);
    double* Wc = ar.take<double>(r * r);
    double* Zc = ar.take<double>(r * r);
    double* Rx1 = ar.take<double>(r * r);
    double* Rx2 = ar.take<double>(r * r);
    double* Gx = ar.take<double>(r * r);
    int32_t* seg_cnt = ar.take<int32_t>(n1 + n2 + 2);
    Segments rows_sg, cols_sg;
    rows_sg.start = ar.take<int64_t>(n1 + 1);
    cols_sg.start = ar.take<int64_t>(n2 + 1);
    int64_t* seg_be = ar.take<int64_t>(4 * nseg_max);
    TG* lspart = ar.take<TG>(nseg_max * (int64_t)std::max(r * r + r, std::max(LANE_PS, LANE2_PS)));
    float* wt = ar.take<float>(nnz);
    TY* Yp = ar.take<TY>(nseg_max * (int64_t)b);
    double* Gc = ar.take<double>(nmax * (int64_t)(r * (r + 1) / 2 + r));

    jacobi_smem_attr();

    // segments (Omega is fixed for the whole call); the count copy is the call's only early host sync
    seg_count_kernel<<<smp::counted(nblocks(n1, 256)), 256, 0, st>>>(c->row_ptr, n1, seg_cnt);
    scan_kernel<<<smp::counted(1), 1024, 0, st>>>(seg_cnt, n1, rows_sg.start);
    seg_count_kernel<<<smp::counted(nblocks(n2, 256)), 256, 0, st>>>(c->col_ptr, n2, seg_cnt + n1 + 1);
    scan_kernel<<<smp::counted(1), 1024, 0, st>>>(seg_cnt + n1 + 1, n2, cols_sg.start);
    int64_t counts[2] = {0, 0};
    cudaMemcpyAsync(&counts[0], rows_sg.start + n1, 8, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&counts[1], cols_sg.start + n2, 8, cudaMemcpyDeviceToHost, st);
    cudaError_t ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
        free_after(ws, st);
        return check_cuda(c, ce, "smp_waltmin: segment counts");
    }
    rows_sg.nseg = counts[0];
    cols_sg.nseg = counts[1];
    rows_sg.b = seg_be;
    rows_sg.e = seg_be + rows_sg.nseg;
    cols_sg.b = seg_be + 2 * rows_sg.nseg;
    cols_sg.e = cols_sg.b + cols_sg.nseg;
    seg_fill_kernel<<<smp::counted(nblocks(n1, 256)), 256, 0, st>>>(c->row_ptr, rows_sg.start, n1, rows_sg.b,
                                                                    rows_sg.e);
    seg_fill_kernel<<<smp::counted(nblocks(n2, 256)), 256, 0, st>>>(c->col_ptr, cols_sg.start, n2, cols_sg.b,
                                                                    cols_sg.e);

    if (split && nnz > 0)
        split_kernel<<<smp::counted(nblocks(nnz, 256)), 256, 0, st>>>(c->erow, c->col, nnz, T, k0, k1, sub);
    const uint8_t* subp = split ? sub : nullptr;
    smp_status status = SMP_OK;
    if (flags & SMP_INIT_GIVEN) {
        convert_kernel<double, TF><<<smp::counted(nblocks(n1 * r, 256)), 256, 0, st>>>(U_init, n1 * r, Uf);
    } else {
        // R_Omega0(M~) values in CSR and CSC order
        if (nnz > 0)
            rvals_kernel<TV, TY><<<smp::counted(nblocks(nnz, 256)), 256, 0, st>>>(vals, c->qhat, subp, 0,
                                                                                  c->csc_pos, nnz, rv, rv_csc);
        start_block_kernel<TY><<<smp::counted(nblocks(n1 * ((b + 3) / 4), 256)), 256, 0, st>>>(n1, b, k0, k1, Y);
        cholqr2<TY, TY, TY>(Y, n1, b, Y, part, G, R1, R2, nullptr, st);
        // Convergence. binary32 iterates: the top-r Ritz values (binary32 Jacobi) change by < 1e-6 relative between
        // checks. binary64 iterates: the top-r Ritz subspace (binary64 Jacobi) moves by < 1e-11 between checks.
        const bool dbl = sizeof(TY) == 8;
        const int max_iter = dbl ? 400 : 200;
        const int every = dbl ? 4 : 2;
        bool have_prev = false;
        std::vector<double> prev_ev(b, 0.0), cur_ev(b, 0.0);
        for (int it = 1; it <= max_iter; ++it) {
            spmm<TY>(cols_sg, c->csc_row, rv_csc, Y, n2, b, Yp, Z, st);   // Z = R^T Y
            spmm<TY>(rows_sg, c->col, rv, Z, n1, b, Yp, Yt, st);          // Y = R Z
            const bool check = it % every == 0 || it == max_iter;
            if (!check) {
                // between checks one Cholesky-QR pass: the next product only needs a well-conditioned basis of the
                // same span (orthogonality error ~ cond(Y) x unit roundoff); the checks orthonormalise twice
                gram_chol<TY>(Yt, n1, b, part, G, R1, st);
                apply_rinv<TY, TY, TY>(Yt, n1, b, R1, Y, st);
                continue;
            }
            cholqr2<TY, TY, TY>(Yt, n1, b, Y, part, G, R1, R2, nullptr, st);
            spmm<TY>(cols_sg, c->csc_row, rv_csc, Y, n2, b, Yp, Z, st);   // C = Z^T Z, Z = R^T Y
            gram<TY, TY>(Z, Z, n2, b, b, part, G, st);
            bool done = false;
            if (dbl) {
                launch_jacobi<double>(G, b, 4e-15, 40, ev, E, st);
                ritz_kernel<TY><<<smp::counted(nblocks(n1 * r, 256)), 256, 0, st>>>(Y, E, n1, b, r, U0);
                if (have_prev) {
                    gram<double, double>(U0, U0p, n1, r, r, part, Gx, st);
                    std::vector<double> hx(r * r);
                    cudaError_t e1 =
                        cudaMemcpyAsync(hx.data(), Gx, sizeof(double) * r * r, cudaMemcpyDeviceToHost, st);
                    if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(st);
                    if (e1 != cudaSuccess) {
                        status = check_cuda(c, e1, "smp_waltmin init check");
                        break;
                    }
                    double fro = 0.0;
                    for (double v : hx) fro += v * v;
                    done = std::sqrt(std::max(0.0, (double)r - fro)) < 1e-11;
                }
                cudaMemcpyAsync(U0p, U0, sizeof(double) * n1 * r, cudaMemcpyDeviceToDevice, st);
            } else {
                launch_jacobi<float>(G, b, 1e-6, 30, ev, E, st);
                cudaError_t e1 = cudaMemcpyAsync(cur_ev.data(), ev, sizeof(double) * b, cudaMemcpyDeviceToHost, st);
                if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(st);
                if (e1 != cudaSuccess) {
                    status = check_cuda(c, e1, "smp_waltmin init check");
                    break;
                }
                if (have_prev) {
                    double worst = 0.0;
                    for (int i = 0; i < r; ++i)
                        worst = std::max(worst, std::fabs(cur_ev[i] - prev_ev[i]) / std::max(cur_ev[0], 1e-300));
                    done = worst < 1e-6;
                }
                prev_ev = cur_ev;
            }
            have_prev = true;
            if (done || it == max_iter) {
                if (!dbl)   // Rayleigh-Ritz vectors from the binary32 eigenvectors of the last check
                    ritz_kernel<TY><<<smp::counted(nblocks(n1 * r, 256)), 256, 0, st>>>(Y, E, n1, b, r, U0);
                break;
            }
            if (!dbl) {   // continue from the Ritz basis
                rotate_kernel<TY><<<smp::counted(nblocks(n1 * b, 256)), 256, 0, st>>>(Y, E, n1, b, Yt);
                std::swap(Y, Yt);
            }
        }
        if (status == SMP_OK) {
            if (!(flags & SMP_NO_TRIM))
                trim_kernel<<<smp::counted(nblocks(n1, 256)), 256, 0, st>>>(U0, n1, r, c->s_all, c->F);
            convert_kernel<double, TF><<<smp::counted(nblocks(n1 * r, 256)), 256, 0, st>>>(U0, n1 * r, Uf);
        }
    }
    if (status == SMP_OK) {
        if (nnz > 0)
            weights_kernel<<<smp::counted(nblocks(nnz, 256)), 256, 0, st>>>(c->qhat, nnz, wt);
        for (int t = 0; t < T; ++t) {
            launch_ls<TF, TG, TV>(r, cols_sg, c->csc_row, c->csc_pos, vals, c->qhat, wt, subp, 2 * t + 1, Uf, n2,
                                  lspart, Gc, Vf, c->dev_err, st);
            launch_ls<TF, TG, TV>(r, rows_sg, c->col, nullptr, vals, c->qhat, wt, subp, 2 * t + 2, Vf, n1, lspart,
                                  Gc, Uf, c->dev_err, st);
        }
        if (T == 0) cudaMemsetAsync(Vf, 0, sizeof(TF) * n2 * r, st);
        // canonical form
        cholqr2<TF, double, double>(Uf, n1, r, Qu, part, Gx, Rx1, Rx2, Ru, st);
        cholqr2<TF, double, double>(Vf, n2, r, Qv, part, Gx, Rx1, Rx2, Rv, st);
        core_kernel<<<smp::counted(nblocks(r * r, 256)), 256, 0, st>>>(Ru, Rv, r, H);
        svd_onesided_kernel<<<smp::counted(1), 256, 0, st>>>(H, r, 4e-15, 40, S, Wc, Zc);
        small_right_mul_kernel<<<smp::counted(nblocks(n1 * r, 256)), 256, 0, st>>>(Qu, Wc, n1, r, U);
        small_right_mul_kernel<<<smp::counted(nblocks(n2 * r, 256)), 256, 0, st>>>(Qv, Zc, n2, r, V);
        sign_kernel<<<smp::counted(r), 256, 0, st>>>(U, n1, V, n2, r);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) status = check_cuda(c, e, "smp_waltmin kernels");
    }
    cudaError_t e = cudaStreamSynchronize(st);
    free_after(ws, st);
    if (status == SMP_OK && e != cudaSuccess) status = check_cuda(c, e, "smp_waltmin sync");
    if (status == SMP_OK) status = read_device_error(c);
    return status;
}

// ---------------------------------------------------------------------------------------------------------------
// Baseline SVD(A~^T B~) (Section 4, the comparison with the SVD of the sketched product): block power iteration on
// M = A~^T B~ through its factors, the n1 x n2 product never formed (the footnote there)
// ---------------------------------------------------------------------------------------------------------------
constexpr int SK_ROWS = 256;   // rows of X per CTA of the reduction X^T Y
constexpr int SK_BMAX = 64;    // block columns

// part[blk][a][c] = sum over the rows i of CTA row block blk of X[i][a] Y[i][c] (a < k, c < b <= 64). CTA (32
// sketch rows a, one row block); thread (a = tid % 32, group of 8 columns c = tid / 32); X and Y staged 32 rows at
// a time.
template <typename TS, typename TY>
__global__ void __launch_bounds__(256) xty_partial_kernel(const TS* __restrict__ X, int64_t ldx, int k,
                                                          const TY* __restrict__ Y, int64_t n, int b, TY* part) {
    __shared__ TY xs[32][33];
    __shared__ TY ys[32][SK_BMAX + 1];
    const int tid = threadIdx.x, al = tid & 31, cg = tid >> 5;
    const int a0 = blockIdx.x * 32;
    const int64_t i0 = (int64_t)blockIdx.y * SK_ROWS, i1 = min(n, i0 + SK_ROWS);
    TY acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = TY(0);
    for (int64_t ib = i0; ib < i1; ib += 32) {
        __syncthreads();
        for (int e = tid; e < 32 * 32; e += 256) {
            const int rr = e >> 5, aa = e & 31;
            const int64_t i = ib + rr;
            xs[rr][aa] = (i < i1 && a0 + aa < k) ? (TY)X[i * ldx + a0 + aa] : TY(0);
        }
        for (int e = tid; e < 32 * SK_BMAX; e += 256) {
            const int rr = e / SK_BMAX, cc = e % SK_BMAX;
            const int64_t i = ib + rr;
            ys[rr][cc] = (i < i1 && cc < b) ? Y[i * b + cc] : TY(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
            const TY x = xs[rr][al];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = fma(x, ys[rr][cg * 8 + q], acc[q]);
        }
    }
    const int a = a0 + al;
    if (a >= k) return;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (cg * 8 + q < b) part[((int64_t)blockIdx.y * k + a) * b + cg * 8 + q] = acc[q];
}

// W[e] = sum over blk of part[blk][e] (fixed order, binary64), e < len.
template <typename TY>
__global__ void part_sum_kernel(const TY* __restrict__ part, int nblk, int64_t len, TY* W) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= len) return;
    double s = 0.0;
    for (int q = 0; q < nblk; ++q) s += (double)part[q * len + e];
    W[e] = (TY)s;
}

// Out[j][c] = sum over a < k of X[j][a] W[a][c] (j < n, c < b <= 64). CTA of 32 rows j; thread (j = tid % 32,
// group of 8 columns); X and W staged 32 sketch rows at a time.
template <typename TS, typename TY>
__global__ void __launch_bounds__(256) xw_kernel(const TS* __restrict__ X, int64_t ldx, int k,
                                                 const TY* __restrict__ W, int64_t n, int b, TY* Out) {
    __shared__ TY xs[32][33];
    __shared__ TY ws[32][SK_BMAX + 1];
    const int tid = threadIdx.x, jl = tid & 31, cg = tid >> 5;
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    TY acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = TY(0);
    for (int ab = 0; ab < k; ab += 32) {
        __syncthreads();
        for (int e = tid; e < 32 * 32; e += 256) {
            const int rr = e >> 5, aa = e & 31;
            const int64_t j = j0 + rr;
            xs[rr][aa] = (j < n && ab + aa < k) ? (TY)X[j * ldx + ab + aa] : TY(0);
        }
        for (int e = tid; e < 32 * SK_BMAX; e += 256) {
            const int aa = e / SK_BMAX, cc = e % SK_BMAX;
            ws[aa][cc] = (ab + aa < k && cc < b) ? W[(int64_t)(ab + aa) * b + cc] : TY(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int aa = 0; aa < 32; ++aa) {
            const TY x = xs[jl][aa];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = fma(x, ws[aa][cg * 8 + q], acc[q]);
        }
    }
    const int64_t j = j0 + jl;
    if (j >= n) return;
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (cg * 8 + q < b) Out[j * b + cg * 8 + q] = acc[q];
}

// V[i][c] /= sigma_c with sigma_c = sqrt(lambda_c) (a zero or negative lambda leaves a zero column); S = sigma.
__global__ void ritz_scale_kernel(double* V, int64_t n2, int r, const double* __restrict__ ev, double* S) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < r) S[e] = sqrt(fmax(ev[e], 0.0));
    if (e >= n2 * r) return;
    const int c = (int)(e % r);
    const double sg = sqrt(fmax(ev[c], 0.0));
    V[e] = sg > 0.0 ? V[e] / sg : 0.0;
}

template <typename TS, typename TY>
struct SketchOp {
    const TS* At;   // n1 x ldk: row i = A~ column i
    const TS* Bt;   // n2 x ldk
    int64_t n1, n2, ldk;
    int k, b;
    TY* W;          // k x b
    TY* part;       // row blocks x k x b
    cudaStream_t st;

    void xty(const TS* X, const TY* Y, int64_t n) const {
        const int nblk = (int)std::max<int64_t>(1, (n + SK_ROWS - 1) / SK_ROWS);
        xty_partial_kernel<TS, TY><<<smp::counted(dim3((unsigned)((k + 31) / 32), (unsigned)nblk)), 256, 0, st>>>(
            X, ldk, k, Y, n, b, part);
        part_sum_kernel<TY><<<smp::counted(nblocks((int64_t)k * b, 256)), 256, 0, st>>>(part, nblk, (int64_t)k * b,
                                                                                      W);
    }
    void xw(const TS* X, int64_t n, TY* Out) const {
        xw_kernel<TS, TY><<<smp::counted(nblocks(n, 32)), 256, 0, st>>>(X, ldk, k, W, n, b, Out);
    }
    void apply(const TY* Z, TY* Y) const {   // Y (n1 x b) = A~^T (B~ Z)
        xty(Bt, Z, n2);
        xw(At, n1, Y);
    }
    void apply_t(const TY* Y, TY* Z) const {   // Z (n2 x b) = B~^T (A~ Y)
        xty(At, Y, n1);
        xw(Bt, n2, Z);
    }
};

template <typename TS, typename TY>
smp_status sketch_svd_typed(smp_ctx* c, int r, uint64_t seed, double* U, double* S, double* V) {
    const int64_t n1 = c->p.n1, n2 = c->p.n2, nmax = std::max(n1, n2);
    const int k = c->p.k;
    cudaStream_t st = c->stream;
    const int b = (int)std::min<int64_t>(std::min<int64_t>(2 * r + 8, SK_BMAX), std::min<int64_t>(std::min(n1, n2), k));
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const int64_t skblk = std::max<int64_t>(1, (nmax + SK_ROWS - 1) / SK_ROWS);
    const int64_t gblk = std::max<int64_t>(1, (nmax + GRAM_ROWS_PER_BLOCK - 1) / GRAM_ROWS_PER_BLOCK);
    size_t need = 0;
    auto add = [&](int64_t n, size_t sz) { need += ((size_t)std::max<int64_t>(n, 1) * sz + 511) & ~size_t(255); };
    add(n1 * b, sizeof(TY));                          // Y
    add(n2 * b, sizeof(TY));                          // Z
    add((int64_t)k * b, sizeof(TY));                  // W
    add(skblk * k * b, sizeof(TY));                   // reduction partials
    add(gblk * MAX_SMALL * MAX_SMALL, 8);             // Gram partials
    add(4 * b * b + 4 * b, 8);                        // G, R1, R2, E, eigenvalues
    add(2 * n1 * r + r * r, 8);                       // Ritz vectors now and at the previous check, their Gram
    void* ws = nullptr;
    if (dev_malloc(&ws, need, st) != cudaSuccess) return fail(c, SMP_ENOMEM, "smp_sketch_svd: scratch");
    Arena ar{(char*)ws, 0, need};
    TY* Y = ar.take<TY>(n1 * b);
    TY* Z = ar.take<TY>(n2 * b);
    SketchOp<TS, TY> op;
    op.At = (const TS*)c->sk;
    op.Bt = c->p.same_ab ? op.At : op.At + n1 * c->ldk;
    op.n1 = n1;
    op.n2 = n2;
    op.ldk = c->ldk;
    op.k = k;
    op.b = b;
    op.st = st;
    op.W = ar.take<TY>((int64_t)k * b);
    op.part = ar.take<TY>(skblk * k * b);
    double* gpart = ar.take<double>(gblk * MAX_SMALL * MAX_SMALL);
    double* G = ar.take<double>(b * b);
    double* R1 = ar.take<double>(b * b);
    double* R2 = ar.take<double>(b * b);
    double* E = ar.take<double>(b * b);
    double* ev = ar.take<double>(4 * b);
    double* U0p = ar.take<double>(n1 * r);
    double* Gx = ar.take<double>(r * r);
    jacobi_smem_attr();

    // Philox start block on the right (TAG_INIT), orthonormalised
    start_block_kernel<TY><<<smp::counted(nblocks(n2 * ((b + 3) / 4), 256)), 256, 0, st>>>(n2, b, k0, k1, Z);
    cholqr2<TY, TY, TY>(Z, n2, b, Z, gpart, G, R1, R2, nullptr, st);
    // Each iteration: Y = M Z, orthonormalise Y, Z = M^T Y. Every `every` iterations the top-r Ritz pairs are
    // compared with those of the previous check (E: eigenvectors of Z^T Z, binary64 Jacobi; vectors Y E_r): the
    // iteration stops once the vectors move by less than tol (sqrt(r - ||U^T Uprev||_F^2)) or the values
    // lambda_1..r change by less than vtol lambda_1 (the values converge at twice the rate of the vectors and do
    // not see rotations inside a cluster of nearly equal singular values, which leave the rank-r error unchanged).
    const bool dbl = sizeof(TY) == 8;
    const int max_iter = dbl ? 400 : 200, every = dbl ? 4 : 2;
    const double tol = dbl ? 1e-11 : 2e-5, vtol = dbl ? 1e-14 : 2e-7;
    std::vector<double> ev_prev(r, 0.0), ev_cur(r, 0.0);
    smp_status status = SMP_OK;
    bool have_prev = false;
    for (int it = 1; it <= max_iter; ++it) {
        const bool check = it % every == 0 || it == max_iter;
        op.apply(Z, Y);
        if (check) {
            cholqr2<TY, TY, TY>(Y, n1, b, Y, gpart, G, R1, R2, nullptr, st);
        } else {
            gram_chol<TY>(Y, n1, b, gpart, G, R1, st);
            apply_rinv<TY, TY, TY>(Y, n1, b, R1, Y, st);
        }
        op.apply_t(Y, Z);
        if (check) {
            gram<TY, TY>(Z, Z, n2, b, b, gpart, G, st);
            launch_jacobi<double>(G, b, 4e-15, 40, ev, E, st);
            ritz_kernel<TY><<<smp::counted(nblocks(n1 * r, 256)), 256, 0, st>>>(Y, E, n1, b, r, U);
            bool done = false;
            if (have_prev) {
                gram<double, double>(U, U0p, n1, r, r, gpart, Gx, st);
            }
            std::vector<double> hx(r * r);
            cudaError_t e1 = cudaMemcpyAsync(ev_cur.data(), ev, sizeof(double) * r, cudaMemcpyDeviceToHost, st);
            if (e1 == cudaSuccess && have_prev)
                e1 = cudaMemcpyAsync(hx.data(), Gx, sizeof(double) * r * r, cudaMemcpyDeviceToHost, st);
            if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(st);
            if (e1 != cudaSuccess) {
                status = check_cuda(c, e1, "smp_sketch_svd check");
                break;
            }
            if (have_prev) {
                double fro = 0.0, dv = 0.0;
                for (double v : hx) fro += v * v;
                for (int i = 0; i < r; ++i) dv = std::max(dv, std::fabs(ev_cur[i] - ev_prev[i]));
                done = std::sqrt(std::max(0.0, (double)r - fro)) < tol || dv < vtol * std::fabs(ev_cur[0]);
            }
            ev_prev = ev_cur;
            have_prev = true;
            if (done || it == max_iter) {
                // M ~ Y Y^T M = Y Z^T = (Y E)(Z E)^T, and Z E has orthogonal columns of norms sqrt(lambda)
                ritz_kernel<TY><<<smp::counted(nblocks(n2 * r, 256)), 256, 0, st>>>(Z, E, n2, b, r, V);
                ritz_scale_kernel<<<smp::counted(nblocks(std::max<int64_t>(n2 * r, r), 256)), 256, 0, st>>>(
                    V, n2, r, ev, S);
                sign_kernel<<<smp::counted(r), 256, 0, st>>>(U, n1, V, n2, r);
                break;
            }
            cudaMemcpyAsync(U0p, U, sizeof(double) * n1 * r, cudaMemcpyDeviceToDevice, st);
        }
        gram_chol<TY>(Z, n2, b, gpart, G, R1, st);
        apply_rinv<TY, TY, TY>(Z, n2, b, R1, Z, st);
    }
    cudaError_t e = cudaGetLastError();
    if (status == SMP_OK && e != cudaSuccess) status = check_cuda(c, e, "smp_sketch_svd kernels");
    e = cudaStreamSynchronize(st);
    free_after(ws, st);
    if (status == SMP_OK && e != cudaSuccess) status = check_cuda(c, e, "smp_sketch_svd sync");
    if (status == SMP_OK) status = read_device_error(c);
    return status;
}

}  // namespace

smp_status run_sketch_svd(smp_ctx* c, int r, uint64_t seed, double* U, double* S, double* V) {
    if (c->acc_bytes == 8) return sketch_svd_typed<double, double>(c, r, seed, U, S, V);
    return sketch_svd_typed<float, float>(c, r, seed, U, S, V);
}

smp_status run_waltmin(smp_ctx* c, const void* vals, int r, int T, uint32_t flags, uint64_t seed,
                       const double* U_init, double* U, double* S, double* V) {
    if (c->acc_bytes == 8 || (flags & SMP_FP64_ALS)) {
        if (c->acc_bytes == 8)
            return waltmin_typed<double, double, double, double>(c, (const double*)vals, r, T, flags, seed, U_init,
                                                                 U, S, V);
        return waltmin_typed<float, double, double, double>(c, (const float*)vals, r, T, flags, seed, U_init, U, S,
                                                            V);
    }
    return waltmin_typed<float, float, float, float>(c, (const float*)vals, r, T, flags, seed, U_init, U, S, V);
}

}  // namespace smp
