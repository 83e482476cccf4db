// Small dense kernels used by WAltMin's initial SVD and the canonical form: tall-skinny Gram matrices with a
// fixed-order reduction, Cholesky of a b x b Gram (one warp), right-multiplication by R^-1, and a parallel-order
// (round-robin pairing) cyclic Jacobi eigensolver for symmetric matrices of order <= 72.
//
// Binary64 divide and square root are long-latency instruction sequences on this part (hundreds of cycles), so
// the binary64 code paths use rsqrt_refined (binary32 estimate + Newton-Raphson) and multiply by reciprocals.
#pragma once
#include "common.cuh"
#include "internal.h"

namespace smp {

constexpr int GRAM_ROWS_PER_BLOCK = 16;
constexpr int MAX_SMALL = 72;   // largest order of the small dense problems (block size 2r + 8, r <= 32)

// part[blk][p][q] = sum over this block's rows of X[i][p] * Y[i][q] (X: n x a, Y: n x b, row-major, ld = a / b).
template <typename TX, typename TY>
__global__ void __launch_bounds__(256) gram_partial_kernel(const TX* __restrict__ X, const TY* __restrict__ Y,
                                                           int64_t n, int a, int b, double* part) {
    __shared__ double xs[GRAM_ROWS_PER_BLOCK][MAX_SMALL + 1];
    __shared__ double ys[GRAM_ROWS_PER_BLOCK][MAX_SMALL + 1];
    const int64_t r0 = (int64_t)blockIdx.x * GRAM_ROWS_PER_BLOCK;
    const int64_t r1 = min(n, r0 + GRAM_ROWS_PER_BLOCK);
    const int rows = (int)(r1 - r0);
    for (int e = threadIdx.x; e < GRAM_ROWS_PER_BLOCK * a; e += blockDim.x) {
        const int rr = e / a, cc = e - rr * a;
        xs[rr][cc] = rr < rows ? (double)X[(r0 + rr) * a + cc] : 0.0;
    }
    for (int e = threadIdx.x; e < GRAM_ROWS_PER_BLOCK * b; e += blockDim.x) {
        const int rr = e / b, cc = e - rr * b;
        ys[rr][cc] = rr < rows ? (double)Y[(r0 + rr) * b + cc] : 0.0;
    }
    __syncthreads();
    const int npair = a * b;
    for (int pq = threadIdx.x; pq < npair; pq += blockDim.x) {
        const int p = pq / b, q = pq - p * b;
        double s = 0.0;
        for (int rr = 0; rr < rows; ++rr) s = fma(xs[rr][p], ys[rr][q], s);
        part[(int64_t)blockIdx.x * npair + pq] = s;
    }
}

// G[pq] = sum over blocks of part[blk][pq]: one warp per entry, lane-strided partial sums then a fixed shuffle
// tree (deterministic).
__global__ void gram_reduce_kernel(const double* __restrict__ part, int nblk, int npair, double* G) {
    const int pq = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (pq >= npair) return;
    double s = 0.0;
    for (int k = lane; k < nblk; k += 32) s += part[(int64_t)k * npair + pq];
    s = warp_sum(s);
    if (lane == 0) G[pq] = s;
}

// Upper Cholesky factor R (G = R^T R, R row-major b x b) of a b x b symmetric matrix, 32 < b <= MAX_SMALL. A pivot
// <= tol * max diag marks a rank-deficient direction: that row of R is zeroed (apply_rinv then zeroes the column).
// Four warps: one thread takes each pivot; the column scaling and the trailing update's (i, k) pairs are spread over
// all 128 threads, so the binary64 work lands on the SM's four sub-partitions (one warp alone: 0.15 ms at b = 48).
__global__ void __launch_bounds__(128) chol_par_kernel(const double* __restrict__ G, int b, double* R, double tol) {
    __shared__ double L[MAX_SMALL][MAX_SMALL + 1];
    __shared__ double rinv_j, maxd_s;
    const int tid = threadIdx.x;
    for (int e = tid; e < b * b; e += 128) {
        const int i = e / b, j = e - i * b;
        L[i][j] = G[e];
    }
    __syncthreads();
    if (tid < 32) {
        double maxd = 0.0;
        for (int i = tid; i < b; i += 32) maxd = fmax(maxd, L[i][i]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) maxd = fmax(maxd, __shfl_xor_sync(0xffffffffu, maxd, o));
        if (tid == 0) maxd_s = maxd;
    }
    __syncthreads();
    const double maxd = maxd_s;
    for (int j = 0; j < b; ++j) {
        if (tid == 0) {
            const double d = L[j][j];
            const bool ok = d > tol * maxd && d > 0.0;
            const double y = ok ? rsqrt_refined(d) : 0.0;
            L[j][j] = ok ? d * y : 0.0;
            rinv_j = y;
        }
        __syncthreads();
        const double y = rinv_j;
        for (int i = j + 1 + tid; i < b; i += 128) L[i][j] *= y;
        __syncthreads();
        // pairs (i, k), j < k <= i < b, numbered p = a (a + 1) / 2 + c with i = j + 1 + a, k = j + 1 + c
        const int m = b - j - 1;
        const int np = m * (m + 1) / 2;
        for (int p = tid; p < np; p += 128) {
            int a = (int)((sqrtf(8.f * (float)p + 1.f) - 1.f) * 0.5f);
            if ((a + 1) * (a + 2) / 2 <= p) ++a;
            if (a * (a + 1) / 2 > p) --a;
            const int i = j + 1 + a, k = j + 1 + (p - a * (a + 1) / 2);
            L[i][k] = fma(-L[i][j], L[k][j], L[i][k]);
        }
        __syncthreads();
    }
    for (int e = tid; e < b * b; e += 128) {
        const int i = e / b, j = e - i * b;
        R[e] = j >= i ? L[j][i] : 0.0;
    }
}

// Upper Cholesky factor of a b x b symmetric matrix (b <= 32), same pivot rule and output as chol_par_kernel, on four
// warps: every warp keeps the whole matrix in registers (lane i holds row i), computes each pivot and its column
// (in parallel, identically), and updates only the trailing columns kk with kk % 4 == its warp id, so the binary64
// work of the trailing updates is spread over the SM's four sub-partitions (on this part each issues about one
// binary64 warp instruction per 64 cycles). Each warp runs its own compile-time list of columns (chol32_update<W>):
// with one shared loop and a runtime warp test the compiler predicates the updates, and the predicated-off binary64
// instructions still take their issue slots. Column j + 1 is then broadcast from the warp that updated it through
// shared memory. Launch with 128 threads.
template <int W>
__device__ __forceinline__ void chol32_update(double (&a)[32], int j, int b, int lane, double lij) {
#pragma unroll
    for (int kk = W; kk < 32; kk += 4) {
        if (kk <= j) continue;   // resolved at compile time once j is (the caller's loop is unrolled)
        if (kk >= b) break;
        const double lkj = __shfl_sync(0xffffffffu, lij, kk);   // L[kk][j]
        if (lane > j) a[kk] = fma(-lij, lkj, a[kk]);
    }
}

__global__ void __launch_bounds__(128) chol32_kernel(const double* __restrict__ G, int b, double* R, double tol) {
    __shared__ double col[2][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double a[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) a[k] = (lane < b && k < b) ? G[lane * b + k] : 0.0;
    double maxd = 0.0;
#pragma unroll
    for (int k = 0; k < 32; ++k)
        if (k == lane && lane < b) maxd = a[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxd = fmax(maxd, __shfl_xor_sync(0xffffffffu, maxd, o));
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        if (j < b) {
            const double d = __shfl_sync(0xffffffffu, a[j], j);
            const bool ok = d > tol * maxd && d > 0.0;
            const double y = ok ? rsqrt_refined(d) : 0.0;
            const double lij = lane == j ? (ok ? d * y : 0.0) : (lane > j ? a[j] * y : 0.0);
            if (lane >= j) a[j] = lij;
            switch (w) {   // warp-uniform
                case 0: chol32_update<0>(a, j, b, lane, lij); break;
                case 1: chol32_update<1>(a, j, b, lane, lij); break;
                case 2: chol32_update<2>(a, j, b, lane, lij); break;
                default: chol32_update<3>(a, j, b, lane, lij); break;
            }
            if (j + 1 < b) {   // broadcast the next pivot column from the warp that updated it
                if (((j + 1) & 3) == w) col[(j + 1) & 1][lane] = a[j + 1];
                __syncthreads();
                a[j + 1] = col[(j + 1) & 1][lane];
            }
        }
    }
    if (w == 0 && lane < b) {
#pragma unroll
        for (int k = 0; k < 32; ++k)
            if (k < b) R[k * b + lane] = k <= lane ? a[k] : 0.0;   // R = L^T
    }
}

// Xout[i] = Xin[i] R^-1 (row vector times the inverse of the upper factor R, b x b row-major, b <= NB), the
// substitution carried out in TC (binary32 for the subspace iteration's first Cholesky-QR pass, whose second pass
// restores orthogonality; binary64 for the canonical form), one thread per row with the row in registers: the substitution's loops are fully
// unrolled (every index of x is a compile-time constant, so x stays in registers instead of local memory; a run-time
// index sent it to local memory: 55 us at n = 1,504, b = 48); b only enters warp-uniform guards. R^-1's
// diagonal comes from rsqrt_refined(d^2), zero where R's diagonal is zero (a rank-deficient direction). Instantiated
// for b <= 32, 48 and 72; the work is that of NB.
template <typename TIn, typename TOut, typename TC, int NB>
__global__ void __launch_bounds__(128) apply_rinv_kernel(const TIn* __restrict__ Xin, int64_t n, int b,
                                                         const double* __restrict__ R, TOut* Xout) {
    // R padded to NB x NB with zeros (and a zero inverse diagonal) beyond b, so the substitution needs no guards
    __shared__ TC Rs[NB * NB];
    __shared__ TC dinv[NB];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int l = e / NB, j = e - l * NB;
        Rs[e] = (l < b && j < b) ? (TC)R[l * b + j] : TC(0);
    }
    for (int j = threadIdx.x; j < NB; j += blockDim.x) {
        const double d = j < b ? R[j * b + j] : 0.0;
        dinv[j] = d > 0.0 ? (TC)rsqrt_refined(d * d) : TC(0);
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const TIn* xin = Xin + i * b;
    TC x[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        TC y = j < b ? (TC)xin[j] : TC(0);
#pragma unroll
        for (int l = 0; l < j; ++l) y -= x[l] * Rs[l * NB + j];
        x[j] = y * dinv[j];
    }
#pragma unroll
    for (int j = 0; j < NB; ++j)
        if (j < b) Xout[i * b + j] = (TOut)x[j];
}

// Rotation (c, s) in the (p, q) plane that zeroes A_pq: theta = (A_qq - A_pp) / (2 A_pq),
// t = sign(theta) / (|theta| + sqrt(theta^2 + 1)), c = 1 / sqrt(1 + t^2), s = t c. The binary64 version takes t
// from binary32 arithmetic (the angle only steers convergence) and c from rsqrt_refined, so c^2 + s^2 = 1 to
// binary64 rounding and the accumulated V stays orthogonal.
__device__ __forceinline__ void jacobi_rotation(float app, float aqq, float apq, float& c, float& s) {
    const float th = (aqq - app) / (2.0f * apq);
    float t = 0.0f;
    if (isfinite(th)) t = (th >= 0.0f ? 1.0f : -1.0f) / (fabsf(th) + sqrtf(fmaf(th, th, 1.0f)));
    c = rsqrtf(fmaf(t, t, 1.0f));
    s = t * c;
}
__device__ __forceinline__ void jacobi_rotation(double app, double aqq, double apq, double& c, double& s) {
    const float thf = (float)(aqq - app) / (2.0f * (float)apq);
    float tf = 0.0f;
    if (isfinite(thf)) tf = (thf >= 0.0f ? 1.0f : -1.0f) / (fabsf(thf) + sqrtf(fmaf(thf, thf, 1.0f)));
    const double t = (double)tf;
    c = rsqrt_refined(fma(t, t, 1.0));
    s = t * c;
}

// Symmetric eigen decomposition A = V diag(lambda) V^T (n <= MAX_SMALL) in precision T by cyclic Jacobi with
// round-robin pairing (n/2 disjoint rotations per step, all applied in parallel). A pair (p, q) is rotated only when
// |A_pq| > tol (|A_pp| + |A_qq|) and |A_pq| > 8 eps_T ||A||_F (the negligibility test of the cyclic Jacobi method;
// below it a rotation only stirs rounding noise); the method stops after a sweep that rotates no pair, or after
// max_sweeps. tol must exceed a few eps_T. Output (binary64): eigenvalues in decreasing order and V's columns
// permuted to match. One CTA of 256 threads, dynamic shared memory 2 n (n + 1) sizeof(T).
template <typename T>
__global__ void __launch_bounds__(256) jacobi_eig_kernel(const double* __restrict__ Ain, int n, double tol,
                                                         int max_sweeps, double* evals, double* Vout) {
    extern __shared__ __align__(16) unsigned char jsm[];
    T* A = (T*)jsm;                  // n x (n+1)
    T* V = A + n * (n + 1);          // n x (n+1)
    __shared__ int rp[MAX_SMALL / 2 + 1], rq[MAX_SMALL / 2 + 1];
    __shared__ T rc[MAX_SMALL / 2 + 1], rs[MAX_SMALL / 2 + 1];
    __shared__ double red[8];
    __shared__ double floor_abs;
    __shared__ int rotated[3];       // per sweep (mod 3): did any pair rotate
    __shared__ int order[MAX_SMALL];
    const int ld = n + 1;
    double fro = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        const double v = Ain[e];
        A[i * ld + j] = (T)v;
        V[i * ld + j] = i == j ? T(1) : T(0);
        fro += v * v;
    }
    fro = warp_sum(fro);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = fro;
    if (threadIdx.x < 3) rotated[threadIdx.x] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        double f = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) f += red[w];
        const double eps = sizeof(T) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
        floor_abs = 8.0 * eps * sqrt(f);
    }
    __syncthreads();
    const T tol_t = (T)tol, floor_t = (T)floor_abs;
    const int m = n + (n & 1);
    const int npairs = m / 2;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) rotated[(sweep + 1) % 3] = 0;   // the flag the next sweep sets; nobody reads it now
        for (int s = 0; s < m - 1; ++s) {
            if (threadIdx.x < npairs) {
                const int k = threadIdx.x;
                const int x0 = k, x1 = m - 1 - k;
                int p = x0 == 0 ? 0 : 1 + (x0 - 1 + s) % (m - 1);
                int q = x1 == 0 ? 0 : 1 + (x1 - 1 + s) % (m - 1);
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                T c = T(1), sn = T(0);
                bool rot = false;
                if (q < n) {
                    const T apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
                    const T aa = apq < T(0) ? -apq : apq;
                    const T dd = (app < T(0) ? -app : app) + (aqq < T(0) ? -aqq : aqq);
                    if (aa > floor_t && aa > tol_t * dd) {
                        jacobi_rotation(app, aqq, apq, c, sn);
                        rot = sn != T(0);   // an angle outside binary32 range comes back as the identity
                        if (rot) rotated[sweep % 3] = 1;
                    }
                }
                if (!rot) q = p;   // no rotation (dummy player or negligible entry)
                rp[k] = p;
                rq[k] = q;
                rc[k] = c;
                rs[k] = sn;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < npairs * n; e += blockDim.x) {   // columns of A and V
                const int k = e / n, i = e - k * n;
                const int p = rp[k], q = rq[k];
                if (p == q) continue;
                const T c = rc[k], sn = rs[k];
                const T ap = A[i * ld + p], aq = A[i * ld + q];
                A[i * ld + p] = c * ap - sn * aq;
                A[i * ld + q] = sn * ap + c * aq;
                const T vp = V[i * ld + p], vq = V[i * ld + q];
                V[i * ld + p] = c * vp - sn * vq;
                V[i * ld + q] = sn * vp + c * vq;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < npairs * n; e += blockDim.x) {   // rows of A
                const int k = e / n, i = e - k * n;
                const int p = rp[k], q = rq[k];
                if (p == q) continue;
                const T c = rc[k], sn = rs[k];
                const T ap = A[p * ld + i], aq = A[q * ld + i];
                A[p * ld + i] = c * ap - sn * aq;
                A[q * ld + i] = sn * ap + c * aq;
            }
            __syncthreads();
        }
        if (!rotated[sweep % 3]) break;
    }
    if (threadIdx.x < n) {   // stable sort, decreasing
        const int i = threadIdx.x;
        const T li = A[i * ld + i];
        int rank = 0;
        for (int j = 0; j < n; ++j) {
            const T lj = A[j * ld + j];
            rank += (lj > li) || (lj == li && j < i);
        }
        order[rank] = i;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, c = e - i * n;
        Vout[e] = (double)V[i * ld + order[c]];
    }
    if (threadIdx.x < n) evals[threadIdx.x] = (double)A[order[threadIdx.x] * ld + order[threadIdx.x]];
}

// Symmetric eigen decomposition (jacobi_eig_kernel semantics). The 256-thread CTA keeps the four binary64 pipes of
// the SM busy; a one-warp variant measured 2.3x slower in binary64 on this part.
template <typename T>
inline void launch_jacobi(const double* A, int n, double tol, int max_sweeps, double* evals, double* V,
                          cudaStream_t st) {
    jacobi_eig_kernel<T><<<smp::counted(1), 256, 2 * n * (n + 1) * (int)sizeof(T), st>>>(A, n, tol, max_sweeps,
                                                                                         evals, V);
}

// Singular value decomposition K = W diag(S) Z^T of an r x r matrix (r <= 32) by one-sided (Hestenes) Jacobi in
// binary64: column pairs (p, q) of U (initially K) are rotated until every pair is orthogonal to
// |u_p . u_q| <= tol ||u_p|| ||u_q||; the rotations accumulate in Z; S_j = ||u_j||, W_j = u_j / S_j (a zero
// singular value leaves a zero column of W). Pairs follow the round-robin order, one warp per pair, so each step's
// n/2 rotations run in parallel; the sweep loop stops after a sweep without rotations or after max_sweeps. K is
// scaled by a power of two (exact) so the binary32 angle computation stays in range. Output sorted by decreasing S.
// One CTA of 256 threads.
__global__ void __launch_bounds__(256) svd_onesided_kernel(const double* __restrict__ K, int r, double tol,
                                                           int max_sweeps, double* S, double* W, double* Z) {
    __shared__ double Us[32][33], Vs[32][33];
    __shared__ double sig[32];
    __shared__ double red[8];
    __shared__ int order[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double mx = 0.0;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) mx = fmax(mx, fabs(K[e]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    mx = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    int ex = 0;
    if (mx > 0.0) frexp(mx, &ex);
    const double scale = ldexp(1.0, -ex), unscale = ldexp(1.0, ex);
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int i = e / r, j = e - i * r;
        Us[i][j] = K[e] * scale;
        Vs[i][j] = i == j ? 1.0 : 0.0;
    }
    __syncthreads();
    const int m = r + (r & 1);
    const int npairs = m / 2;
    const double tol2 = tol * tol;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        int any = 0;
        for (int st = 0; st < m - 1; ++st) {
            int my_rot = 0;
            for (int k = warp; k < npairs; k += (int)(blockDim.x >> 5)) {
                const int x0 = k, x1 = m - 1 - k;
                int ip = x0 - 1 + st, iq = x1 - 1 + st;
                if (ip >= m - 1) ip -= m - 1;
                if (iq >= m - 1) iq -= m - 1;
                int p = x0 == 0 ? 0 : 1 + ip;
                int q = x1 == 0 ? 0 : 1 + iq;
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                if (q >= r) continue;
                const double a = lane < r ? Us[lane][p] : 0.0;
                const double b = lane < r ? Us[lane][q] : 0.0;
                const double alpha = warp_sum(a * a), beta = warp_sum(b * b), gamma = warp_sum(a * b);
                if (gamma != 0.0 && gamma * gamma > tol2 * alpha * beta) {
                    double c, sn;
                    jacobi_rotation(alpha, beta, gamma, c, sn);
                    if (sn != 0.0) {
                        if (lane < r) {
                            Us[lane][p] = c * a - sn * b;
                            Us[lane][q] = sn * a + c * b;
                            const double vp = Vs[lane][p], vq = Vs[lane][q];
                            Vs[lane][p] = c * vp - sn * vq;
                            Vs[lane][q] = sn * vp + c * vq;
                        }
                        my_rot = 1;
                    }
                }
            }
            any |= __syncthreads_or(my_rot);
        }
        if (!any) break;
    }
    for (int j = warp; j < r; j += (int)(blockDim.x >> 5)) {
        const double a = lane < r ? Us[lane][j] : 0.0;
        const double n2 = warp_sum(a * a);
        if (lane == 0) sig[j] = sqrt(n2);
    }
    __syncthreads();
    if (threadIdx.x < r) {   // stable sort, decreasing
        const int i = threadIdx.x;
        const double si = sig[i];
        int rank = 0;
        for (int j = 0; j < r; ++j) rank += (sig[j] > si) || (sig[j] == si && j < i);
        order[rank] = i;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int i = e / r, cc = e - i * r;
        const int j = order[cc];
        const double sj = sig[j];
        W[e] = sj > 0.0 ? Us[i][j] / sj : 0.0;
        Z[e] = Vs[i][j];
    }
    if (threadIdx.x < r) S[threadIdx.x] = sig[order[threadIdx.x]] * unscale;
}

}  // namespace smp
