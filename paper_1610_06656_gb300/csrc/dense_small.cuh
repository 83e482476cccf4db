// Small dense binary64 kernels used by WAltMin's initial SVD and the canonical form: tall-skinny Gram matrices
// with a fixed-order reduction, Cholesky of a b x b Gram (one warp), right-multiplication by R^-1, and a
// parallel-order (round-robin pairing) cyclic Jacobi eigensolver for symmetric matrices of order <= 72.
#pragma once
#include "common.cuh"

namespace smp {

constexpr int GRAM_ROWS_PER_BLOCK = 256;
constexpr int MAX_SMALL = 72;   // largest order of the small dense problems (block size 2r + 8, r <= 32)
constexpr int GRAM_STAGE = 16;

// part[blk][p][q] = sum over this block's rows of X[i][p] * Y[i][q] (X: n x a, Y: n x b, row-major, ld = a / b).
template <typename TX, typename TY>
__global__ void __launch_bounds__(256) gram_partial_kernel(const TX* __restrict__ X, const TY* __restrict__ Y,
                                                           int64_t n, int a, int b, double* part) {
    __shared__ double xs[GRAM_STAGE][MAX_SMALL + 1];
    __shared__ double ys[GRAM_STAGE][MAX_SMALL + 1];
    const int64_t r0 = (int64_t)blockIdx.x * GRAM_ROWS_PER_BLOCK;
    const int64_t r1 = min(n, r0 + GRAM_ROWS_PER_BLOCK);
    const int npair = a * b;
    double acc[MAX_SMALL * MAX_SMALL / 256 + 1];
    const int nmine = (npair + 255 - threadIdx.x) / 256;
    for (int e = 0; e < nmine; ++e) acc[e] = 0.0;
    for (int64_t base = r0; base < r1; base += GRAM_STAGE) {
        const int rows = (int)(r1 - base < GRAM_STAGE ? r1 - base : GRAM_STAGE);
        for (int e = threadIdx.x; e < GRAM_STAGE * a; e += blockDim.x) {
            const int rr = e / a, cc = e - rr * a;
            xs[rr][cc] = rr < rows ? (double)X[(base + rr) * a + cc] : 0.0;
        }
        for (int e = threadIdx.x; e < GRAM_STAGE * b; e += blockDim.x) {
            const int rr = e / b, cc = e - rr * b;
            ys[rr][cc] = rr < rows ? (double)Y[(base + rr) * b + cc] : 0.0;
        }
        __syncthreads();
        for (int e = 0; e < nmine; ++e) {
            const int pq = threadIdx.x + 256 * e;
            const int p = pq / b, q = pq - p * b;
            double s = acc[e];
            for (int rr = 0; rr < rows; ++rr) s = fma(xs[rr][p], ys[rr][q], s);
            acc[e] = s;
        }
        __syncthreads();
    }
    for (int e = 0; e < nmine; ++e) part[(int64_t)blockIdx.x * npair + threadIdx.x + 256 * e] = acc[e];
}

// G[pq] = sum over blocks (in order) of part[blk][pq].
__global__ void gram_reduce_kernel(const double* __restrict__ part, int nblk, int npair, double* G) {
    const int pq = blockIdx.x * blockDim.x + threadIdx.x;
    if (pq >= npair) return;
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += part[(int64_t)k * npair + pq];
    G[pq] = s;
}

// Upper Cholesky factor R (G = R^T R) of a b x b symmetric matrix by one warp. A pivot <= tol * max diag marks a
// rank-deficient direction: that row of R is zeroed (apply_rinv then zeroes the column) and the flag is counted.
__global__ void chol_kernel(const double* __restrict__ G, int b, double* R, double tol, int* ndropped) {
    __shared__ double L[MAX_SMALL][MAX_SMALL + 1];
    __shared__ double dj;
    const int lane = threadIdx.x;
    double maxd = 0.0;
    for (int e = lane; e < b * b; e += 32) {
        const int i = e / b, j = e - i * b;
        L[i][j] = G[e];
        if (i == j) maxd = fmax(maxd, G[e]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxd = fmax(maxd, __shfl_xor_sync(0xffffffffu, maxd, o));
    __syncwarp();
    int dropped = 0;
    for (int j = 0; j < b; ++j) {
        if (lane == 0) {
            const double d = L[j][j];
            dj = (d > tol * maxd && d > 0.0) ? sqrt(d) : 0.0;
            L[j][j] = dj;
        }
        __syncwarp();
        const double d = dj;
        if (d == 0.0) ++dropped;
        for (int i = j + 1 + lane; i < b; i += 32) L[i][j] = d > 0.0 ? L[i][j] / d : 0.0;
        __syncwarp();
        for (int i = j + 1 + lane; i < b; i += 32) {
            const double lij = L[i][j];
            for (int kk = j + 1; kk <= i; ++kk) L[i][kk] -= lij * L[kk][j];
        }
        __syncwarp();
    }
    // R = L^T (upper)
    for (int e = lane; e < b * b; e += 32) {
        const int i = e / b, j = e - i * b;
        R[e] = j >= i ? L[j][i] : 0.0;
    }
    if (lane == 0 && ndropped) *ndropped = dropped;
}

// X_out[i] = X_in[i] R^-1 (row vector times inverse upper factor); a zero pivot zeroes that column.
template <typename TIn, typename TOut>
__global__ void __launch_bounds__(128) apply_rinv_kernel(const TIn* __restrict__ Xin, int64_t n, int b,
                                                         const double* __restrict__ R, TOut* Xout) {
    __shared__ double Rs[MAX_SMALL * MAX_SMALL];
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) Rs[e] = R[e];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[MAX_SMALL];
    for (int j = 0; j < b; ++j) {
        double y = (double)Xin[i * b + j];
        for (int l = 0; l < j; ++l) y -= x[l] * Rs[l * b + j];
        const double d = Rs[j * b + j];
        x[j] = d != 0.0 ? y / d : 0.0;
    }
    for (int j = 0; j < b; ++j) Xout[i * b + j] = (TOut)x[j];
}

// Symmetric eigen decomposition A = V diag(lambda) V^T (n <= MAX_SMALL) by cyclic Jacobi with round-robin pairing
// (n/2 disjoint rotations per step, all applied in parallel). Rotation in the (p, q) plane with
// theta = (A_qq - A_pp) / (2 A_pq), t = sign(theta) / (|theta| + sqrt(theta^2 + 1)), c = 1/sqrt(1 + t^2), s = t c
// zeroes A_pq. Stops when the off-diagonal square sum (summed directly) is <= tol^2 times the diagonal's.
// Output: eigenvalues in decreasing order and V's columns permuted to match. One CTA of 256 threads, dynamic
// shared memory 2 * n * (n + 1) doubles.
__global__ void __launch_bounds__(256) jacobi_eig_kernel(const double* __restrict__ Ain, int n, double tol,
                                                         int max_sweeps, double* evals, double* Vout) {
    extern __shared__ double sm[];
    double* A = sm;                  // n x (n+1)
    double* V = sm + n * (n + 1);    // n x (n+1)
    __shared__ int rp[MAX_SMALL / 2 + 1], rq[MAX_SMALL / 2 + 1];
    __shared__ double rc[MAX_SMALL / 2 + 1], rs[MAX_SMALL / 2 + 1];
    __shared__ double red[8];
    __shared__ int stop;
    __shared__ int order[MAX_SMALL];
    const int ld = n + 1;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e - i * n;
        A[i * ld + j] = Ain[e];
        V[i * ld + j] = i == j ? 1.0 : 0.0;
    }
    __syncthreads();
    const int m = n + (n & 1);
    const int npairs = m / 2;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = e / n, j = e - i * n;
            const double v = A[i * ld + j];
            if (i == j) dia += v * v;
            else off += v * v;
        }
        off = warp_sum(off);
        dia = warp_sum(dia);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = off;
        __syncthreads();
        if (threadIdx.x == 0) {
            double o = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) o += red[w];
            red[0] = o;
        }
        __syncthreads();
        const double off_total = red[0];
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dia;
        __syncthreads();
        if (threadIdx.x == 0) {
            double d = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) d += red[w];
            stop = off_total <= tol * tol * d;
        }
        __syncthreads();
        if (stop) break;
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
                double c = 1.0, sn = 0.0;
                if (q < n) {
                    const double apq = A[p * ld + q];
                    if (apq != 0.0) {
                        const double th = (A[q * ld + q] - A[p * ld + p]) / (2.0 * apq);
                        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        sn = t * c;
                    }
                } else {
                    q = p;   // dummy player: no rotation
                }
                rp[k] = p;
                rq[k] = q;
                rc[k] = c;
                rs[k] = sn;
            }
            __syncthreads();
            // columns of A and V
            for (int e = threadIdx.x; e < npairs * n; e += blockDim.x) {
                const int k = e / n, i = e - k * n;
                const int p = rp[k], q = rq[k];
                if (p == q) continue;
                const double c = rc[k], sn = rs[k];
                const double ap = A[i * ld + p], aq = A[i * ld + q];
                A[i * ld + p] = c * ap - sn * aq;
                A[i * ld + q] = sn * ap + c * aq;
                const double vp = V[i * ld + p], vq = V[i * ld + q];
                V[i * ld + p] = c * vp - sn * vq;
                V[i * ld + q] = sn * vp + c * vq;
            }
            __syncthreads();
            // rows of A
            for (int e = threadIdx.x; e < npairs * n; e += blockDim.x) {
                const int k = e / n, i = e - k * n;
                const int p = rp[k], q = rq[k];
                if (p == q) continue;
                const double c = rc[k], sn = rs[k];
                const double ap = A[p * ld + i], aq = A[q * ld + i];
                A[p * ld + i] = c * ap - sn * aq;
                A[q * ld + i] = sn * ap + c * aq;
            }
            __syncthreads();
        }
    }
    // sort eigenvalues decreasing (stable: ties keep the lower index first)
    if (threadIdx.x < n) {
        const int i = threadIdx.x;
        const double li = A[i * ld + i];
        int rank = 0;
        for (int j = 0; j < n; ++j) {
            const double lj = A[j * ld + j];
            rank += (lj > li) || (lj == li && j < i);
        }
        order[rank] = i;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, c = e - i * n;
        Vout[e] = V[i * ld + order[c]];
    }
    if (threadIdx.x < n) evals[threadIdx.x] = A[order[threadIdx.x] * ld + order[threadIdx.x]];
}

}  // namespace smp
