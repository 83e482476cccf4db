// WAltMin (Algorithm 2, Appendix A) and the canonical form of its output.
//
//  * weights w = 1/q^ (step 2); optional split of Omega into 2T+1 subsets by the split coin (step 3);
//  * U0: top-r left singular subspace of R_Omega0(M~) = w .* P_Omega0(M~) (steps 4-5) by block subspace iteration
//    with b = min(2r + 8, n1, n2) columns: Y <- orth(R (R^T Y)) with CSR / CSC sparse products and a Cholesky-QR
//    (twice) in binary64, then a Rayleigh-Ritz step on Z = R^T Y; trim (step 6);
//  * T rounds of the two weighted least-squares half-steps (steps 8 and 9): one warp per output row builds
//    G = sum w f f^T and b = sum w M~ f with warp shuffles, adds the ridge 1e-10 tr(G)/r, and solves by a binary64
//    Cholesky held in shared memory;
//  * canonical form: Cholesky-QR (twice) of U^ and V^, the SVD of the r x r core Ru Rv^T via the symmetric
//    eigenproblem of [[0, K], [K^T, 0]], and the sign rule (largest-magnitude entry of each U column positive).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "dense_small.cuh"
#include "internal.h"

namespace smp {
namespace {

constexpr int LS_WARPS = 4;

// ---------------------------------------------------------------------------------------------------------------
// weights, split, values of R_Omega(M~)
// ---------------------------------------------------------------------------------------------------------------
__global__ void erow_kernel(const int64_t* __restrict__ row_ptr, int64_t n1, int32_t* erow) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n1) return;
    for (int64_t p = row_ptr[warp] + lane; p < row_ptr[warp + 1]; p += 32) erow[p] = (int32_t)warp;
}

__global__ void split_kernel(const int32_t* __restrict__ erow, const int32_t* __restrict__ col, int64_t nnz, int T,
                             uint32_t k0, uint32_t k1, uint8_t* sub) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const double u = coin((uint32_t)erow[e], (uint32_t)col[e], TAG_SPLIT, k0, k1);
    const double f = floor(__dmul_rn(u, (double)(2 * T + 1)));
    sub[e] = (uint8_t)min((int)f, 2 * T);
}

template <typename TV, typename TR>
__global__ void rvals_kernel(const TV* __restrict__ vals, const double* __restrict__ qhat,
                             const uint8_t* __restrict__ sub, int sid, int64_t nnz, TR* rv) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const double q = qhat[e];
    const double w = q > 0.0 ? 1.0 / q : 0.0;
    const bool in = sub == nullptr || sub[e] == sid;
    rv[e] = in ? (TR)(w * (double)vals[e]) : TR(0);
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

// Y[i] = sum over row i of rv * Z[col]   (warp per row, lanes over the b columns)
template <typename TY>
__global__ void spmm_csr_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                const TY* __restrict__ rv, const TY* __restrict__ Z, int64_t n1, int b, TY* Y) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n1) return;
    TY acc[3] = {TY(0), TY(0), TY(0)};
    for (int64_t p = row_ptr[warp]; p < row_ptr[warp + 1]; ++p) {
        const TY v = rv[p];
        const TY* z = Z + (int64_t)col[p] * b;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (lane + 32 * q < b) acc[q] = fma(v, z[lane + 32 * q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
        if (lane + 32 * q < b) Y[warp * b + lane + 32 * q] = acc[q];
}

// Z[j] = sum over column j of rv * Y[row]   (warp per column)
template <typename TY>
__global__ void spmm_csc_kernel(const int64_t* __restrict__ col_ptr, const int32_t* __restrict__ csc_row,
                                const int64_t* __restrict__ csc_pos, const TY* __restrict__ rv,
                                const TY* __restrict__ Y, int64_t n2, int b, TY* Z) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n2) return;
    TY acc[3] = {TY(0), TY(0), TY(0)};
    for (int64_t p = col_ptr[warp]; p < col_ptr[warp + 1]; ++p) {
        const TY v = rv[csc_pos[p]];
        const TY* y = Y + (int64_t)csc_row[p] * b;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (lane + 32 * q < b) acc[q] = fma(v, y[lane + 32 * q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
        if (lane + 32 * q < b) Z[warp * b + lane + 32 * q] = acc[q];
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
// For every output row o: x_o = argmin sum_{e in row o} w_e (F[idx_e] . x - M~_e)^2 over the entries of subset sid
// (all entries when sub is null). ptr/idx walk CSR (pos = null) or CSC (pos maps to CSR positions, where vals,
// qhat and sub live). Lane l holds column l of G; the factor row of each sample is loaded once (lane c -> F[c])
// and broadcast with shuffles.
template <typename TF, typename TG, typename TV, int RMAX>
__global__ void __launch_bounds__(32 * LS_WARPS) ls_kernel(const int64_t* __restrict__ ptr,
                                                           const int32_t* __restrict__ idx,
                                                           const int64_t* __restrict__ pos,
                                                           const TV* __restrict__ vals,
                                                           const double* __restrict__ qhat,
                                                           const uint8_t* __restrict__ sub, int sid,
                                                           const TF* __restrict__ Fin, int r, int64_t n_out,
                                                           TF* Xout, int* err) {
    __shared__ double Gs[LS_WARPS][RMAX][RMAX + 1];
    __shared__ double bs[LS_WARPS][RMAX];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t o = (int64_t)blockIdx.x * LS_WARPS + wid;
    if (o >= n_out) return;
    TG g[RMAX];
#pragma unroll
    for (int a = 0; a < RMAX; ++a) g[a] = TG(0);
    TG bl = TG(0);
    const int64_t p0 = ptr[o], p1 = ptr[o + 1];
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
        for (int s = 0; s < cnt; ++s) {
            const int32_t in_s = __shfl_sync(0xffffffffu, in, s);
            const TG w_s = __shfl_sync(0xffffffffu, wv, s);
            const TG m_s = __shfl_sync(0xffffffffu, mv, s);
            const TG f = lane < r ? (TG)Fin[(int64_t)in_s * r + lane] : TG(0);
            const TG wf = w_s * f;
#pragma unroll
            for (int a = 0; a < RMAX; ++a) g[a] = fma(wf, __shfl_sync(0xffffffffu, f, a), g[a]);
            bl = fma(wf, m_s, bl);
        }
    }
    // G (column lane) -> shared binary64; trace; ridge
    if (lane < r) {
#pragma unroll
        for (int a = 0; a < RMAX; ++a)
            if (a < r) Gs[wid][a][lane] = (double)g[a];
        bs[wid][lane] = (double)bl;
    }
    __syncwarp();
    double tr = 0.0;
    for (int a = 0; a < r; ++a) tr += Gs[wid][a][a];
    if (!(tr > 0.0)) {
        if (lane < r) Xout[o * r + lane] = TF(0);
        return;
    }
    if (lane < r) Gs[wid][lane][lane] += 1e-10 * tr / (double)r;
    __syncwarp();
    // in-place lower Cholesky
    for (int j = 0; j < r; ++j) {
        const double d = Gs[wid][j][j];
        if (!(d > 0.0)) {
            if (lane == 0) set_error(err, DEVERR_NUMERIC);
            if (lane < r) Xout[o * r + lane] = TF(0);
            return;
        }
        const double sd = sqrt(d);
        __syncwarp();
        if (lane == j) Gs[wid][j][j] = sd;
        if (lane > j && lane < r) Gs[wid][lane][j] /= sd;
        __syncwarp();
        if (lane > j && lane < r) {
            const double lij = Gs[wid][lane][j];
            for (int kk = j + 1; kk <= lane; ++kk) Gs[wid][lane][kk] -= lij * Gs[wid][kk][j];
        }
        __syncwarp();
    }
    // forward L y = b, then backward L^T x = y (lane j finalises entry j, the others update)
    for (int j = 0; j < r; ++j) {
        if (lane == j) bs[wid][j] /= Gs[wid][j][j];
        __syncwarp();
        const double yj = bs[wid][j];
        if (lane > j && lane < r) bs[wid][lane] -= Gs[wid][lane][j] * yj;
        __syncwarp();
    }
    for (int j = r - 1; j >= 0; --j) {
        if (lane == j) bs[wid][j] /= Gs[wid][j][j];
        __syncwarp();
        const double xj = bs[wid][j];
        if (lane < j) bs[wid][lane] -= Gs[wid][j][lane] * xj;
        __syncwarp();
    }
    if (lane < r) Xout[o * r + lane] = (TF)bs[wid][lane];
}

// ---------------------------------------------------------------------------------------------------------------
// canonical form
// ---------------------------------------------------------------------------------------------------------------
// K = Ru Rv^T and the augmented symmetric H = [[0, K], [K^T, 0]] (2r x 2r).
__global__ void core_kernel(const double* __restrict__ Ru, const double* __restrict__ Rv, int r, double* H) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = 2 * r;
    if (e >= n * n) return;
    const int i = e / n, j = e - i * n;
    double v = 0.0;
    if (i < r && j >= r) {
        const int jj = j - r;
        for (int l = 0; l < r; ++l) v += Ru[i * r + l] * Rv[jj * r + l];
    } else if (i >= r && j < r) {
        const int ii = i - r;
        for (int l = 0; l < r; ++l) v += Ru[j * r + l] * Rv[ii * r + l];
    }
    H[e] = v;
}

// From the eigenvectors of H (2r x 2r, sorted decreasing): S[c] = lambda_c, W = sqrt2 * top block, Z = sqrt2 *
// bottom block of the first r eigenvectors, each renormalised (a zero singular value leaves a zero column).
__global__ void core_split_kernel(const double* __restrict__ ev, const double* __restrict__ EV, int r, double* S,
                                  double* Wc, double* Zc) {
    const int c = threadIdx.x;
    if (c >= r) return;
    const int n = 2 * r;
    double nu = 0.0, nv = 0.0;
    for (int i = 0; i < r; ++i) {
        nu += EV[i * n + c] * EV[i * n + c];
        nv += EV[(r + i) * n + c] * EV[(r + i) * n + c];
    }
    nu = sqrt(nu);
    nv = sqrt(nv);
    const double lam = ev[c];
    S[c] = lam > 0.0 ? lam : 0.0;
    for (int i = 0; i < r; ++i) {
        Wc[i * r + c] = (lam > 0.0 && nu > 0.0) ? EV[i * n + c] / nu : 0.0;
        Zc[i * r + c] = (lam > 0.0 && nv > 0.0) ? EV[(r + i) * n + c] / nv : 0.0;
    }
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

unsigned nblocks(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Gram of X (n x a) with Y (n x b) into G (a x b), fixed-order reduction.
template <typename TX, typename TY>
void gram(const TX* X, const TY* Y, int64_t n, int a, int b, double* part, double* G, cudaStream_t st) {
    const int nblk = (int)std::max<int64_t>(1, (n + GRAM_ROWS_PER_BLOCK - 1) / GRAM_ROWS_PER_BLOCK);
    gram_partial_kernel<TX, TY><<<smp::counted(nblk), 256, 0, st>>>(X, Y, n, a, b, part);
    gram_reduce_kernel<<<smp::counted(nblocks(a * b, 256)), 256, 0, st>>>(part, nblk, a * b, G);
}

// Cholesky-QR twice: Q = X R^-1 with X = Q R; Rout = R2 R1 (upper). Q may alias nothing of X.
template <typename TX, typename TQ>
void cholqr2(const TX* X, int64_t n, int b, TQ* Q, double* part, double* G, double* R1, double* R2, double* Rout,
             cudaStream_t st);

__global__ void upper_mul_kernel(const double* __restrict__ R2, const double* __restrict__ R1, int b, double* R) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= b * b) return;
    const int i = e / b, j = e - i * b;
    double s = 0.0;
    for (int l = i; l <= j; ++l) s += R2[i * b + l] * R1[l * b + j];
    R[e] = j >= i ? s : 0.0;
}

template <typename TX, typename TQ>
void cholqr2(const TX* X, int64_t n, int b, TQ* Q, double* part, double* G, double* R1, double* R2, double* Rout,
             cudaStream_t st) {
    gram<TX, TX>(X, X, n, b, b, part, G, st);
    chol_kernel<<<smp::counted(1), 32, 0, st>>>(G, b, R1, 1e-28, nullptr);
    apply_rinv_kernel<TX, TQ><<<smp::counted(nblocks(n, 128)), 128, 0, st>>>(X, n, b, R1, Q);
    gram<TQ, TQ>(Q, Q, n, b, b, part, G, st);
    chol_kernel<<<smp::counted(1), 32, 0, st>>>(G, b, R2, 1e-28, nullptr);
    apply_rinv_kernel<TQ, TQ><<<smp::counted(nblocks(n, 128)), 128, 0, st>>>(Q, n, b, R2, Q);
    if (Rout) upper_mul_kernel<<<smp::counted(nblocks(b * b, 256)), 256, 0, st>>>(R2, R1, b, Rout);
}

template <typename TF, typename TG, typename TV>
void launch_ls(int r, const int64_t* ptr, const int32_t* idx, const int64_t* pos, const TV* vals,
               const double* qhat, const uint8_t* sub, int sid, const TF* Fin, int64_t n_out, TF* Xout, int* err,
               cudaStream_t st) {
    const unsigned g = nblocks(n_out, LS_WARPS);
    if (r <= 8)
        ls_kernel<TF, TG, TV, 8><<<smp::counted(g), 32 * LS_WARPS, 0, st>>>(ptr, idx, pos, vals, qhat, sub, sid, Fin, r, n_out,
                                                              Xout, err);
    else if (r <= 16)
        ls_kernel<TF, TG, TV, 16><<<smp::counted(g), 32 * LS_WARPS, 0, st>>>(ptr, idx, pos, vals, qhat, sub, sid, Fin, r,
                                                               n_out, Xout, err);
    else
        ls_kernel<TF, TG, TV, 32><<<smp::counted(g), 32 * LS_WARPS, 0, st>>>(ptr, idx, pos, vals, qhat, sub, sid, Fin, r,
                                                               n_out, Xout, err);
}

template <typename TV, typename TF, typename TG, typename TY>
smp_status waltmin_typed(smp_ctx* c, const TV* vals, int r, int T, uint32_t flags, uint64_t seed,
                         const double* U_init, double* U, double* S, double* V) {
    const int64_t n1 = c->p.n1, n2 = c->p.n2, nnz = c->nnz;
    cudaStream_t st = c->stream;
    const int b = (int)std::min<int64_t>(std::min<int64_t>(2 * r + 8, MAX_SMALL), std::min(n1, n2));
    const bool split = (flags & SMP_SPLIT_OMEGA) != 0;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);

    // scratch sizes
    const int64_t nmax = std::max(n1, n2);
    const int64_t gblk = std::max<int64_t>(1, (nmax + GRAM_ROWS_PER_BLOCK - 1) / GRAM_ROWS_PER_BLOCK);
    size_t need = 0;
    auto add = [&](int64_t n, size_t sz) { need += ((size_t)std::max<int64_t>(n, 1) * sz + 511) & ~size_t(255); };
    add(nnz, 4);                 // erow
    add(nnz, 1);                 // sub
    add(nnz, sizeof(TY));        // rv
    add(n1 * b, sizeof(TY));     // Y
    add(n2 * b, sizeof(TY));     // Z
    add(n1 * b, sizeof(TY));     // Ytmp
    add(gblk * b * b, 8);        // gram partials
    add(5 * b * b + 4 * b, 8);   // G, R1, R2, E, evals...
    add(2 * n1 * r, 8);          // U0, U0prev
    add(n1 * r, sizeof(TF));     // Uf
    add(n2 * r, sizeof(TF));     // Vf
    add(n1 * r, 8);              // Qu
    add(n2 * r, 8);              // Qv
    add(8 * r * r + 8 * r, 8);   // Ru, Rv, H, EV, W, Z, ...
    void* ws = nullptr;
    if (cudaMallocAsync(&ws, need, st) != cudaSuccess) return fail(c, SMP_ENOMEM, "smp_waltmin: scratch");
    Arena ar{(char*)ws, 0, need};
    int32_t* erow = ar.take<int32_t>(nnz);
    uint8_t* sub = ar.take<uint8_t>(nnz);
    TY* rv = ar.take<TY>(nnz);
    TY* Y = ar.take<TY>(n1 * b);
    TY* Z = ar.take<TY>(n2 * b);
    TY* Yt = ar.take<TY>(n1 * b);
    double* part = ar.take<double>(gblk * b * b);
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
    double* EV = ar.take<double>(4 * r * r);
    double* evh = ar.take<double>(2 * r);
    double* Wc = ar.take<double>(r * r);
    double* Zc = ar.take<double>(r * r);
    double* Rx1 = ar.take<double>(r * r);
    double* Rx2 = ar.take<double>(r * r);
    double* Gx = ar.take<double>(r * r);

    static bool attr_done = false;
    if (!attr_done) {
        cudaFuncSetAttribute(jacobi_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * MAX_SMALL * (MAX_SMALL + 1) * 8);
        attr_done = true;
    }
    auto jacobi = [&](const double* Ain, int n, double tol, double* evals, double* Vout) {
        jacobi_eig_kernel<<<smp::counted(1), 256, 2 * n * (n + 1) * 8, st>>>(Ain, n, tol, 40, evals, Vout);
    };

    if (nnz > 0) erow_kernel<<<smp::counted(nblocks(n1 * 32, 256)), 256, 0, st>>>(c->row_ptr, n1, erow);
    if (split && nnz > 0)
        split_kernel<<<smp::counted(nblocks(nnz, 256)), 256, 0, st>>>(erow, c->col, nnz, T, k0, k1, sub);
    const uint8_t* subp = split ? sub : nullptr;

    smp_status status = SMP_OK;
    if (flags & SMP_INIT_GIVEN) {
        convert_kernel<double, TF><<<smp::counted(nblocks(n1 * r, 256)), 256, 0, st>>>(U_init, n1 * r, Uf);
    } else {
        // R_Omega0(M~) values
        if (nnz > 0) rvals_kernel<TV, TY><<<smp::counted(nblocks(nnz, 256)), 256, 0, st>>>(vals, c->qhat, subp, 0, nnz, rv);
        start_block_kernel<TY><<<smp::counted(nblocks(n1 * ((b + 3) / 4), 256)), 256, 0, st>>>(n1, b, k0, k1, Y);
        cholqr2<TY, TY>(Y, n1, b, Y, part, G, R1, R2, nullptr, st);
        const bool dbl = sizeof(TY) == 8;
        const int max_iter = dbl ? 400 : 300;
        const double tol = dbl ? 1e-11 : 1e-5;
        const int check = 10;
        std::vector<double> hbuf(2);
        for (int it = 1; it <= max_iter; ++it) {
            spmm_csc_kernel<TY><<<smp::counted(nblocks(n2 * 32, 256)), 256, 0, st>>>(c->col_ptr, c->csc_row, c->csc_pos, rv, Y,
                                                                      n2, b, Z);
            spmm_csr_kernel<TY><<<smp::counted(nblocks(n1 * 32, 256)), 256, 0, st>>>(c->row_ptr, c->col, rv, Z, n1, b, Yt);
            cholqr2<TY, TY>(Yt, n1, b, Y, part, G, R1, R2, nullptr, st);
            if (it % check == 0 || it == max_iter) {
                // Rayleigh-Ritz on span(Y): C = Z^T Z with Z = R^T Y; U0 = Y E[:, :r]
                spmm_csc_kernel<TY><<<smp::counted(nblocks(n2 * 32, 256)), 256, 0, st>>>(c->col_ptr, c->csc_row, c->csc_pos,
                                                                          rv, Y, n2, b, Z);
                gram<TY, TY>(Z, Z, n2, b, b, part, G, st);
                jacobi(G, b, 1e-15, ev, E);
                ritz_kernel<TY><<<smp::counted(nblocks(n1 * r, 256)), 256, 0, st>>>(Y, E, n1, b, r, U0);
                if (it > check) {
                    // subspace change: dist^2 = r - ||U0^T U0prev||_F^2
                    gram<double, double>(U0, U0p, n1, r, r, part, Gx, st);
                    std::vector<double> hx(r * r);
                    if (cudaMemcpyAsync(hx.data(), Gx, sizeof(double) * r * r, cudaMemcpyDeviceToHost, st) !=
                            cudaSuccess ||
                        cudaStreamSynchronize(st) != cudaSuccess) {
                        status = check_cuda(c, cudaGetLastError(), "smp_waltmin init check");
                        break;
                    }
                    double fro = 0.0;
                    for (double v : hx) fro += v * v;
                    const double d2 = std::max(0.0, (double)r - fro);
                    if (std::sqrt(d2) < tol) break;
                }
                cudaMemcpyAsync(U0p, U0, sizeof(double) * n1 * r, cudaMemcpyDeviceToDevice, st);
            }
        }
        if (status == SMP_OK) {
            if (!(flags & SMP_NO_TRIM)) trim_kernel<<<smp::counted(nblocks(n1, 256)), 256, 0, st>>>(U0, n1, r, c->s_all, c->F);
            convert_kernel<double, TF><<<smp::counted(nblocks(n1 * r, 256)), 256, 0, st>>>(U0, n1 * r, Uf);
        }
    }
    if (status == SMP_OK) {
        for (int t = 0; t < T; ++t) {
            launch_ls<TF, TG, TV>(r, c->col_ptr, c->csc_row, c->csc_pos, vals, c->qhat, subp, 2 * t + 1, Uf, n2, Vf,
                                  c->dev_err, st);
            launch_ls<TF, TG, TV>(r, c->row_ptr, c->col, nullptr, vals, c->qhat, subp, 2 * t + 2, Vf, n1, Uf,
                                  c->dev_err, st);
        }
        if (T == 0) cudaMemsetAsync(Vf, 0, sizeof(TF) * n2 * r, st);
        // canonical form
        cholqr2<TF, double>(Uf, n1, r, Qu, part, Gx, Rx1, Rx2, Ru, st);
        cholqr2<TF, double>(Vf, n2, r, Qv, part, Gx, Rx1, Rx2, Rv, st);
        core_kernel<<<smp::counted(nblocks(4 * r * r, 256)), 256, 0, st>>>(Ru, Rv, r, H);
        jacobi(H, 2 * r, 1e-16, evh, EV);
        core_split_kernel<<<smp::counted(1), 32, 0, st>>>(evh, EV, r, S, Wc, Zc);
        small_right_mul_kernel<<<smp::counted(nblocks(n1 * r, 256)), 256, 0, st>>>(Qu, Wc, n1, r, U);
        small_right_mul_kernel<<<smp::counted(nblocks(n2 * r, 256)), 256, 0, st>>>(Qv, Zc, n2, r, V);
        sign_kernel<<<smp::counted(r), 256, 0, st>>>(U, n1, V, n2, r);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) status = check_cuda(c, e, "smp_waltmin kernels");
    }
    cudaFreeAsync(ws, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (status == SMP_OK && e != cudaSuccess) status = check_cuda(c, e, "smp_waltmin sync");
    if (status == SMP_OK) status = read_device_error(c);
    return status;
}

}  // namespace

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
