// Biased Bernoulli sampling of Omega (Algorithm 1, step 3; Eq. (1)).
//
// The coin of (i, j) is u_ij < q^_ij with q_ij = alpha_i + beta_j, alpha_i = m * (s_A,i / ((2 n2) F_A)),
// beta_j = m * (s_B,j / ((2 n1) F_B)), F = sum of the column sums of squares left to right. Every floating-point
// step is a single round-to-nearest binary64 operation written with the _rn intrinsics (never contracted), so two
// implementations that follow the same order draw the same Omega bit for bit.
//
// Pipeline: terms (alpha, beta from F) -> coin words (one warp per 32 columns of a row: ballot of the 32 coins,
// popcount per word, column counts) -> per-row prefix over words -> scans to row_ptr / col_ptr -> CSR fill from
// the bit words -> CSC fill (one CTA per column, block scan over rows, CSR position from the word prefix).
//
// Row-wise multinomial sampling (Appendix, "Sampling"): blocked prefix sums Bcum of beta (1,024-element blocks,
// sequential within and across blocks) -> row totals S_i = n2 alpha_i + Bcum_{n2-1} and draws c_i = floor(S_i + 1/2)
// -> one thread per draw s of row i: u (Philox counter (i, s, 0, TAG_MULTI)), t = u S_i, binary search for the
// smallest j with t < (j + 1) alpha_i + Bcum_j; the drawn pair sets its bit in the same words as the coins (the first
// draw of a pair counts its column) -> the Bernoulli path's prefix, scans and fills -> per draw, the count of its
// CSR entry -> q^ = (c_i ((alpha_i + beta_j) / S_i)) / count_ij.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace smp {
namespace {

// alpha, beta from the column sums of squares and the Frobenius squares F (left-to-right sums, already in F).
__global__ void terms_kernel(const double* __restrict__ s_all, int64_t n1, int64_t n2, int same_ab, double m,
                             const double* __restrict__ F, double* alpha, double* beta) {
    const double fa = F[0], fb = F[1];
    const double* sB = same_ab ? s_all : s_all + n1;
    const double da = __dmul_rn((double)(2 * n2), fa);
    const double db = __dmul_rn((double)(2 * n1), fb);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n1) alpha[t] = fa > 0.0 ? __dmul_rn(m, __ddiv_rn(s_all[t], da)) : 0.0;
    if (t < n2) beta[t] = fb > 0.0 ? __dmul_rn(m, __ddiv_rn(sB[t], db)) : 0.0;
}

__device__ __forceinline__ double qhat_of(double a, double b) {
    const double q = __dadd_rn(a, b);
    return q < 1.0 ? q : 1.0;
}

// One warp per (row i, word w): lane l flips the coin of column 32 w + l.
__global__ void coin_kernel(const double* __restrict__ alpha, const double* __restrict__ beta, int64_t n1,
                            int64_t n2, int64_t W, uint32_t k0, uint32_t k1, uint32_t* mask, int32_t* col_cnt) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n1 * W) return;
    const int64_t i = warp / W, w = warp - i * W;
    const int64_t j = w * 32 + lane;
    bool keep = false;
    if (j < n2) {
        const double u = coin((uint32_t)i, (uint32_t)j, TAG_SAMPLE, k0, k1);
        keep = u < qhat_of(alpha[i], beta[j]);
    }
    const uint32_t bits = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) mask[warp] = bits;
    if (keep) atomicAdd(&col_cnt[j], 1);
}

// Per row: exclusive prefix of the word popcounts and the row total (one CTA per row, sequential in chunks).
__global__ void row_prefix_kernel(const uint32_t* __restrict__ mask, int64_t n1, int64_t W, int32_t* wpre,
                                  int32_t* row_cnt) {
    __shared__ int32_t wsum[32];
    __shared__ int32_t carry;
    const int64_t i = blockIdx.x;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < W; base += blockDim.x) {
        const int64_t w = base + threadIdx.x;
        const int32_t c = w < W ? __popc(mask[i * W + w]) : 0;
        // block exclusive scan of c
        int32_t x = c;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int32_t v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            wsum[lane] = v;
        }
        __syncthreads();
        const int32_t excl = x - c + (wid ? wsum[wid - 1] : 0) + carry;
        if (w < W) wpre[i * W + w] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + c;
        __syncthreads();
    }
    if (threadIdx.x == 0) row_cnt[i] = carry;
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

// CSR fill: one warp per word; kept lanes write their column and q^ at row_ptr + word prefix + lanes below.
__global__ void fill_csr_kernel(const uint32_t* __restrict__ mask, const int32_t* __restrict__ wpre,
                                const int64_t* __restrict__ row_ptr, const double* __restrict__ alpha,
                                const double* __restrict__ beta, int64_t n1, int64_t n2, int64_t W, int32_t* col,
                                int32_t* erow, double* qhat) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n1 * W) return;
    const uint32_t bits = mask[warp];
    if (!((bits >> lane) & 1u)) return;
    const int64_t i = warp / W, w = warp - i * W;
    const int64_t j = w * 32 + lane;
    const int64_t pos = row_ptr[i] + wpre[warp] + __popc(bits & ((1u << lane) - 1u));
    col[pos] = (int32_t)j;
    erow[pos] = (int32_t)i;
    qhat[pos] = qhat_of(alpha[i], beta[j]);
}

// CSC fill: one CTA per column j; block scan over rows keeps rows in increasing order.
__global__ void fill_csc_kernel(const uint32_t* __restrict__ mask, const int32_t* __restrict__ wpre,
                                const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ col_ptr,
                                int64_t n1, int64_t W, int32_t* csc_row, int64_t* csc_pos) {
    __shared__ int32_t wsum[32];
    __shared__ int64_t carry;
    const int64_t j = blockIdx.x;
    const int64_t w = j >> 5;
    const int b = (int)(j & 31);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = col_ptr[j];
    __syncthreads();
    for (int64_t base = 0; base < n1; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        uint32_t bits = 0;
        int32_t keep = 0;
        if (i < n1) {
            bits = mask[i * W + w];
            keep = (bits >> b) & 1u;
        }
        int32_t x = keep;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int32_t v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            wsum[lane] = v;
        }
        __syncthreads();
        const int32_t excl = x - keep + (wid ? wsum[wid - 1] : 0);
        if (keep) {
            const int64_t p = carry + excl;
            csc_row[p] = (int32_t)i;
            csc_pos[p] = row_ptr[i] + wpre[i * W + w] + __popc(bits & ((1u << b) - 1u));
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += excl + keep;
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------------ multinomial
constexpr int MN_BLOCK = 1024;   // prefix-sum block of beta

// Within-block inclusive prefix of beta, left to right (one thread per block); the block total into btot[b].
__global__ void mn_block_prefix_kernel(const double* __restrict__ beta, int64_t n2, double* bcum, double* btot) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t j0 = b * MN_BLOCK;
    if (j0 >= n2) return;
    const int64_t j1 = min(n2, j0 + MN_BLOCK);
    double s = beta[j0];
    bcum[j0] = s;
    for (int64_t j = j0 + 1; j < j1; ++j) {
        s = __dadd_rn(s, beta[j]);
        bcum[j] = s;
    }
    btot[b] = s;
}

// Block offsets, sequential: btot[b] <- sum of the totals of the blocks before b (btot[0] = 0). One thread.
__global__ void mn_block_offsets_kernel(double* btot, int64_t nb) {
    double off = 0.0;
    for (int64_t b = 0; b < nb; ++b) {
        const double t = btot[b];
        btot[b] = off;
        off = __dadd_rn(off, t);
    }
}

// Bcum_j = offset of j's block + within-block prefix (one addition, also for the first block's 0).
__global__ void mn_add_offsets_kernel(double* bcum, const double* __restrict__ boff, int64_t n2) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n2) bcum[j] = __dadd_rn(boff[j / MN_BLOCK], bcum[j]);
}

// S_i = n2 alpha_i + Bcum_{n2-1}; c_i = floor(S_i + 1/2).
__global__ void mn_rows_kernel(const double* __restrict__ alpha, const double* __restrict__ bcum, int64_t n1,
                               int64_t n2, double* S, int32_t* cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n1) return;
    const double s = __dadd_rn(__dmul_rn((double)n2, alpha[i]), bcum[n2 - 1]);
    S[i] = s;
    cnt[i] = (int32_t)floor(__dadd_rn(s, 0.5));
}

// Row of draw d: the last i with off[i] <= d (off non-decreasing, off[0] = 0 <= d < off[n1]).
__device__ __forceinline__ int64_t mn_row_of(const int64_t* __restrict__ off, int64_t n1, int64_t d) {
    int64_t lo = 0, hi = n1;   // answer in [lo, hi)
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= d) lo = mid;
        else hi = mid;
    }
    return lo;
}

// One thread per draw: the column by binary search on the row's CDF; sets the pair's bit (the first draw of a pair
// counts its column).
__global__ void mn_draw_kernel(const double* __restrict__ alpha, const double* __restrict__ bcum,
                               const double* __restrict__ S, const int64_t* __restrict__ off, int64_t n1, int64_t n2,
                               int64_t W, int64_t ndraw, uint32_t k0, uint32_t k1, int32_t* draw, uint32_t* mask,
                               int32_t* col_cnt) {
    const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= ndraw) return;
    const int64_t i = mn_row_of(off, n1, d);
    const int64_t s = d - off[i];
    const double u = coin((uint32_t)i, (uint32_t)s, TAG_MULTI, k0, k1);
    const double t = __dmul_rn(u, S[i]);
    const double a = alpha[i];
    int64_t lo = 0, hi = n2;   // smallest j with t < (j + 1) a + Bcum_j; n2 if none
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const double v = __dadd_rn(__dmul_rn((double)(mid + 1), a), bcum[mid]);
        if (t < v) hi = mid;
        else lo = mid + 1;
    }
    const int64_t j = lo < n2 ? lo : n2 - 1;
    draw[d] = (int32_t)j;
    const uint32_t bit = 1u << (j & 31);
    const uint32_t old = atomicOr(&mask[i * W + (j >> 5)], bit);
    if (!(old & bit)) atomicAdd(&col_cnt[j], 1);
}

// Per draw: one more count on its CSR entry (position from the word prefix, as in the CSR fill).
__global__ void mn_count_kernel(const int32_t* __restrict__ draw, const int64_t* __restrict__ off, int64_t n1,
                                int64_t W, int64_t ndraw, const uint32_t* __restrict__ mask,
                                const int32_t* __restrict__ wpre, const int64_t* __restrict__ row_ptr, int32_t* count) {
    const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= ndraw) return;
    const int64_t i = mn_row_of(off, n1, d);
    const int64_t j = draw[d];
    const int64_t w = j >> 5;
    const int b = (int)(j & 31);
    const int64_t pos = row_ptr[i] + wpre[i * W + w] + __popc(mask[i * W + w] & ((1u << b) - 1u));
    atomicAdd(&count[pos], 1);
}

// q^ of each entry: (c_i ((alpha_i + beta_j) / S_i)) / count_ij.
__global__ void mn_qhat_kernel(const int32_t* __restrict__ erow, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ count, const double* __restrict__ alpha,
                               const double* __restrict__ beta, const double* __restrict__ S,
                               const int32_t* __restrict__ rows_cnt, int64_t nnz, double* qhat) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    const int64_t i = erow[p], j = col[p];
    const double q = __ddiv_rn(__dadd_rn(alpha[i], beta[j]), S[i]);
    qhat[p] = __ddiv_rn(__dmul_rn((double)rows_cnt[i], q), (double)count[p]);
}

template <typename T>
cudaError_t ensure(T*& p, int64_t& have, int64_t need, cudaStream_t st) {
    if (have >= need && p) return cudaSuccess;
    free_after(p, st);
    p = nullptr;
    have = 0;
    cudaError_t e = dev_malloc((void**)&p, (size_t)std::max<int64_t>(need, 1) * sizeof(T), st);
    if (e == cudaSuccess) have = need;
    return e;
}

}  // namespace

smp_status run_sample(smp_ctx* c, double m, uint64_t seed, int64_t* nnz_out, bool multinomial) {
    const int64_t n1 = c->p.n1, n2 = c->p.n2;
    const int64_t W = (n2 + 31) / 32;
    cudaStream_t st = c->stream;
    if (c->mask_words < n1 * W) {
        free_after(c->mask, st);
        free_after(c->wpre, st);
        c->mask = nullptr;
        c->wpre = nullptr;
        c->mask_words = 0;
        if (dev_malloc((void**)&c->mask, (size_t)(n1 * W) * 4, st) != cudaSuccess ||
            dev_malloc((void**)&c->wpre, (size_t)(n1 * W) * 4, st) != cudaSuccess)
            return fail(c, SMP_ENOMEM, "smp_sample: cannot allocate the coin bit words");
        c->mask_words = n1 * W;
    }
    cudaError_t e;
    terms_kernel<<<smp::counted((unsigned)((std::max(n1, n2) + 255) / 256)), 256, 0, st>>>(c->s_all, n1, n2, c->p.same_ab, m,
                                                                                    c->F, c->alpha, c->beta);
    if ((e = cudaMemsetAsync(c->col_cnt, 0, (size_t)n2 * 4, st)) != cudaSuccess) return check_cuda(c, e, "memset");
    const int64_t warps = n1 * W;
    const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    int64_t ndraw = 0;
    if (!multinomial) {
        coin_kernel<<<smp::counted(blocks), 256, 0, st>>>(c->alpha, c->beta, n1, n2, W, k0, k1, c->mask, c->col_cnt);
    } else {
        const int64_t nb = (n2 + MN_BLOCK - 1) / MN_BLOCK;
        if (!c->mn_S) {
            if (dev_malloc((void**)&c->mn_S, (size_t)n1 * 8, st) != cudaSuccess ||
                dev_malloc((void**)&c->mn_bcum, (size_t)n2 * 8, st) != cudaSuccess ||
                dev_malloc((void**)&c->mn_btot, (size_t)nb * 8, st) != cudaSuccess ||
                dev_malloc((void**)&c->mn_rows, (size_t)n1 * 4, st) != cudaSuccess ||
                dev_malloc((void**)&c->mn_off, (size_t)(n1 + 1) * 8, st) != cudaSuccess)
                return fail(c, SMP_ENOMEM, "smp_sample_multinomial: cannot allocate the row tables");
        }
        if ((e = cudaMemsetAsync(c->mask, 0, (size_t)(n1 * W) * 4, st)) != cudaSuccess)
            return check_cuda(c, e, "memset");
        mn_block_prefix_kernel<<<smp::counted((unsigned)((nb + 127) / 128)), 128, 0, st>>>(c->beta, n2, c->mn_bcum,
                                                                                           c->mn_btot);
        mn_block_offsets_kernel<<<smp::counted(1), 1, 0, st>>>(c->mn_btot, nb);
        mn_add_offsets_kernel<<<smp::counted((unsigned)((n2 + 255) / 256)), 256, 0, st>>>(c->mn_bcum, c->mn_btot, n2);
        mn_rows_kernel<<<smp::counted((unsigned)((n1 + 255) / 256)), 256, 0, st>>>(c->alpha, c->mn_bcum, n1, n2,
                                                                                   c->mn_S, c->mn_rows);
        scan_kernel<<<smp::counted(1), 1024, 0, st>>>(c->mn_rows, n1, c->mn_off);
        if ((e = cudaMemcpyAsync(&ndraw, c->mn_off + n1, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return check_cuda(c, e, "smp_sample_multinomial draw count");
        if (ndraw > c->mn_draw_cap) {
            free_after(c->mn_draw, st);
            c->mn_draw = nullptr;
            c->mn_draw_cap = 0;
            if (dev_malloc((void**)&c->mn_draw, (size_t)ndraw * 4, st) != cudaSuccess)
                return fail(c, SMP_ENOMEM, "smp_sample_multinomial: cannot allocate the draws");
            c->mn_draw_cap = ndraw;
        }
        if (ndraw > 0)
            mn_draw_kernel<<<smp::counted((unsigned)((ndraw + 255) / 256)), 256, 0, st>>>(
                c->alpha, c->mn_bcum, c->mn_S, c->mn_off, n1, n2, W, ndraw, k0, k1, c->mn_draw, c->mask, c->col_cnt);
    }

    row_prefix_kernel<<<smp::counted((unsigned)n1), 256, 0, st>>>(c->mask, n1, W, c->wpre, c->row_cnt);
    scan_kernel<<<smp::counted(1), 1024, 0, st>>>(c->row_cnt, n1, c->row_ptr);
    scan_kernel<<<smp::counted(1), 1024, 0, st>>>(c->col_cnt, n2, c->col_ptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return check_cuda(c, e, "smp_sample count kernels");
    int64_t nnz = 0;
    if ((e = cudaMemcpyAsync(&nnz, c->row_ptr + n1, sizeof(int64_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return check_cuda(c, e, "smp_sample nnz copy");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return check_cuda(c, e, "smp_sample sync");
    if (nnz > c->cap) {
        int64_t have = c->cap, h2 = c->cap, h3 = c->cap, h4 = c->cap, h5 = c->cap;
        const int64_t want = nnz + nnz / 8 + 1024;
        if (ensure(c->col, have, want, st) != cudaSuccess || ensure(c->qhat, h2, want, st) != cudaSuccess ||
            ensure(c->csc_row, h3, want, st) != cudaSuccess || ensure(c->csc_pos, h4, want, st) != cudaSuccess ||
            ensure(c->erow, h5, want, st) != cudaSuccess)
            return fail(c, SMP_ENOMEM, "smp_sample: cannot allocate Omega");
        c->cap = want;
    }
    if (nnz > 0) {
        fill_csr_kernel<<<smp::counted(blocks), 256, 0, st>>>(c->mask, c->wpre, c->row_ptr, c->alpha, c->beta, n1, n2, W, c->col,
                                                c->erow, c->qhat);
        fill_csc_kernel<<<smp::counted((unsigned)n2), 256, 0, st>>>(c->mask, c->wpre, c->row_ptr, c->col_ptr, n1, W, c->csc_row,
                                                      c->csc_pos);
        if (multinomial) {
            if (nnz > c->mn_count_cap) {
                free_after(c->mn_count, st);
                c->mn_count = nullptr;
                c->mn_count_cap = 0;
                if (dev_malloc((void**)&c->mn_count, (size_t)c->cap * 4, st) != cudaSuccess)
                    return fail(c, SMP_ENOMEM, "smp_sample_multinomial: cannot allocate the counts");
                c->mn_count_cap = c->cap;
            }
            if ((e = cudaMemsetAsync(c->mn_count, 0, (size_t)nnz * 4, st)) != cudaSuccess)
                return check_cuda(c, e, "memset");
            mn_count_kernel<<<smp::counted((unsigned)((ndraw + 255) / 256)), 256, 0, st>>>(
                c->mn_draw, c->mn_off, n1, W, ndraw, c->mask, c->wpre, c->row_ptr, c->mn_count);
            mn_qhat_kernel<<<smp::counted((unsigned)((nnz + 255) / 256)), 256, 0, st>>>(
                c->erow, c->col, c->mn_count, c->alpha, c->beta, c->mn_S, c->mn_rows, nnz, c->qhat);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return check_cuda(c, e, "smp_sample fill kernels");
    }

    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return check_cuda(c, e, "smp_sample fill sync");
    c->nnz = nnz;
    c->sampled = true;
    if (nnz_out) *nnz_out = nnz;
    return SMP_OK;
}

}  // namespace smp
