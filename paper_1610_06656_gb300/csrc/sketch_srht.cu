// Block subsampled randomized Hadamard transform as the sketching matrix (Section 4: the Spark implementation's
// Pi; its footnote: O(nd log d) time instead of O(ndk)). Data rows are cut into blocks of R = 2^p rows (the
// context's max_rows) and block b is sketched with Pi_b = k^-1/2 S_b H_R D_b: D_b random signs (Philox counter
// (t mod 2^32, t >> 32, 0, TAG_SRHT_SIGN), bit 0 of x0 set: -1), H_R the unnormalised Sylvester Walsh-Hadamard
// matrix, S_b k rows of H_R drawn uniformly with replacement (row a: the top p bits of x0 of counter
// (a, b mod 2^32, b >> 32, TAG_SRHT_ROW)).
//
// H_R factors over the bits of the row index: with t = 256 t1 + t2 and s = 256 s1 + s2,
// H_R[s][t] = H_{R/256}[s1][t1] H_256[s2][t2]. Stage A transforms every 256-row chunk t1 of the block over t2
// (registers: a length-64 transform over bits 2-7, a shared-memory exchange, length-4 transforms over bits 0-1),
// after the signs, into Y[t1][s2][c]; it also folds the squares of the raw values into compensated column sums.
// Stage B forms, for every sampled row a (bucketed by s2_a), At[c][a] += k^-1/2 sum over t1 of
// (-1)^popcount(s1_a & t1) Y[t1][s2_a][c]. Columns are processed in groups of SR_GROUP so that a group's Y
// (R x SR_GROUP binary32) stays in L2 between the two stages.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace smp {
namespace {

constexpr int SR_CHUNK = 256;   // rows per stage-A chunk (the H_256 factor)
constexpr int SR_COLS = 64;     // columns per CTA
constexpr int SR_GROUP = 256;   // columns per group (width of the Y scratch)
constexpr int SR_MAX_CHUNKS = 256;   // chunks per block: blocks of at most 2^16 rows

__device__ __forceinline__ bool srht_negative(int64_t t, uint32_t k0, uint32_t k1) {
    const U32x4 x = philox4x32_10((uint32_t)t, (uint32_t)((uint64_t)t >> 32), 0u, TAG_SRHT_SIGN, k0, k1);
    return (x.x & 1u) != 0u;
}

// In-register unnormalised Walsh-Hadamard transform of v[0..N) (N a power of two), Sylvester order.
template <int N>
__device__ __forceinline__ void fwht_regs(float* v) {
#pragma unroll
    for (int h = 1; h < N; h <<= 1)
#pragma unroll
        for (int i = 0; i < N; ++i)
            if ((i & h) == 0) {
                const float a = v[i], b = v[i + h];
                v[i] = a + b;
                v[i + h] = a - b;
            }
}

// Stage A. CTA (chunk t1, 64 columns of the group); thread (column cl = tid % 64, quarter q = tid / 64) holds the
// chunk's rows q + 4 i, i < 64. Output Y[(256 t1 + s) * SR_GROUP + column in group], s = 4 s_hi + s_lo; column sums
// of squares of the raw values into nsq_part[t1 * SR_GROUP + column in group].
__global__ void __launch_bounds__(256) srht_stage_a_kernel(const float* __restrict__ A, int64_t lda,
                                                           const float* __restrict__ B, int64_t ldb, int64_t n1,
                                                           int64_t row0, int64_t nrows, int64_t c0, int ncols,
                                                           uint32_t k0, uint32_t k1, float* Y, double* nsq_part) {
    extern __shared__ float ys[];   // [256][SR_COLS]
    __shared__ uint32_t neg[SR_CHUNK / 32];
    __shared__ double colsum[4][SR_COLS];
    const int tid = threadIdx.x, cl = tid & (SR_COLS - 1), q = tid >> 6;
    const int64_t t1 = blockIdx.x;
    const int64_t tb = t1 * SR_CHUNK;                       // first row of the chunk within the block
    const int gcol = blockIdx.y * SR_COLS + cl;             // column within the group
    const bool cvalid = gcol < ncols;
    const int64_t c = c0 + gcol;
    const float* src = (c < n1) ? A + c : B + (c - n1);
    const int64_t ld = (c < n1) ? lda : ldb;

    // all 64 loads first (the data is read once: streaming loads keep it from evicting the group's Y from L2),
    // the signs of the chunk's 256 rows (one Philox block per row) while they are in flight
    float v[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) {
        const int r = q + 4 * i;
        v[i] = (cvalid && tb + r < nrows) ? __ldcs(src + (tb + r) * ld) : 0.f;
    }
    {
        const int64_t t = tb + tid;
        const bool ng = t < nrows && srht_negative(row0 + t, k0, k1);
        const uint32_t bits = __ballot_sync(0xffffffffu, ng);
        if ((tid & 31) == 0) neg[tid >> 5] = bits;
    }
    __syncthreads();
    uint64_t hi2 = 0ull, lo2 = 0ull;
#pragma unroll
    for (int i = 0; i < 64; i += 2) {
        const int r0 = q + 4 * i, r1 = r0 + 4;
        tc::two_sum_square_x2(tc::pack2(v[i], v[i + 1]), hi2, lo2);
        if ((neg[r0 >> 5] >> (r0 & 31)) & 1u) v[i] = -v[i];
        if ((neg[r1 >> 5] >> (r1 & 31)) & 1u) v[i + 1] = -v[i + 1];
    }
    // bits 2-7 of the row index: v[i] is row 4 i + q
    fwht_regs<64>(v);
#pragma unroll
    for (int i = 0; i < 64; ++i) ys[(4 * i + q) * SR_COLS + cl] = v[i];
    {
        float h0, h1, l0, l1;
        tc::unpack2(hi2, h0, h1);
        tc::unpack2(lo2, l0, l1);
        colsum[q][cl] = ((double)h0 + (double)h1) + ((double)l0 + (double)l1);
    }
    __syncthreads();
    // bits 0-1: thread (cl, q) takes s_hi = q + 4 j, j < 16
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int sh = q + 4 * j;
        float w[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) w[l] = ys[(4 * sh + l) * SR_COLS + cl];
        fwht_regs<4>(w);
        if (cvalid)
#pragma unroll
            for (int l = 0; l < 4; ++l) Y[(tb + 4 * sh + l) * SR_GROUP + gcol] = w[l];
    }
    if (q == 0 && cvalid)
        nsq_part[t1 * SR_GROUP + gcol] = (colsum[0][cl] + colsum[1][cl]) + (colsum[2][cl] + colsum[3][cl]);
}

// Hadamard rows of block b: s_a = top p bits of x0; bucketed by s2 = s mod 256 (list[off[s2] .. off[s2 + 1])),
// s1 = s >> 8 alongside. One CTA.
__global__ void __launch_bounds__(1024) srht_rows_kernel(int k, int p, uint64_t b, uint32_t k0, uint32_t k1,
                                                         int32_t* off, int32_t* list, int32_t* s1) {
    __shared__ int32_t cnt[256], fill[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) cnt[i] = fill[i] = 0;
    __syncthreads();
    for (int a = threadIdx.x; a < k; a += blockDim.x) {
        const U32x4 x = philox4x32_10((uint32_t)a, (uint32_t)b, (uint32_t)(b >> 32), TAG_SRHT_ROW, k0, k1);
        const uint32_t s = x.x >> (32 - p);
        s1[a] = (int32_t)(s >> 8);
        atomicAdd(&cnt[s & 255u], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t acc = 0;
        for (int i = 0; i < 256; ++i) {
            off[i] = acc;
            acc += cnt[i];
        }
        off[256] = acc;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < k; a += blockDim.x) {
        const U32x4 x = philox4x32_10((uint32_t)a, (uint32_t)b, (uint32_t)(b >> 32), TAG_SRHT_ROW, k0, k1);
        const uint32_t s2 = (x.x >> (32 - p)) & 255u;
        list[off[s2] + atomicAdd(&fill[s2], 1)] = a;
    }
}

// Stage B. CTA (s2, 64 columns of the group): stages Y[t1][s2][cols] for the t1 < nchunks present, then for every
// sampled row a in bucket s2: part[c][a] += k^-1/2 sum_t1 (-1)^popcount(s1_a & t1) Y[t1][s2][c].
__global__ void __launch_bounds__(256) srht_stage_b_kernel(const float* __restrict__ Y, int nchunks,
                                                           const int32_t* __restrict__ off,
                                                           const int32_t* __restrict__ list,
                                                           const int32_t* __restrict__ s1, int64_t c0, int ncols,
                                                           float inv_sqrt_k, float* part, int64_t ldk) {
    extern __shared__ float ys[];   // [nchunks][SR_COLS]
    __shared__ float red[4][SR_COLS];
    const int s2 = blockIdx.x;
    const int a0 = off[s2], a1 = off[s2 + 1];
    if (a0 == a1) return;
    const int tid = threadIdx.x, cl = tid & (SR_COLS - 1), q = tid >> 6;
    const int gcol = blockIdx.y * SR_COLS + cl;
    const bool cvalid = gcol < ncols;
    for (int base = q; base < nchunks; base += 64) {   // 16 independent loads per thread at a time
        float tmp[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int t1 = base + 4 * u;
            tmp[u] = (cvalid && t1 < nchunks) ? __ldcs(Y + ((int64_t)t1 * SR_CHUNK + s2) * SR_GROUP + gcol) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u)
            if (base + 4 * u < nchunks) ys[(base + 4 * u) * SR_COLS + cl] = tmp[u];
    }
    __syncthreads();
    for (int e = a0; e < a1; ++e) {
        const int a = list[e];
        const uint32_t sa = (uint32_t)s1[a];
        float acc = 0.f;
        for (int t1 = q; t1 < nchunks; t1 += 4) {
            const float y = ys[t1 * SR_COLS + cl];
            acc += (__popc(sa & (uint32_t)t1) & 1) ? -y : y;
        }
        red[q][cl] = acc;
        __syncthreads();
        if (q == 0 && cvalid) {
            float* dst = part + (c0 + gcol) * ldk + a;
            *dst += inv_sqrt_k * ((red[0][cl] + red[1][cl]) + (red[2][cl] + red[3][cl]));
        }
        __syncthreads();
    }
}

// nsq[c] += sum over the chunks of nsq_part[t1][c - c0]: one warp per column, lane l sums chunks l, l + 32, ...
// in order, then a fixed shuffle tree.
__global__ void srht_norms_kernel(const double* __restrict__ nsq_part, int nchunks, int64_t c0, int ncols,
                                  double* nsq) {
    const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= ncols) return;
    double s = 0.0;
    for (int t1 = lane; t1 < nchunks; t1 += 32) s += nsq_part[(int64_t)t1 * SR_GROUP + g];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) nsq[c0 + g] += s;
}

}  // namespace

bool srht_block_ok(const smp_ctx* c, int64_t row0, int64_t nrows) {
    const int64_t R = c->max_rows;
    return row0 % R == 0 && nrows <= R;
}

cudaError_t launch_sketch_srht(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                               int64_t nrows) {
    const int64_t R = c->max_rows;
    int p = 0;
    while (((int64_t)1 << p) < R) ++p;
    const int nchunks = (int)((nrows + SR_CHUNK - 1) / SR_CHUNK);
    const int k = c->p.k;
    cudaStream_t st = c->stream;
    if (!c->srht_y) {
        cudaError_t e = cudaMallocAsync((void**)&c->srht_y, (size_t)R * SR_GROUP * 4, st);
        if (e == cudaSuccess) e = cudaMallocAsync((void**)&c->srht_nsq, (size_t)(R / SR_CHUNK) * SR_GROUP * 8, st);
        if (e == cudaSuccess) e = cudaMallocAsync((void**)&c->srht_rows, (size_t)(257 + 2 * 1024) * 4, st);
        if (e != cudaSuccess) return e;
        static std::atomic<bool> attr{false};
        if (!attr) {
            e = cudaFuncSetAttribute(srht_stage_a_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     SR_CHUNK * SR_COLS * 4);
            if (e == cudaSuccess)   // up to 256 chunks (2^16-row blocks)
                e = cudaFuncSetAttribute(srht_stage_b_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         SR_MAX_CHUNKS * SR_COLS * 4);
            if (e != cudaSuccess) return e;
            attr = true;
        }
    }
    const uint32_t k0 = (uint32_t)c->p.seed, k1 = (uint32_t)(c->p.seed >> 32);
    int32_t* off = c->srht_rows;
    int32_t* list = off + 257;
    int32_t* s1 = list + 1024;
    srht_rows_kernel<<<smp::counted(1), 1024, 0, st>>>(k, p, (uint64_t)(row0 / R), k0, k1, off, list, s1);
    const float* Af = (const float*)A;
    const float* Bf = c->p.same_ab ? Af : (const float*)B;
    const int64_t ldb_eff = c->p.same_ab ? lda : ldb;
    float* part = (float*)c->part;   // split 0
    const float inv_sqrt_k = (float)(1.0 / std::sqrt((double)k));
    for (int64_t c0 = 0; c0 < c->ntot; c0 += SR_GROUP) {
        const int ncols = (int)std::min<int64_t>(SR_GROUP, c->ntot - c0);
        const unsigned tiles = (unsigned)((ncols + SR_COLS - 1) / SR_COLS);
        srht_stage_a_kernel<<<smp::counted(dim3((unsigned)nchunks, tiles)), 256, SR_CHUNK * SR_COLS * 4, st>>>(
            Af, lda, Bf, ldb_eff, c->p.n1, row0, nrows, c0, ncols, k0, k1, c->srht_y, c->srht_nsq);
        srht_stage_b_kernel<<<smp::counted(dim3(256u, tiles)), 256, (size_t)nchunks * SR_COLS * 4, st>>>(
            c->srht_y, nchunks, off, list, s1, c0, ncols, inv_sqrt_k, part, c->ldk);
        srht_norms_kernel<<<smp::counted((unsigned)((ncols * 32 + 255) / 256)), 256, 0, st>>>(c->srht_nsq, nchunks,
                                                                                             c0, ncols, c->nsq);
    }
    return cudaGetLastError();
}

}  // namespace smp
