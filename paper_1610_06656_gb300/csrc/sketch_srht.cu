// Block subsampled randomized Hadamard transform as the sketching matrix (Section 4: the Spark implementation's
// Pi; its footnote: O(nd log d) time instead of O(ndk)). Data rows are cut into blocks of R = 2^p rows (the
// context's max_rows) and block b is sketched with Pi_b = k^-1/2 S_b H_R D_b: D_b random signs (Philox counter
// (t mod 2^32, t >> 32, 0, TAG_SRHT_SIGN), bit 0 of x0 set: -1), H_R the unnormalised Sylvester Walsh-Hadamard
// matrix, S_b k rows of H_R drawn uniformly with replacement (row a: the top p bits of x0 of counter
// (a, b mod 2^32, b >> 32, TAG_SRHT_ROW)).
//
// H_R factors over the bits of the row index: with t = 256 t1 + t2 and s = 256 s1 + s2,
// H_R[s][t] = H_{R/256}[s1][t1] H_256[s2][t2]. One pass: a CTA owns 32 columns, a range of 256-row chunks t1 and up
// to 512 sampled rows a. For every chunk it loads the 256 x 32 tile once, folds the squares of the raw values into
// compensated column sums, applies the signs and transforms the tile over t2 (a length-32 transform in registers
// over row-index bits 3-7, a shared-memory exchange, length-8 transforms over bits 0-2) into Y[s2][c]; then every
// sampled row a adds (-1)^popcount(s1_a & t1) Y[s2_a][c] to its accumulator, held in registers (thread (c, q) owns
// rows a = q + 8 j). The row splits of the chunk range write the context's per-split partials, which the finalize
// step sums in a fixed order, like the other engines.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace smp {
namespace {

constexpr int SR_CHUNK = 256;    // rows per chunk (the H_256 factor)
constexpr int SR_COLS = 32;      // columns per CTA
constexpr int SR_AROWS = 512;    // sampled rows per CTA (64 accumulators per thread)
constexpr int SR_ACC = SR_AROWS / 8;
constexpr int SR_THREADS = 256;  // thread (column c = tid % 32, octet q = tid / 32)

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

struct SrhtArgs {
    const float* A;
    const float* B;
    int64_t lda, ldb, n1, ntot;
    int64_t row0, nrows;
    int k, p, nchunks, chunks_per_split;
    uint64_t block;          // global block index b = row0 / R
    uint32_t k0, k1;
    float inv_sqrt_k;
    float* part;             // [splits][ntot][ldk]
    double* nsq;             // [splits][ntot]
    int64_t ldk;
};

__global__ void __launch_bounds__(SR_THREADS, 2) srht_fused_kernel(const SrhtArgs a) {
    __shared__ float ys[SR_CHUNK][SR_COLS];   // the chunk, then its transform over t2 (row s2)
    __shared__ uint32_t srow[SR_AROWS];       // sampled Hadamard row of a0 + i: s1 << 8 | s2
    __shared__ uint32_t neg[SR_CHUNK / 32];
    __shared__ double colsum[8][SR_COLS];
    const int tid = threadIdx.x, cl = tid & (SR_COLS - 1), q = tid >> 5;
    const int64_t c = (int64_t)blockIdx.x * SR_COLS + cl;
    const bool cvalid = c < a.ntot;
    const int split = blockIdx.y;
    const int a0 = blockIdx.z * SR_AROWS;
    const int ka = min(SR_AROWS, a.k - a0);
    const int cs = split * a.chunks_per_split, ce = min(a.nchunks, cs + a.chunks_per_split);
    if (cs >= ce || ka <= 0) return;
    const float* src = !cvalid ? a.A : (c < a.n1 ? a.A + c : a.B + (c - a.n1));
    const int64_t ld = c < a.n1 ? a.lda : a.ldb;

    for (int i = tid; i < ka; i += SR_THREADS) {
        const U32x4 x = philox4x32_10((uint32_t)(a0 + i), (uint32_t)a.block, (uint32_t)(a.block >> 32), TAG_SRHT_ROW,
                                      a.k0, a.k1);
        srow[i] = x.x >> (32 - a.p);   // s = 256 s1 + s2 (p >= 8)
    }
    float acc[SR_ACC];
#pragma unroll
    for (int j = 0; j < SR_ACC; ++j) acc[j] = 0.f;
    uint64_t hi2 = 0ull, lo2 = 0ull;

    for (int t1 = cs; t1 < ce; ++t1) {
        const int64_t tb = (int64_t)t1 * SR_CHUNK;
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {   // rows q + 8 i of the chunk: every warp reads 32 consecutive columns
            const int r = q + 8 * i;
            v[i] = (cvalid && tb + r < a.nrows) ? __ldcs(src + (tb + r) * ld) : 0.f;
        }
        {
            const int64_t t = tb + tid;
            const bool ng = t < a.nrows && srht_negative(a.row0 + t, a.k0, a.k1);
            const uint32_t bits = __ballot_sync(0xffffffffu, ng);
            if ((tid & 31) == 0) neg[tid >> 5] = bits;
        }
        __syncthreads();   // signs ready; the previous chunk's accumulation has read ys
#pragma unroll
        for (int i = 0; i < 32; i += 2) {
            tc::two_sum_square_x2(tc::pack2(v[i], v[i + 1]), hi2, lo2);
            const int r0 = q + 8 * i, r1 = r0 + 8;
            if ((neg[r0 >> 5] >> (r0 & 31)) & 1u) v[i] = -v[i];
            if ((neg[r1 >> 5] >> (r1 & 31)) & 1u) v[i + 1] = -v[i + 1];
        }
        fwht_regs<32>(v);   // over row-index bits 3-7: v[i] is row 8 i + q
#pragma unroll
        for (int i = 0; i < 32; ++i) ys[8 * i + q][cl] = v[i];
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {   // bits 0-2: thread (cl, q) owns rows 8 sh .. 8 sh + 7, sh = q + 8 jj
            const int sh = q + 8 * jj;
            float w[8];
#pragma unroll
            for (int l = 0; l < 8; ++l) w[l] = ys[8 * sh + l][cl];
            fwht_regs<8>(w);
#pragma unroll
            for (int l = 0; l < 8; ++l) ys[8 * sh + l][cl] = w[l];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < SR_ACC; ++j) {
            const int i = q + 8 * j;
            if (i < ka) {
                const uint32_t s = srow[i];
                const float y = ys[s & 255u][cl];
                acc[j] += (__popc((s >> 8) & (uint32_t)t1) & 1) ? -y : y;
            }
        }
    }
    // compensated column sums: the eight octets of each column in a fixed order (first sampled-row group only)
    {
        float h0, h1, l0, l1;
        tc::unpack2(hi2, h0, h1);
        tc::unpack2(lo2, l0, l1);
        colsum[q][cl] = ((double)h0 + (double)h1) + ((double)l0 + (double)l1);
    }
    __syncthreads();   // also: the last accumulation has read ys
    if (blockIdx.z == 0 && q == 0 && cvalid) {
        double s = 0.0;
#pragma unroll
        for (int g = 0; g < 8; ++g) s += colsum[g][cl];
        a.nsq[(int64_t)split * a.ntot + c] += s;
    }
    // accumulators out through shared memory so that each warp adds 32 consecutive sketch rows of one column
    float* stage = &ys[0][0];   // 8,192 floats: 256 sampled rows x 32 columns per round
    for (int round = 0; round < 2; ++round) {
#pragma unroll
        for (int jj = 0; jj < SR_ACC / 2; ++jj)   // local row q + 8 jj of this round holds sampled row 256 round + ..
            stage[(q + 8 * jj) * SR_COLS + cl] = acc[round * (SR_ACC / 2) + jj];
        __syncthreads();
        const int i = round * 256 + tid;   // sampled row (relative to a0) this thread writes out
        if (i < ka) {
            for (int cc = 0; cc < SR_COLS; ++cc) {
                const int64_t col = (int64_t)blockIdx.x * SR_COLS + cc;
                if (col >= a.ntot) break;
                float* dst = a.part + ((int64_t)split * a.ntot + col) * a.ldk + a0 + i;
                *dst += a.inv_sqrt_k * stage[tid * SR_COLS + cc];
            }
        }
        __syncthreads();
    }
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
    SrhtArgs a;
    a.A = (const float*)A;
    a.B = c->p.same_ab ? a.A : (const float*)B;
    a.lda = lda;
    a.ldb = c->p.same_ab ? lda : ldb;
    a.n1 = c->p.n1;
    a.ntot = c->ntot;
    a.row0 = row0;
    a.nrows = nrows;
    a.k = c->p.k;
    a.p = p;
    a.nchunks = (int)((nrows + SR_CHUNK - 1) / SR_CHUNK);
    a.block = (uint64_t)(row0 / R);
    a.k0 = (uint32_t)c->p.seed;
    a.k1 = (uint32_t)(c->p.seed >> 32);
    a.inv_sqrt_k = (float)(1.0 / std::sqrt((double)a.k));
    a.part = (float*)c->part;
    a.nsq = c->nsq;
    a.ldk = c->ldk;
    const int tiles = (int)((c->ntot + SR_COLS - 1) / SR_COLS);
    const int agroups = (a.k + SR_AROWS - 1) / SR_AROWS;
    // row splits of the chunk range: about two waves of two CTAs per SM, at most the context's partial buffers
    int splits = (int)std::max<int64_t>(1, (4 * (int64_t)c->sm_count + tiles * agroups - 1) / (tiles * agroups));
    splits = std::min(splits, std::min(c->splits, a.nchunks));
    a.chunks_per_split = (a.nchunks + splits - 1) / splits;
    splits = (a.nchunks + a.chunks_per_split - 1) / a.chunks_per_split;
    srht_fused_kernel<<<smp::counted(dim3((unsigned)tiles, (unsigned)splits, (unsigned)agroups)), SR_THREADS, 0,
                        c->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace smp
