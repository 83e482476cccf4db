// LELA, the two-pass method SMP-PCA is compared with (Section 1; Section 4, Table 1 and Fig. 5(a)): pass 1 reads
// the data for the column norms alone, pass 2 reads it again for the exact entries M_ij = A_i^T B_j of A^T B on
// the sampled set Omega; WAltMin then runs on those entries instead of SMP-PCA's estimates.
//
// Pass 1 (norms_kernel): compensated column sums of squares into the context's row-split partials, the same fold
// and the same partials as the sketch engines, so smp_sketch_finalize closes it unchanged.
//
// Pass 2 on tensor cores (exact_tc_kernel; SMP_F32 row blocks, 16-byte aligned): the block of A is first written
// transposed and rounded to TF32 (cvt.rna) into a K-major buffer A^T (n1 rows of the block's data rows). A CTA owns
// 128 columns j of B, up to 512 columns i of A and a range of data rows. It forms the dense 128 x 512 tile of
// B^T A in TMEM with tcgen05.mma kind::tf32: B's tile comes through TMA into a staging ring and copy warps write
// its K-major TF32 copy; A^T's boxes come through TMA straight from the transposed buffer. The epilogue keeps only
// the entries of Omega in the tile: TMEM lane j walks its column's CSC entries (rows i increasing) and adds the
// value into the entry's binary64 partial of this row split. The rest of the tile is dropped: at the default
// budget m = 4 n r ln n, Omega holds 4 r ln n / n of A^T B (15% at n = 2,000, r = 10), and the dense tensor-core
// tile still costs several times less than gathering column pairs entry by entry on the CUDA cores.
//
// Pass 2 elsewhere (exact_simt_kernel; binary64, BF16, unaligned blocks): a CTA owns a 32 x 32 tile of (i, j),
// stages 32-row chunks of both column sets in shared memory and each lane sums one Omega entry of its column.
//
// Entry partials are [EXACT_SPLITS][nnz] in CSC order, one writer per (split, entry) per launch; smp_exact_values
// sums the splits in a fixed order (bitwise reproducible) and scatters the result to CSR order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace smp {
namespace {

using namespace tc;

// ------------------------------------------------------------------------------------------------ pass 1: norms
// Compensated x^2 accumulation (the product's error from an FMA, the sum's from TwoSum), binary32 or binary64.
__device__ __forceinline__ void sq_add(float x, float& hi, float& lo) {
    const float p = __fmul_rn(x, x);
    const float e = __fmaf_rn(x, x, -p);
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}
__device__ __forceinline__ void sq_add(double x, double& hi, double& lo) {
    const double p = __dmul_rn(x, x);
    const double e = __fma_rn(x, x, -p);
    const double s = __dadd_rn(hi, p);
    const double bp = __dsub_rn(s, hi);
    const double err = __dadd_rn(__dsub_rn(hi, __dsub_rn(s, bp)), __dsub_rn(p, bp));
    hi = s;
    lo = __dadd_rn(lo, __dadd_rn(err, e));
}
__device__ __forceinline__ float load_as(const float* p, float) { return __ldcs(p); }
__device__ __forceinline__ float load_as(const __nv_bfloat16* p, float) { return __bfloat162float(*p); }
__device__ __forceinline__ double load_as(const double* p, double) { return __ldcs(p); }

// Four consecutive elements (16 bytes of binary32, 8 of BF16, 32 of binary64) when the group is aligned and whole.
__device__ __forceinline__ void load4(const float* p, float (&x)[4]) {
    const float4 v = __ldcs((const float4*)p);
    x[0] = v.x, x[1] = v.y, x[2] = v.z, x[3] = v.w;
}
__device__ __forceinline__ void load4(const __nv_bfloat16* p, float (&x)[4]) {
    const uint2 v = __ldcs((const uint2*)p);
    x[0] = __uint_as_float(v.x << 16), x[1] = __uint_as_float(v.x & 0xFFFF0000u);
    x[2] = __uint_as_float(v.y << 16), x[3] = __uint_as_float(v.y & 0xFFFF0000u);
}
__device__ __forceinline__ void load4(const double* p, double (&x)[4]) {
    const double2 a = __ldcs((const double2*)p), b = __ldcs((const double2*)p + 1);
    x[0] = a.x, x[1] = a.y, x[2] = b.x, x[3] = b.y;
}

constexpr int NRM_COLS = 128;    // columns per CTA: lane l of every warp owns columns 4 l .. 4 l + 3
constexpr int NRM_WARPS = 8;     // warp w reads rows rs + w, rs + w + 8, ...
constexpr int NRM_UNROLL = 8;    // rows in flight per thread

// Column tiles cover A's columns, then B's (a tile never straddles the two). vec: every four-column group that
// lies inside its matrix starts on an element-vector boundary (aligned base, ld a multiple of 4).
template <typename TIn, typename TAcc>
__global__ void __launch_bounds__(256) norms_kernel(const TIn* __restrict__ A, int64_t lda, const TIn* __restrict__ B,
                                                    int64_t ldb, int64_t n1, int64_t n2, int tiles_a, int64_t nrows,
                                                    int64_t rows_per_split, int64_t ntot, bool vec,
                                                    double* __restrict__ nsq) {
    __shared__ double red[NRM_WARPS][NRM_COLS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool on_b = (int)blockIdx.x >= tiles_a;
    const int64_t c0 = (int64_t)(on_b ? blockIdx.x - tiles_a : blockIdx.x) * NRM_COLS + 4 * lane;
    const int64_t n = on_b ? n2 : n1;
    const TIn* src = (on_b ? B : A) + c0;
    const int64_t ld = on_b ? ldb : lda;
    const int split = blockIdx.y;
    const int64_t rs = (int64_t)split * rows_per_split, re = min(nrows, rs + rows_per_split);
    const int nv = (int)max((int64_t)0, min((int64_t)4, n - c0));   // valid columns of this lane's group
    TAcc hi[4] = {TAcc(0), TAcc(0), TAcc(0), TAcc(0)}, lo[4] = {TAcc(0), TAcc(0), TAcc(0), TAcc(0)};
    if (nv == 4 && vec) {
        int64_t t = rs + warp;
        for (; t + (NRM_UNROLL - 1) * NRM_WARPS < re; t += NRM_UNROLL * NRM_WARPS) {
            TAcc x[NRM_UNROLL][4];
#pragma unroll
            for (int u = 0; u < NRM_UNROLL; ++u) load4(src + (t + u * NRM_WARPS) * ld, x[u]);
#pragma unroll
            for (int u = 0; u < NRM_UNROLL; ++u)
#pragma unroll
                for (int q = 0; q < 4; ++q) sq_add(x[u][q], hi[q], lo[q]);
        }
        for (; t < re; t += NRM_WARPS) {
            TAcc x[4];
            load4(src + t * ld, x);
#pragma unroll
            for (int q = 0; q < 4; ++q) sq_add(x[q], hi[q], lo[q]);
        }
    } else if (nv > 0) {
        for (int64_t t = rs + warp; t < re; t += NRM_WARPS)
            for (int q = 0; q < nv; ++q) sq_add(load_as(src + t * ld + q, TAcc(0)), hi[q], lo[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) red[warp][4 * lane + q] = (double)hi[q] + (double)lo[q];
    __syncthreads();
    if (threadIdx.x < NRM_COLS) {
        const int cl = threadIdx.x;
        const int64_t col = (int64_t)(on_b ? blockIdx.x - tiles_a : blockIdx.x) * NRM_COLS + cl;
        if (col < n) {
            double v = red[0][cl];
#pragma unroll
            for (int w = 1; w < NRM_WARPS; ++w) v += red[w][cl];
            nsq[(int64_t)split * ntot + (on_b ? n1 + col : col)] += v;
        }
    }
}

template <typename TIn, typename TAcc>
cudaError_t launch_norms_typed(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t nrows) {
    const bool same = c->p.same_ab;
    const int64_t n1 = c->p.n1, n2 = same ? 0 : c->p.n2;
    const int tiles_a = (int)((n1 + NRM_COLS - 1) / NRM_COLS);
    const int tiles = tiles_a + (int)((n2 + NRM_COLS - 1) / NRM_COLS);
    const size_t vbytes = 4 * sizeof(TIn);
    auto aligned = [&](const void* p, int64_t ld) { return (uintptr_t)p % vbytes == 0 && ld % 4 == 0; };
    const bool vec = aligned(A, lda) && (same || aligned(B, ldb));
    // row splits: about two CTAs per SM, at most the context's partial buffers, at least 64 rows each
    int splits = (int)std::max<int64_t>(1, (2 * (int64_t)c->sm_count + tiles - 1) / tiles);
    splits = (int)std::min<int64_t>(std::min(splits, c->splits), std::max<int64_t>(1, nrows / 64));
    const int64_t rps = (nrows + splits - 1) / splits;
    splits = (int)((nrows + rps - 1) / rps);
    norms_kernel<TIn, TAcc><<<smp::counted(dim3((unsigned)tiles, (unsigned)splits)), 256, 0, c->stream>>>(
        (const TIn*)A, lda, same ? (const TIn*)A : (const TIn*)B, same ? lda : ldb, n1, n2, tiles_a, nrows, rps,
        c->ntot, vec, c->nsq);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------ pass 2: SIMT
constexpr int SX_T = 32;   // (i, j) tile side and rows per staged chunk

template <typename TIn, typename TAcc>
__global__ void __launch_bounds__(256) exact_simt_kernel(const TIn* __restrict__ A, int64_t lda,
                                                         const TIn* __restrict__ B, int64_t ldb, int64_t n1,
                                                         int64_t n2, int64_t nrows,
                                                         const int64_t* __restrict__ col_ptr,
                                                         const int32_t* __restrict__ csc_row,
                                                         double* __restrict__ part) {
    __shared__ TAcc as[SX_T][SX_T + 1];   // [row][i - i0]
    __shared__ TAcc bs[SX_T][SX_T + 1];   // [row][j - j0]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t j0 = (int64_t)blockIdx.x * SX_T, i0 = (int64_t)blockIdx.y * SX_T;
    // warp w: columns j0 + 4 w + u (u < 4); lane: the lane-th Omega entry of that column with i in [i0, i0 + 32)
    int64_t pe[4];
    int ie[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t j = j0 + 4 * warp + u;
        pe[u] = -1;
        ie[u] = 0;
        if (j < n2) {
            int64_t lo = col_ptr[j], hi = col_ptr[j + 1];
            while (lo < hi) {   // first entry with row >= i0
                const int64_t mid = (lo + hi) >> 1;
                if (csc_row[mid] < i0) lo = mid + 1;
                else hi = mid;
            }
            const int64_t p = lo + lane;
            if (p < col_ptr[j + 1] && csc_row[p] < i0 + SX_T) {
                pe[u] = p;
                ie[u] = (int)(csc_row[p] - i0);
            }
        }
    }
    TAcc acc[4] = {TAcc(0), TAcc(0), TAcc(0), TAcc(0)};
    for (int64_t t0 = 0; t0 < nrows; t0 += SX_T) {
#pragma unroll
        for (int e = 0; e < (SX_T * SX_T) / 256; ++e) {
            const int idx = tid + 256 * e, r = idx / SX_T, cc = idx % SX_T;
            const int64_t t = t0 + r;
            as[r][cc] = (t < nrows && i0 + cc < n1) ? load_as(A + t * lda + i0 + cc, TAcc(0)) : TAcc(0);
            bs[r][cc] = (t < nrows && j0 + cc < n2) ? load_as(B + t * ldb + j0 + cc, TAcc(0)) : TAcc(0);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int jl = 4 * warp + u;
#pragma unroll 8
            for (int r = 0; r < SX_T; ++r) acc[u] = fma(as[r][ie[u]], bs[r][jl], acc[u]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (pe[u] >= 0) part[pe[u]] += (double)acc[u];
}

template <typename TIn, typename TAcc>
cudaError_t launch_exact_simt_typed(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb,
                                    int64_t nrows) {
    const int64_t n1 = c->p.n1, n2 = c->p.same_ab ? c->p.n1 : c->p.n2;
    const dim3 g((unsigned)((n2 + SX_T - 1) / SX_T), (unsigned)((n1 + SX_T - 1) / SX_T));
    exact_simt_kernel<TIn, TAcc><<<smp::counted(g), 256, 0, c->stream>>>(
        (const TIn*)A, lda, c->p.same_ab ? (const TIn*)A : (const TIn*)B, c->p.same_ab ? lda : ldb, n1, n2, nrows,
        c->col_ptr, c->csc_row, c->ex_part);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------ pass 2: tcgen05
constexpr int TILE_M = 128;        // columns j of B per CTA (MMA M, TMEM lanes)
constexpr int KS = 16;             // data rows per pipeline stage (two K = 8 MMA slices)
constexpr int PSTAGES = 4, ASTAGES = 4, DSTAGES = 8;
constexpr int AT_BOX_ROWS = 256;   // columns i of A per A^T box (MMA N)
constexpr int MAX_NI = 512;        // columns i of A per CTA (TMEM columns)
constexpr int DATA_BOX_ROWS = 8;
constexpr int DATA_BOX_BYTES = 32 * DATA_BOX_ROWS * 4;      // 32 columns x 8 rows, fp32 (one 128B swizzle atom)
constexpr int DATA_STAGE_BYTES = 4 * KS * 32 * 4;           // 128 columns x KS rows: [8-row group][32-col box]
constexpr int KGROUP_BYTES = 4 * DATA_BOX_BYTES;
constexpr int C_STAGE_BYTES = TILE_M * KS * 4;              // K-major copy of B's tile: 128 rows x 64 B
constexpr int AT_BOX_BYTES = AT_BOX_ROWS * KS * 4;          // 256 rows x KS fp32
constexpr int AT_STAGE_BYTES = (MAX_NI / AT_BOX_ROWS) * AT_BOX_BYTES;
constexpr int DRING_BYTES = DSTAGES * DATA_STAGE_BYTES;
constexpr int CRING_BYTES = ASTAGES * C_STAGE_BYTES;
constexpr int PRING_BYTES = PSTAGES * AT_STAGE_BYTES;
constexpr int BAR_BYTES = 8 * (2 * (DSTAGES + ASTAGES + PSTAGES) + 1) + 8;
constexpr int SMEM_BYTES = DRING_BYTES + CRING_BYTES + PRING_BYTES + 1024 /* alignment */ + BAR_BYTES;
static_assert(SMEM_BYTES <= 232448, "shared memory budget");
constexpr int THREADS = 512;       // 16 warps: producers 0 and 2, MMA 1, copy warps on schedulers 0, 2, 3
constexpr int NCOPY = 8;
constexpr int SCRATCH_LD = 33;     // epilogue: per-warp 32 x 33 floats of one TMEM column chunk
static_assert(16 * 32 * SCRATCH_LD * 4 <= DRING_BYTES + CRING_BYTES, "epilogue scratch fits the free rings");

__device__ __forceinline__ int copy_index(int warp) {
    switch (warp) {
        case 4: return 0;
        case 6: return 1;
        case 7: return 2;
        case 8: return 3;
        case 10: return 4;
        case 11: return 5;
        case 12: return 6;
        case 14: return 7;
        default: return -1;
    }
}

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return __uint_as_float(y);
}

// A^T[i][t] = tf32(A[t][i]) for t < nrows, i < n1 (32 x 32 tiles through shared memory: both sides coalesced).
__global__ void __launch_bounds__(256) transpose_tf32_kernel(const float* __restrict__ A, int64_t lda, int64_t n1,
                                                             int64_t nrows, float* __restrict__ at, int64_t ldt) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * 32, t0 = (int64_t)blockIdx.y * 32;
#pragma unroll
    for (int r = ty; r < 32; r += 8) {
        const int64_t t = t0 + r, i = i0 + tx;
        tile[r][tx] = (t < nrows && i < n1) ? __ldcs(A + t * lda + i) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = i0 + r, t = t0 + tx;
        if (i < n1 && t < nrows) at[i * ldt + t] = to_tf32(tile[tx][r]);
    }
}

struct ExactArgs {
    int64_t n1, n2;                 // columns i of A, columns j of B
    int64_t nrows;
    int64_t steps;          // KS-row stages of the block (split s takes stages s, s + splits, ...)
    const int64_t* col_ptr;         // CSC of Omega
    const int32_t* csc_row;
    double* part;                   // [splits][ld], CSC order
    int64_t ld;
    int* err;
};

__global__ void __launch_bounds__(THREADS, 1) exact_tc_kernel(const __grid_constant__ CUtensorMap tm_b,
                                                              const __grid_constant__ CUtensorMap tm_at,
                                                              const ExactArgs args) {
    extern __shared__ uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int split = blockIdx.y;
    // row splits interleaved by pipeline stage (stage it of split s: rows (it * splits + s) * KS ..), so all CTAs
    // stream rows from one narrow window of the block (better DRAM locality than contiguous splits)
    const int splits = (int)gridDim.y;
    const int n_it = split < args.steps ? (int)((args.steps - split + splits - 1) / splits) : 0;
    if (n_it <= 0) return;
    const int64_t j0 = (int64_t)blockIdx.x * TILE_M;
    const int64_t i0 = (int64_t)blockIdx.z * MAX_NI;
    const int ni = (int)min((int64_t)MAX_NI, args.n1 - i0);      // columns i of this CTA
    const int kmma = (ni + 15) & ~15;                             // MMA N coverage (multiple of 16)
    const int nh = (kmma + AT_BOX_ROWS - 1) / AT_BOX_ROWS;
    const int n_last = kmma - (nh - 1) * AT_BOX_ROWS;
    const int kc = (ni + 31) & ~31;                               // TMEM columns drained

    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* base_ptr = smem_raw + (base - raw);
    const uint32_t dring = base;
    const uint32_t cring = base + DRING_BYTES;
    const uint32_t pring = cring + CRING_BYTES;
    const uint32_t bar_base = pring + PRING_BYTES;
    uint64_t* bars = (uint64_t*)(base_ptr + DRING_BYTES + CRING_BYTES + PRING_BYTES);
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * (DSTAGES + ASTAGES + PSTAGES) + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    auto dfull_bar = [&](int d) { return bar_base + 8u * d; };
    auto dempty_bar = [&](int d) { return bar_base + 8u * (DSTAGES + d); };
    auto cfull_bar = [&](int s) { return bar_base + 8u * (2 * DSTAGES + s); };
    auto cempty_bar = [&](int s) { return bar_base + 8u * (2 * DSTAGES + ASTAGES + s); };
    auto pfull_bar = [&](int s) { return bar_base + 8u * (2 * DSTAGES + 2 * ASTAGES + s); };
    auto pempty_bar = [&](int s) { return bar_base + 8u * (2 * DSTAGES + 2 * ASTAGES + PSTAGES + s); };
    const uint32_t acc_bar = bar_base + 8u * (2 * DSTAGES + 2 * ASTAGES + 2 * PSTAGES);

    if (threadIdx.x == 0) {
        for (int d = 0; d < DSTAGES; ++d) {
            mbar_init(dfull_bar(d), 1);
            mbar_init(dempty_bar(d), NCOPY);
        }
        for (int s = 0; s < ASTAGES; ++s) {
            mbar_init(cfull_bar(s), NCOPY);
            mbar_init(cempty_bar(s), 1);
        }
        for (int s = 0; s < PSTAGES; ++s) {
            mbar_init(pfull_bar(s), 1);
            mbar_init(pempty_bar(s), 1);
        }
        mbar_init(acc_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_addr(tmem_slot), MAX_NI);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- B producer: 128 columns x KS rows of B per stage into the staging ring
        if (lane == 0) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_b) : "memory");
        int issued = 0;
        for (int it = 0; it < n_it; ++it) {
            const int d = it % DSTAGES;
            const uint32_t ph = (uint32_t)(it / DSTAGES) & 1u;
            bool ok = true;
            if (it >= DSTAGES) ok = __all_sync(0xffffffffu, mbar_wait(dempty_bar(d), ph ^ 1u, abort_flag));
            if (!ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    set_error(args.err, DEVERR_TIMEOUT | (1 << 8));
                }
                break;
            }
            if (lane == 0) {
                mbar_arrive_expect_tx(dfull_bar(d), DATA_STAGE_BYTES);
                const int t = (int)(((int64_t)it * splits + split) * KS);
                const uint32_t dst = dring + d * DATA_STAGE_BYTES;
#pragma unroll
                for (int g = 0; g < KS / 8; ++g)
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        tma_load_2d(dst + g * KGROUP_BYTES + b * DATA_BOX_BYTES, &tm_b, (int)j0 + 32 * b, t + 8 * g,
                                    dfull_bar(d));
            }
            issued = it + 1;
            __syncwarp();
        }
        // the CTA may not finish while a load it issued is still landing (even after an abort)
        for (int it = max(0, issued - DSTAGES); it < issued; ++it)
            mbar_wait_landed(dfull_bar(it % DSTAGES), (uint32_t)(it / DSTAGES) & 1u, WAIT_NS);
    } else if (warp == 2) {
        // ---------------- A^T producer: nh boxes of 256 columns i x KS rows per stage
        if (lane == 0) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_at) : "memory");
        const uint32_t bytes = nh * AT_BOX_BYTES;
        int issued = 0;
        for (int it = 0; it < n_it; ++it) {
            const int s = it % PSTAGES;
            const uint32_t ph = (uint32_t)(it / PSTAGES) & 1u;
            bool ok = true;
            if (it >= PSTAGES) ok = __all_sync(0xffffffffu, mbar_wait(pempty_bar(s), ph ^ 1u, abort_flag));
            if (!ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    set_error(args.err, DEVERR_TIMEOUT | (1 << 12));
                }
                break;
            }
            if (lane == 0) {
                mbar_arrive_expect_tx(pfull_bar(s), bytes);
                const int t = (int)(((int64_t)it * splits + split) * KS);
                for (int h = 0; h < nh; ++h)
                    tma_load_2d(pring + s * AT_STAGE_BYTES + h * AT_BOX_BYTES, &tm_at, t,
                                (int)i0 + h * AT_BOX_ROWS, pfull_bar(s));
            }
            issued = it + 1;
            __syncwarp();
        }
        for (int it = max(0, issued - PSTAGES); it < issued; ++it)
            mbar_wait_landed(pfull_bar(it % PSTAGES), (uint32_t)(it / PSTAGES) & 1u, WAIT_NS);
    } else if (warp == 1) {
        // ---------------- MMA issuer: D[j][i] += sum_t B[t][j] A[t][i] (lane 0 issues)
        const uint32_t id_full = idesc_tf32(TILE_M, AT_BOX_ROWS);
        const uint32_t id_last = idesc_tf32(TILE_M, n_last);
        bool ok = true;
        for (int it = 0; it < n_it; ++it) {
            const int sp = it % PSTAGES, sa = it % ASTAGES;
            const uint32_t pph = (uint32_t)(it / PSTAGES) & 1u, aph = (uint32_t)(it / ASTAGES) & 1u;
            ok = __all_sync(0xffffffffu,
                            mbar_wait(pfull_bar(sp), pph, abort_flag) && mbar_wait(cfull_bar(sa), aph, abort_flag));
            if (!ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    set_error(args.err, DEVERR_TIMEOUT | (1 << 9));
                }
                break;
            }
            tc_fence_after();
            if (lane == 0) {
                const uint32_t abase = cring + sa * C_STAGE_BYTES, pbase = pring + sp * AT_STAGE_BYTES;
#pragma unroll
                for (int kb = 0; kb < KS / 8; ++kb) {
                    // both operands K-major, 64B swizzle: rows of 64 B, 8-row groups 512 B apart, K slice at +32 B
                    const uint64_t ad = smem_desc(abase + kb * 32, 16, 512, SWZ_64B);
                    for (int h = 0; h < nh; ++h) {
                        const uint64_t bd = smem_desc(pbase + h * AT_BOX_BYTES + kb * 32, 16, 512, SWZ_64B);
                        mma_tf32(tmem + h * AT_BOX_ROWS, ad, bd, h == nh - 1 ? id_last : id_full,
                                 (it > 0 || kb > 0) ? 1u : 0u);
                    }
                }
                mma_commit(cempty_bar(sa));
                mma_commit(pempty_bar(sp));
            }
            __syncwarp();
        }
        if (ok && lane == 0) mma_commit(acc_bar);
        __syncwarp();
    } else if (copy_index(warp) >= 0) {
        // ---------------- copy warps: one (32-column box, 8-row group) of the stage each, K-major TF32 copy
        const int ci = copy_index(warp);
        const int box = ci & 3, grp = ci >> 2;
        const int m = box * 32 + lane;
        for (int it = 0; it < n_it; ++it) {
            const int d = it % DSTAGES;
            const uint32_t dph = (uint32_t)(it / DSTAGES) & 1u;
            const int s = it % ASTAGES;
            const uint32_t ph = (uint32_t)(it / ASTAGES) & 1u;
            bool ok = mbar_wait(dfull_bar(d), dph, abort_flag);
            if (ok && it >= ASTAGES) ok = mbar_wait(cempty_bar(s), ph ^ 1u, abort_flag);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    set_error(args.err, DEVERR_TIMEOUT | (1 << 10));
                }
                break;
            }
            // staged box: 128B swizzle, the 16-byte chunk q of row t sits at chunk q ^ (t & 7)
            const float* box_p =
                (const float*)(base_ptr + d * DATA_STAGE_BYTES + grp * KGROUP_BYTES + box * DATA_BOX_BYTES);
            float x[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) x[t] = box_p[t * 32 + (((lane >> 2) ^ t) << 2) + (lane & 3)];
            __syncwarp();
            if (lane == 0) mbar_arrive(dempty_bar(d));
            // K-major copy: column m of the tile is row m (64 B = KS values); chunk q at q ^ ((m >> 1) & 3)
            float4* crow = (float4*)(base_ptr + DRING_BYTES + s * C_STAGE_BYTES + m * (KS * 4));
            const int q0 = 2 * grp;
            crow[q0 ^ ((m >> 1) & 3)] = make_float4(to_tf32(x[0]), to_tf32(x[1]), to_tf32(x[2]), to_tf32(x[3]));
            crow[(q0 + 1) ^ ((m >> 1) & 3)] = make_float4(to_tf32(x[4]), to_tf32(x[5]), to_tf32(x[6]), to_tf32(x[7]));
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(cfull_bar(s));
        }
    }
    __syncthreads();   // every role has left its loop: the staging and copy rings are free
    {
        // ---------------- sampled epilogue by all 16 warps: warp w owns TMEM lanes 32 (w % 4) ... (columns j) and
        // the column quarter w / 4 of the accumulator (columns i); lane j adds the Omega entries of its column whose
        // row i falls in that quarter
        const int q = warp & 3;
        const int m = q * 32 + lane;
        const int64_t j = j0 + m;
        const int cq = ((kc / 32 + 3) / 4) * 32;
        const int cbeg = (warp >> 2) * cq, cend = min(kc, cbeg + cq);
        float* scratch = (float*)base_ptr + warp * 32 * SCRATCH_LD;
        const bool acc_ok = __all_sync(0xffffffffu, !*abort_flag && mbar_wait(acc_bar, 0, abort_flag));
        if (acc_ok) {
            tc_fence_after();
            int64_t p = 0, pend = 0;
            if (j < args.n2 && cbeg < cend) {
                int64_t lo = args.col_ptr[j], hi = args.col_ptr[j + 1];
                pend = hi;
                const int64_t first = i0 + cbeg;
                while (lo < hi) {   // first entry of column j with row i >= i0 + cbeg
                    const int64_t mid = (lo + hi) >> 1;
                    if (args.csc_row[mid] < first) lo = mid + 1;
                    else hi = mid;
                }
                p = lo;
            }
            int inext = p < pend ? args.csc_row[p] : INT32_MAX;
            double* dst = args.part + (int64_t)split * args.ld;
            for (int cc = cbeg; cc < cend; cc += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)cc, v);
#pragma unroll
                for (int e = 0; e < 32; ++e) scratch[lane * SCRATCH_LD + e] = v[e];
                __syncwarp();
                const int64_t cut = i0 + cc + 32;
                while (inext < cut) {
                    dst[p] += (double)scratch[lane * SCRATCH_LD + (int)(inext - (i0 + cc))];
                    ++p;
                    inext = p < pend ? args.csc_row[p] : INT32_MAX;
                }
                __syncwarp();
            }
        } else if (lane == 0) {
            *abort_flag = 1;
            set_error(args.err, DEVERR_TIMEOUT | (1 << 11));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, MAX_NI);
    }
}

int64_t round_up_i64(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

// ------------------------------------------------------------------------------------------------ host side
cudaError_t launch_norms(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t nrows) {
    switch (c->p.dtype) {
        case SMP_F32: return launch_norms_typed<float, float>(c, A, lda, B, ldb, nrows);
        case SMP_BF16: return launch_norms_typed<__nv_bfloat16, float>(c, A, lda, B, ldb, nrows);
        default: return launch_norms_typed<double, double>(c, A, lda, B, ldb, nrows);
    }
}

bool exact_tc_ok(const smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb) {
    auto al = [](const void* p, int64_t ld) { return (uintptr_t)p % 16 == 0 && ld % 4 == 0; };
    return c->p.dtype == SMP_F32 && encode_fn() != nullptr && al(A, lda) && (c->p.same_ab || al(B, ldb));
}

cudaError_t exact_prepare(smp_ctx* c) {
    if (c->ex_ready) return cudaSuccess;
    const int64_t want = std::max<int64_t>(c->nnz, 1);
    if (want > c->ex_cap) {
        free_after(c->ex_part, c->stream);
        c->ex_part = nullptr;
        c->ex_cap = 0;
        const int64_t cap = want + want / 8 + 1024;
        cudaError_t e = dev_malloc((void**)&c->ex_part, (size_t)EXACT_SPLITS * cap * 8, c->stream);
        if (e != cudaSuccess) return e;
        c->ex_cap = cap;
    }
    cudaError_t e = cudaMemsetAsync(c->ex_part, 0, (size_t)EXACT_SPLITS * c->ex_cap * 8, c->stream);
    if (e == cudaSuccess) c->ex_ready = true;
    return e;
}

cudaError_t launch_exact(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t nrows,
                         bool tensor_cores) {
    cudaError_t e = exact_prepare(c);
    if (e != cudaSuccess || c->nnz == 0) return e;
    if (!tensor_cores) {
        switch (c->p.dtype) {
            case SMP_F32: return launch_exact_simt_typed<float, float>(c, A, lda, B, ldb, nrows);
            case SMP_BF16: return launch_exact_simt_typed<__nv_bfloat16, float>(c, A, lda, B, ldb, nrows);
            default: return launch_exact_simt_typed<double, double>(c, A, lda, B, ldb, nrows);
        }
    }
    static std::atomic<bool> attr{false};
    if (!attr) {
        e = cudaFuncSetAttribute(exact_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t n1 = c->p.n1, n2 = c->p.same_ab ? c->p.n1 : c->p.n2;
    // A^T of the block, TF32-rounded, rows of ldt floats (a multiple of 4: TMA strides are multiples of 16 bytes)
    const int64_t ldt = round_up_i64(c->max_rows, 4);
    const size_t at_bytes = (size_t)n1 * ldt * 4;
    if (c->ex_at_bytes < at_bytes) {
        free_after(c->ex_at, c->stream);
        c->ex_at = nullptr;
        c->ex_at_bytes = 0;
        if ((e = dev_malloc((void**)&c->ex_at, at_bytes, c->stream)) != cudaSuccess) return e;
        c->ex_at_bytes = at_bytes;
    }
    transpose_tf32_kernel<<<smp::counted(dim3((unsigned)((n1 + 31) / 32), (unsigned)((nrows + 31) / 32))), 256, 0,
                            c->stream>>>((const float*)A, lda, n1, nrows, c->ex_at, ldt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    CUtensorMap mb, mat;
    const void* Bp = c->p.same_ab ? A : B;
    const int64_t ldb_ = c->p.same_ab ? lda : ldb;
    // B boxes: 32 columns (128 B, one swizzle row) x 8 rows; A^T boxes: KS rows (64 B) x 256 columns i
    if (!make_map(&mb, Bp, (uint64_t)n2, (uint64_t)nrows, (uint64_t)ldb_, 32, DATA_BOX_ROWS,
                  CU_TENSOR_MAP_SWIZZLE_128B) ||
        !make_map(&mat, c->ex_at, (uint64_t)nrows, (uint64_t)n1, (uint64_t)ldt, KS, AT_BOX_ROWS,
                  CU_TENSOR_MAP_SWIZZLE_64B))
        return cudaErrorInvalidValue;
    ExactArgs a;
    a.n1 = n1;
    a.n2 = n2;
    a.nrows = nrows;
    a.col_ptr = c->col_ptr;
    a.csc_row = c->csc_row;
    a.part = c->ex_part;
    a.ld = c->ex_cap;
    a.err = c->dev_err;
    const int tiles = (int)((n2 + TILE_M - 1) / TILE_M);
    const int chunks = (int)((n1 + MAX_NI - 1) / MAX_NI);
    const int64_t steps = (nrows + KS - 1) / KS;
    int splits = std::max(1, std::min(EXACT_SPLITS, c->sm_count / std::max(1, tiles * chunks)));
    splits = (int)std::min<int64_t>(splits, steps);
    a.steps = steps;
    exact_tc_kernel<<<smp::counted(dim3((unsigned)tiles, (unsigned)splits, (unsigned)chunks)), THREADS, SMEM_BYTES,
                      c->stream>>>(mb, mat, a);
    return cudaGetLastError();
}

namespace {
template <typename TOut>
__global__ void exact_values_kernel(const double* __restrict__ part, int64_t cap, int64_t nnz,
                                    const int64_t* __restrict__ csc_pos, TOut* __restrict__ vals) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nnz) return;
    double v = part[p];
#pragma unroll
    for (int s = 1; s < EXACT_SPLITS; ++s) v += part[(int64_t)s * cap + p];
    vals[csc_pos[p]] = (TOut)v;
}
}  // namespace

cudaError_t launch_exact_values(smp_ctx* c, void* vals) {
    cudaError_t e = exact_prepare(c);
    if (e != cudaSuccess || c->nnz == 0) return e;
    const unsigned blocks = (unsigned)((c->nnz + 255) / 256);
    if (c->p.dtype == SMP_F64)
        exact_values_kernel<double><<<smp::counted(blocks), 256, 0, c->stream>>>(c->ex_part, c->ex_cap, c->nnz,
                                                                                c->csc_pos, (double*)vals);
    else
        exact_values_kernel<float><<<smp::counted(blocks), 256, 0, c->stream>>>(c->ex_part, c->ex_cap, c->nnz,
                                                                               c->csc_pos, (float*)vals);
    return cudaGetLastError();
}

}  // namespace smp
