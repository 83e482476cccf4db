// Tensor-core sketch engine with FP8 E4M3 operands derived from BF16 row blocks (Algorithm 1, step 2; Section 2.1
// "Step 1"): At += s_A Pi8 A8 / sqrt(k) and Bt += s_B Pi8 B8 / sqrt(k), where A8 = e4m3(A_blk / s_A) with one
// power-of-two scale s_A = 2^ceil(log2(amax|A_blk| / 448)) per row block (likewise for B) and Pi8 = e4m3 of the
// N(0, 1) Philox normals; kind::f8f6f4 products accumulate in FP32 in TMEM. The column norms are those of the
// stored BF16 values (compensated sums), so Omega does not see the quantisation.
//
// Per block: amax_kernel reduces |A_blk|, |B_blk| and writes the two scales; sketch_fp8_kernel then runs one CTA per
// (128-column tile, row split, half of the sketch rows). Warp 0 loads BF16 data tiles (64-column x 8-row boxes,
// 128-byte swizzle) into a staging ring, warp 2 the Pi8 tiles (K-major, 64-byte rows, 64-byte swizzle) into a Pi
// ring; eight conversion warps read each staged element once (two columns per 32-bit word), fold the squares into
// packed compensated sums, scale, convert pairs to E4M3 (cvt.rn.satfinite.e4m3x2) and write the tile MN-major
// (128-column x 8-row atoms, 128-byte swizzle; layout found with a probe) into an operand ring; warp 1 (one thread)
// issues tcgen05.mma kind::f8f6f4 with M = 128 data columns, N = 256 sketch rows, K = 32 rows per instruction. The
// drain multiplies the accumulator by s / sqrt(k). Every wait is bounded (%globaltimer).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace smp {
namespace {
using namespace tc;

constexpr int TILE_M = 128;          // data columns per CTA (MMA M)
constexpr int KS = 64;               // data rows per pipeline stage (two K = 32 MMA slices)
constexpr int MMA_N = 256;           // sketch rows per instruction
constexpr int KC_CTA = 512;          // sketch rows per CTA (TMEM columns)
constexpr int MAX_K = 1024;
constexpr int BOX_COLS = 64;         // bf16 columns per staged box (128 B)
constexpr int BOX_BYTES = BOX_COLS * 8 * 2;
constexpr int KGROUP_BYTES = (TILE_M / BOX_COLS) * BOX_BYTES;   // one 8-row group of both boxes (bf16)
constexpr int DATA_STAGE_BYTES = (KS / 8) * KGROUP_BYTES;       // 128 columns x 64 rows of bf16
constexpr int ATOM_BYTES = TILE_M * 8;                          // e4m3 operand: 128 columns x 8 rows per atom
constexpr int A_STAGE_BYTES = (KS / 8) * ATOM_BYTES;            // 128 columns x 64 rows of e4m3
constexpr int PI_BOX_BYTES = MMA_N * KS;                        // 256 sketch rows x 64 e4m3
constexpr int PI_STAGE_BYTES = (KC_CTA / MMA_N) * PI_BOX_BYTES;
#ifndef SMP_FP8_DSTAGES
#define SMP_FP8_DSTAGES 4
#endif
#ifndef SMP_FP8_ASTAGES
#define SMP_FP8_ASTAGES 3
#endif
#ifndef SMP_FP8_PSTAGES
#define SMP_FP8_PSTAGES 4
#endif
constexpr int DSTAGES = SMP_FP8_DSTAGES;   // staged BF16 data tiles
constexpr int ASTAGES = SMP_FP8_ASTAGES;   // E4M3 operand tiles
constexpr int PSTAGES = SMP_FP8_PSTAGES;   // Pi tiles
constexpr int DRING_BYTES = DSTAGES * DATA_STAGE_BYTES;
constexpr int ARING_BYTES = ASTAGES * A_STAGE_BYTES;
constexpr int PRING_BYTES = PSTAGES * PI_STAGE_BYTES;
constexpr int BAR_BYTES = 8 * (2 * (DSTAGES + ASTAGES + PSTAGES) + 1) + 8;   // mbarriers, TMEM address, abort flag
constexpr int SMEM_BYTES = DRING_BYTES + ARING_BYTES + PRING_BYTES + 1024 /* alignment */ + BAR_BYTES;
static_assert(SMEM_BYTES <= 232448, "shared memory budget");
constexpr int THREADS = 512;         // 16 warps: producers 0 and 2, MMA 1, conversion warps on schedulers 0, 2, 3
constexpr int NCONV = 8;
// conversion warp c handles box c % 2 (64 columns) and the 8-row groups 2 (c / 2), 2 (c / 2) + 1 of every stage;
// the warps sit on schedulers 0, 2, 3, leaving scheduler 1 to the MMA issuer
__device__ __forceinline__ int conv_index(int warp) {
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

// Power-of-two block scale: s = 2^ceil(log2(amax / 448)) (1 for an all-zero block), so |x / s| <= 448; the exponent
// is kept at or above -126 so that 1 / s stays finite.
__device__ __forceinline__ float pow2_scale(float amax) {
    if (!(amax > 0.f)) return 1.f;
    int e;
    const float m = frexpf(amax / 448.f, &e);   // amax / 448 = m 2^e, m in [0.5, 1)
    return ldexpf(1.f, max(-126, m == 0.5f ? e - 1 : e));
}

__device__ __forceinline__ float bf16_abs_max2(uint32_t w, float m) {
    return fmaxf(m, fmaxf(fabsf(__uint_as_float(w << 16)), fabsf(__uint_as_float(w & 0xFFFF0000u))));
}

// scale[0] = s_A, scale[1] = s_B of this row block (max over |x| in binary32, exact for BF16 inputs). Rows are
// 16-byte aligned (ld % 8 == 0): warp w of matrix blockIdx.y reads rows w, w + (warps in the grid), ..., eight
// values per 16-byte load and four loads in flight per lane.
__global__ void __launch_bounds__(256) amax_kernel(const __nv_bfloat16* __restrict__ A, int64_t lda, int64_t n1,
                                                   const __nv_bfloat16* __restrict__ B, int64_t ldb, int64_t n2,
                                                   int64_t nrows, unsigned* amax_bits, float* scale, int* done) {
    const int which = blockIdx.y;   // 0: A, 1: B
    const __nv_bfloat16* X = which ? B : A;
    const int64_t ld = which ? ldb : lda, n = which ? n2 : n1;
    const int lane = threadIdx.x & 31;
    float m = 0.f;
    if (X != nullptr && n > 0) {
        const int64_t n8 = n / 8;
        const int tail = (int)(n - 8 * n8);
        const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
        for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nrows; r += nw) {
            const __nv_bfloat16* row = X + r * ld;
            const uint4* row16 = (const uint4*)row;
            int64_t j = lane;
            for (; j + 96 < n8; j += 128) {
                const uint4 w0 = __ldg(row16 + j), w1 = __ldg(row16 + j + 32), w2 = __ldg(row16 + j + 64),
                            w3 = __ldg(row16 + j + 96);
                m = bf16_abs_max2(w0.x, bf16_abs_max2(w0.y, bf16_abs_max2(w0.z, bf16_abs_max2(w0.w, m))));
                m = bf16_abs_max2(w1.x, bf16_abs_max2(w1.y, bf16_abs_max2(w1.z, bf16_abs_max2(w1.w, m))));
                m = bf16_abs_max2(w2.x, bf16_abs_max2(w2.y, bf16_abs_max2(w2.z, bf16_abs_max2(w2.w, m))));
                m = bf16_abs_max2(w3.x, bf16_abs_max2(w3.y, bf16_abs_max2(w3.z, bf16_abs_max2(w3.w, m))));
            }
            for (; j < n8; j += 32) {
                const uint4 w = __ldg(row16 + j);
                m = bf16_abs_max2(w.x, bf16_abs_max2(w.y, bf16_abs_max2(w.z, bf16_abs_max2(w.w, m))));
            }
            if (lane < tail) m = fmaxf(m, fabsf(__bfloat162float(row[8 * n8 + lane])));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&amax_bits[which], __float_as_uint(m));   // non-negative floats order like their bits
        __threadfence();
    }
    __syncthreads();
    // the last CTA to finish turns the maxima into scales (and resets the counters for the next block)
    if (threadIdx.x == 0) {
        __threadfence();
        const int total_ctas = gridDim.x * gridDim.y;
        if (atomicAdd(done, 1) == total_ctas - 1) {
            __threadfence();
            const float a0 = __uint_as_float(atomicExch(&amax_bits[0], 0u));
            const float a1 = __uint_as_float(atomicExch(&amax_bits[1], 0u));
            scale[0] = pow2_scale(a0);
            scale[1] = pow2_scale(a1);
            *done = 0;
        }
    }
}

struct Fp8Args {
    int64_t n1, n2, ntot;
    int tiles_a;
    int k, kmma;
    uint32_t tmem_cols;
    int64_t nrows;
    int64_t steps;          // KS-row stages of the block (split s takes stages s, s + splits, ...)
    int64_t ldk;
    float* part;
    double* nsq;
    const float* scale;      // [2]: s_A, s_B of this block
    float pi_scale;          // 1 / sqrt(k) for generated Pi, 1 for a caller's
    int* err;
};

__global__ void __launch_bounds__(THREADS, 1) sketch_fp8_kernel(const __grid_constant__ CUtensorMap tm_a,
                                                                const __grid_constant__ CUtensorMap tm_b,
                                                                const __grid_constant__ CUtensorMap tm_pi,
                                                                const Fp8Args args) {
    extern __shared__ uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int split = blockIdx.y;
    const int kh = blockIdx.z;
    // row splits interleaved by pipeline stage (stage it of split s: rows (it * splits + s) * KS ..), so all CTAs
    // stream rows from one narrow window of the block (better DRAM locality than contiguous splits)
    const int splits = (int)gridDim.y;
    const int n_it = split < args.steps ? (int)((args.steps - split + splits - 1) / splits) : 0;
    const int n_cta = min(KC_CTA, args.kmma - kh * KC_CTA);
    if (n_it <= 0 || n_cta <= 0) return;
    const int nh = (n_cta + MMA_N - 1) / MMA_N;
    const int n_last = n_cta - (nh - 1) * MMA_N;
    const int kc_cta = min(KC_CTA, (args.k + 31) / 32 * 32 - kh * KC_CTA);

    const int tile = blockIdx.x;
    const bool on_b = tile >= args.tiles_a;
    const int64_t col0 = on_b ? (int64_t)(tile - args.tiles_a) * TILE_M : (int64_t)tile * TILE_M;
    const int64_t ncols_src = on_b ? args.n2 : args.n1;
    const int valid = (int)(ncols_src - col0 < TILE_M ? ncols_src - col0 : TILE_M);
    const int64_t cbase = on_b ? args.n1 + col0 : col0;
    const CUtensorMap* tm_data = on_b ? &tm_b : &tm_a;
    const float s_blk = args.scale[on_b ? 1 : 0];
    const float inv_s = 1.f / s_blk;   // a power of two: exact

    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* base_ptr = smem_raw + (base - raw);
    const uint32_t dring = base;
    const uint32_t aring = base + DRING_BYTES;
    const uint32_t pring = aring + ARING_BYTES;
    const uint32_t bar_base = pring + PRING_BYTES;
    uint64_t* bars = (uint64_t*)(base_ptr + DRING_BYTES + ARING_BYTES + PRING_BYTES);
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * (DSTAGES + ASTAGES + PSTAGES) + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    auto dfull_bar = [&](int d) { return bar_base + 8u * d; };
    auto dempty_bar = [&](int d) { return bar_base + 8u * (DSTAGES + d); };
    auto afull_bar = [&](int s) { return bar_base + 8u * (2 * DSTAGES + s); };
    auto aempty_bar = [&](int s) { return bar_base + 8u * (2 * DSTAGES + ASTAGES + s); };
    auto pfull_bar = [&](int s) { return bar_base + 8u * (2 * DSTAGES + 2 * ASTAGES + s); };
    auto pempty_bar = [&](int s) { return bar_base + 8u * (2 * DSTAGES + 2 * ASTAGES + PSTAGES + s); };
    const uint32_t acc_bar = bar_base + 8u * (2 * DSTAGES + 2 * ASTAGES + 2 * PSTAGES);
    uint64_t hi2 = 0ull, lo2 = 0ull;   // conversion warps: compensated sums of squares of their two columns

    if (threadIdx.x == 0) {
        for (int d = 0; d < DSTAGES; ++d) {
            mbar_init(dfull_bar(d), 1);
            mbar_init(dempty_bar(d), NCONV);
        }
        for (int s = 0; s < ASTAGES; ++s) {
            mbar_init(afull_bar(s), NCONV);
            mbar_init(aempty_bar(s), 1);
        }
        for (int s = 0; s < PSTAGES; ++s) {
            mbar_init(pfull_bar(s), 1);
            mbar_init(pempty_bar(s), 1);
        }
        mbar_init(acc_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_addr(tmem_slot), args.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- data producer: BF16 tiles into the staging ring (lane 0 issues)
        if (lane == 0) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)tm_data) : "memory");
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
                    for (int b = 0; b < TILE_M / BOX_COLS; ++b)
                        tma_load_2d(dst + g * KGROUP_BYTES + b * BOX_BYTES, tm_data, (int)col0 + BOX_COLS * b,
                                    t + 8 * g, dfull_bar(d));
            }
            issued = it + 1;
            __syncwarp();
        }
        // the CTA may not finish while a load it issued is still landing (even after an abort)
        for (int it = max(0, issued - DSTAGES); it < issued; ++it)
            mbar_wait_landed(dfull_bar(it % DSTAGES), (uint32_t)(it / DSTAGES) & 1u, WAIT_NS);
    } else if (warp == 2) {
        // ---------------- Pi producer: E4M3 tiles of this CTA's sketch rows
        if (lane == 0) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_pi) : "memory");
        const uint32_t bytes = nh * PI_BOX_BYTES;
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
                    tma_load_2d(pring + s * PI_STAGE_BYTES + h * PI_BOX_BYTES, &tm_pi, t, kh * KC_CTA + h * MMA_N,
                                pfull_bar(s));
            }
            issued = it + 1;
            __syncwarp();
        }
        for (int it = max(0, issued - PSTAGES); it < issued; ++it)
            mbar_wait_landed(pfull_bar(it % PSTAGES), (uint32_t)(it / PSTAGES) & 1u, WAIT_NS);
    } else if (warp == 1) {
        // ---------------- MMA issuer (the whole warp waits; lane 0 issues)
        const uint32_t id_full = idesc_e4m3(TILE_M, MMA_N, true);
        const uint32_t id_last = idesc_e4m3(TILE_M, n_last, true);
        bool ok = true;
        for (int it = 0; it < n_it; ++it) {
            const int sa = it % ASTAGES, sp = it % PSTAGES;
            const uint32_t aph = (uint32_t)(it / ASTAGES) & 1u, pph = (uint32_t)(it / PSTAGES) & 1u;
            ok = __all_sync(0xffffffffu,
                            mbar_wait(pfull_bar(sp), pph, abort_flag) && mbar_wait(afull_bar(sa), aph, abort_flag));
            if (!ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    set_error(args.err, DEVERR_TIMEOUT | (1 << 9));
                }
                break;
            }
            tc_fence_after();
            if (lane == 0) {
                const uint32_t abase = aring + sa * A_STAGE_BYTES, pbase = pring + sp * PI_STAGE_BYTES;
#pragma unroll
                for (int kk = 0; kk < KS / 32; ++kk) {
                    // A (data) MN-major, 128B swizzle, one 128-column atom per 8-row group (SBO 1 KB), the next 32
                    // rows four groups on; B (Pi) K-major, 64-byte rows, 64B swizzle, the next 32 rows at +32 B
                    const uint64_t ad = smem_desc(abase + kk * 4 * ATOM_BYTES, ATOM_BYTES, ATOM_BYTES, SWZ_128B);
                    for (int h = 0; h < nh; ++h) {
                        const uint64_t bd = smem_desc(pbase + h * PI_BOX_BYTES + kk * 32, 16, 512, SWZ_64B);
                        mma_e4m3(tmem + h * MMA_N, ad, bd, h == nh - 1 ? id_last : id_full,
                                 (it > 0 || kk > 0) ? 1u : 0u);
                    }
                }
                mma_commit(aempty_bar(sa));
                mma_commit(pempty_bar(sp));
            }
            __syncwarp();
        }
        if (ok && lane == 0) mma_commit(acc_bar);
        __syncwarp();
    } else if (conv_index(warp) >= 0) {
        // ---------------- conversion warps: lane l holds columns 2l, 2l + 1 of its box, one 32-bit word per row
        const int ci = conv_index(warp);
        const int box = ci & 1, g0 = 2 * (ci >> 1);
        const bool do_norms = kh == 0;
        const int mcol = box * BOX_COLS + 2 * lane;   // first of the lane's two columns within the tile
        for (int it = 0; it < n_it; ++it) {
            const int d = it % DSTAGES, s = it % ASTAGES;
            const uint32_t dph = (uint32_t)(it / DSTAGES) & 1u, aph = (uint32_t)(it / ASTAGES) & 1u;
            bool ok = mbar_wait(dfull_bar(d), dph, abort_flag);
            if (ok && it >= ASTAGES) ok = mbar_wait(aempty_bar(s), aph ^ 1u, abort_flag);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    set_error(args.err, DEVERR_TIMEOUT | (1 << 10));
                }
                break;
            }
            const uint8_t* stage = base_ptr + d * DATA_STAGE_BYTES + box * BOX_BYTES;
            uint8_t* atoms = base_ptr + DRING_BYTES + s * A_STAGE_BYTES;
            uint32_t w[16];
#pragma unroll
            for (int gg = 0; gg < 2; ++gg)
#pragma unroll
                for (int t = 0; t < 8; ++t)   // staged bf16 box: 16-byte chunk c of row t at c ^ (t & 7)
                    w[gg * 8 + t] = *(const uint32_t*)(stage + (g0 + gg) * KGROUP_BYTES + t * 128 +
                                                      (((lane >> 2) ^ t) << 4) + ((lane & 3) << 2));
            __syncwarp();
            if (lane == 0) mbar_arrive(dempty_bar(d));
#pragma unroll
            for (int gg = 0; gg < 2; ++gg) {
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float x0 = __uint_as_float(w[gg * 8 + t] << 16);
                    const float x1 = __uint_as_float(w[gg * 8 + t] & 0xFFFF0000u);
                    if (do_norms) two_sum_square_x2(pack2(x0, x1), hi2, lo2);
                    uint16_t q;
                    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(q) : "f"(x1 * inv_s), "f"(x0 * inv_s));
                    // e4m3 atom row t of group g0 + gg: 16-byte chunk c at c ^ (t & 7)
                    *(uint16_t*)(atoms + (g0 + gg) * ATOM_BYTES + t * 128 + (((mcol >> 4) ^ t) << 4) + (mcol & 15)) =
                        q;
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(afull_bar(s));
        }
    }
    __syncthreads();   // every role has left its loop
    const bool acc_ok = __all_sync(0xffffffffu, !*abort_flag && mbar_wait(acc_bar, 0, abort_flag));
    tc_fence_after();
    // every MMA has completed and the staging ring is drained: norm hand-off through it
    double* nsum = (double*)base_ptr;   // [group quarter][128 columns]
    if (conv_index(warp) >= 0) {
        const int ci = conv_index(warp);
        float h0, h1, l0, l1;
        unpack2(hi2, h0, h1);
        unpack2(lo2, l0, l1);
        const int m = (ci & 1) * BOX_COLS + 2 * lane;
        nsum[(ci >> 1) * TILE_M + m] = (double)h0 + (double)l0;
        nsum[(ci >> 1) * TILE_M + m + 1] = (double)h1 + (double)l1;
    }
    __syncthreads();
    {
        // ---------------- TMEM drain by all 16 warps, scaled by s / sqrt(k)
        const int q = warp & 3;
        const int m = q * 32 + lane;
        const int cq = ((kc_cta / 32 + 3) / 4) * 32;
        const int cbeg = (warp >> 2) * cq, cend = min(kc_cta, cbeg + cq);
        const float sc = s_blk * args.pi_scale;
        if (acc_ok) {
            const int64_t c = cbase + m;
            float* dst = args.part + ((int64_t)split * args.ntot + c) * args.ldk + kh * KC_CTA;
            const int kmax = args.k - kh * KC_CTA;
            for (int cc = cbeg; cc < cend; cc += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)cc, v);
                if (m < valid) {
                    if (args.ldk % 4 == 0) {
#pragma unroll
                        for (int i = 0; i < 32; i += 4)
                            if (kh * KC_CTA + cc + i < args.ldk) {
                                float4* p4 = (float4*)(dst + cc + i);
                                float4 o = *p4;
                                o.x = fmaf(v[i], sc, o.x);
                                o.y = fmaf(v[i + 1], sc, o.y);
                                o.z = fmaf(v[i + 2], sc, o.z);
                                o.w = fmaf(v[i + 3], sc, o.w);
                                *p4 = o;
                            }
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (cc + i < kmax) dst[cc + i] = fmaf(v[i], sc, dst[cc + i]);
                    }
                }
            }
            if (kh == 0 && warp < 4 && m < valid)
                args.nsq[(int64_t)split * args.ntot + c] +=
                    (nsum[m] + nsum[TILE_M + m]) + (nsum[2 * TILE_M + m] + nsum[3 * TILE_M + m]);
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
        tmem_dealloc(tmem, args.tmem_cols);
    }
}

bool aligned_bf16(const void* p, int64_t ld) { return ((uintptr_t)p % 16 == 0) && (ld % 8 == 0); }

}  // namespace

bool fp8_block_ok(const smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb) {
    return c->p.dtype == SMP_BF16 && c->p.k <= MAX_K && encode_fn() != nullptr && aligned_bf16(A, lda) &&
           (c->p.same_ab || aligned_bf16(B, ldb));
}

cudaError_t launch_sketch_fp8(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                              int64_t nrows, const float* Pi, int64_t ldp) {
    static std::atomic<bool> attr{false};
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(sketch_fp8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaStream_t st = c->stream;
    if (!c->fp8_ws) {   // [0, 8): amax bits of A, B; [8, 16): scales; [16, 20): completion counter
        cudaError_t e = dev_malloc(&c->fp8_ws, 32, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->fp8_ws, 0, 32, st);
        if (e != cudaSuccess) return e;
    }
    unsigned* amax_bits = (unsigned*)c->fp8_ws;
    float* scale = (float*)((char*)c->fp8_ws + 8);
    int* done = (int*)((char*)c->fp8_ws + 16);
    const int64_t n2 = c->p.same_ab ? 0 : c->p.n2;
    amax_kernel<<<smp::counted(dim3((unsigned)std::max(1, 4 * c->sm_count), 2u)), 256, 0, st>>>(
        (const __nv_bfloat16*)A, lda, c->p.n1, (const __nv_bfloat16*)(c->p.same_ab ? nullptr : B), ldb, n2, nrows,
        amax_bits, scale, done);
    const int k = c->p.k;
    const int kmma = (int)round_up(k, 16);
    const int khalves = (kmma + KC_CTA - 1) / KC_CTA;
    const int64_t tpad = round_up(nrows, KS);
    int buf = -1;
    cudaError_t e = Pi ? pi_import(c, Pi, ldp, nrows, &buf) : pi_acquire(c, row0, nrows, &buf);
    if (e != cudaSuccess) return e;
    const PiGeom gm = pi_geom(c);
    CUtensorMap ma, mb, mp;
    const void* Bp = c->p.same_ab ? A : B;
    if (!make_map(&ma, A, (uint64_t)c->p.n1, (uint64_t)nrows, (uint64_t)lda, BOX_COLS, 8, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2) ||
        !make_map(&mb, Bp, (uint64_t)(c->p.same_ab ? c->p.n1 : c->p.n2), (uint64_t)nrows,
                  (uint64_t)(c->p.same_ab ? lda : ldb), BOX_COLS, 8, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2) ||
        !make_map(&mp, c->pi_buf[buf], (uint64_t)tpad, (uint64_t)gm.kpad, (uint64_t)gm.ld, KS, MMA_N,
                  CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1))
        return cudaErrorInvalidValue;
    Fp8Args a;
    a.n1 = c->p.n1;
    a.n2 = n2;
    a.ntot = c->ntot;
    a.tiles_a = (int)((c->p.n1 + TILE_M - 1) / TILE_M);
    const int tiles = a.tiles_a + (int)((n2 + TILE_M - 1) / TILE_M);
    a.k = k;
    a.kmma = kmma;
    const int kc = (int)std::min<int64_t>(KC_CTA, round_up(k, 32));
    uint32_t cols = 32;
    while ((int)cols < kc) cols <<= 1;
    a.tmem_cols = cols;
    a.nrows = nrows;
    const int64_t steps = tpad / KS;
    int splits = std::max(1, std::min(c->splits, c->sm_count / std::max(1, tiles * khalves)));
    splits = (int)std::min<int64_t>(splits, steps);
    a.steps = steps;
    a.ldk = c->ldk;
    a.part = (float*)c->part;
    a.nsq = c->nsq;
    a.scale = scale;
    a.pi_scale = Pi ? 1.f : (float)(1.0 / std::sqrt((double)k));
    a.err = c->dev_err;
    sketch_fp8_kernel<<<smp::counted(dim3((unsigned)tiles, (unsigned)splits, (unsigned)khalves)), THREADS,
                        SMEM_BYTES, st>>>(ma, mb, mp, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (Pi) {
        c->pi_last = buf;
        return cudaEventRecord(c->pi_free[buf], st);
    }
    return pi_release(c, buf, row0, nrows);
}

}  // namespace smp
