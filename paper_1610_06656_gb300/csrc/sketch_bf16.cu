// Tensor-core sketch engine for BF16 inputs (Algorithm 1, step 2; Section 2.1 "Step 1"): At += Pi[:, rows] A_blk
// and Bt += Pi[:, rows] B_blk with BF16 operands (kind::f16) and FP32 accumulation in TMEM, fused with the
// compensated column sums of squares of the stored BF16 values, so each element of A and B is read from HBM once.
//
// kind::f16 reads 16-bit operands MN-major, so the data tile lands from TMA straight into its operand slot (rows of
// A are contiguous along the columns: 64-column x 8-row boxes, 128-byte swizzle) and no copy pass is needed; Pi
// (rounded to BF16 by the generator) is the K-major operand. One CTA per (128-column tile, row split, half of the
// sketch rows): TMEM holds 512 FP32 columns, so k > 512 splits the sketch rows over two CTAs that read the same data
// tile (through L2). Warp 0 loads the data tiles into an 8-slot ring, warp 2 the Pi tiles into a 4-slot ring,
// warp 1 (one thread) issues tcgen05.mma with M = 128 data columns, N = 256 sketch rows, K = 16 rows per
// instruction; four norm warps read each staged tile once (bf16 pairs, squares exact in binary32) into packed
// compensated sums. A data slot is free when the MMA's commit and the four norm warps have arrived. All eight
// warps then drain TMEM into the split's partial sketch. Every wait is bounded (%globaltimer); a timeout sets the
// device error word and the CTA unwinds.
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
constexpr int KS = 32;               // data rows per pipeline stage (two K = 16 MMA slices)
constexpr int MMA_N = 256;           // sketch rows per instruction
constexpr int KC_CTA = 512;          // sketch rows per CTA (TMEM columns)
constexpr int MAX_K = 1024;          // two sketch-row halves
constexpr int BOX_COLS = 64;         // bf16 columns per data box (128 B)
#ifndef SMP_BF16_BOX_ROWS
#define SMP_BF16_BOX_ROWS 32
#endif
constexpr int BOX_ROWS = SMP_BF16_BOX_ROWS;   // rows per data box: 8 ([8-row group][box]) or KS ([box][row])
static_assert(BOX_ROWS == 8 || BOX_ROWS == KS, "data box rows");
constexpr int BOX_BYTES = BOX_COLS * BOX_ROWS * 2;
constexpr int KGROUP_BYTES = (TILE_M / BOX_COLS) * BOX_COLS * 8 * 2;   // one 8-row group of both 64-column boxes
constexpr int DATA_STAGE_BYTES = (KS / 8) * KGROUP_BYTES;              // 128 columns x 32 rows
// byte offset, within a stage, of 8-row group g of 64-column box b (the MN-major atom the MMA reads)
__device__ __forceinline__ constexpr int grp_off(int g, int b) {
    return BOX_ROWS == 8 ? g * KGROUP_BYTES + b * BOX_COLS * 8 * 2 : b * BOX_BYTES + g * BOX_COLS * 8 * 2;
}
constexpr uint32_t A_LBO = BOX_ROWS == 8 ? BOX_COLS * 8 * 2 : BOX_BYTES;   // between 64-column atoms
constexpr uint32_t A_SBO = BOX_ROWS == 8 ? KGROUP_BYTES : BOX_COLS * 8 * 2;   // between 8-row groups
constexpr int PI_BOX_BYTES = MMA_N * KS * 2;                 // 256 sketch rows x 32 bf16 (64-byte rows)
constexpr int PI_STAGE_BYTES = (KC_CTA / MMA_N) * PI_BOX_BYTES;
#ifndef SMP_BF16_DSTAGES
#define SMP_BF16_DSTAGES 8
#endif
#ifndef SMP_BF16_PSTAGES
#define SMP_BF16_PSTAGES 4
#endif
constexpr int DSTAGES = SMP_BF16_DSTAGES;   // data tiles (the MMA's A operand)
constexpr int PSTAGES = SMP_BF16_PSTAGES;   // Pi tiles
constexpr int DRING_BYTES = DSTAGES * DATA_STAGE_BYTES;
constexpr int PRING_BYTES = PSTAGES * PI_STAGE_BYTES;
constexpr int BAR_BYTES = 8 * (2 * (DSTAGES + PSTAGES) + 1) + 8;   // mbarriers, TMEM address, abort flag
constexpr int SMEM_BYTES = DRING_BYTES + PRING_BYTES + 1024 /* alignment */ + BAR_BYTES;
static_assert(SMEM_BYTES <= 232448, "shared memory budget");
constexpr int THREADS = 256;         // 8 warps: data producer 0, MMA 1, Pi producer 2, norm warps 3, 4, 6, 7
constexpr int NNORM = 4;
__device__ __forceinline__ int norm_index(int warp) {
    switch (warp) {
        case 3: return 0;
        case 4: return 1;
        case 6: return 2;
        case 7: return 3;
        default: return -1;
    }
}

struct Bf16Args {
    int64_t n1, n2, ntot;
    int tiles_a;
    int k, kmma;             // sketch rows, rows covered by MMA N (multiple of 16)
    uint32_t tmem_cols;
    int64_t nrows;
    int64_t steps;          // KS-row stages of the block (split s takes stages s, s + splits, ...)
    int64_t ldk;
    float* part;             // [splits][ntot][ldk]
    double* nsq;             // [splits][ntot]
    int* err;
};

__global__ void __launch_bounds__(THREADS, 1) sketch_bf16_kernel(const __grid_constant__ CUtensorMap tm_a,
                                                                 const __grid_constant__ CUtensorMap tm_b,
                                                                 const __grid_constant__ CUtensorMap tm_pi,
                                                                 const Bf16Args args) {
    extern __shared__ uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int split = blockIdx.y;
    const int kh = blockIdx.z;   // half of the sketch rows
    // row splits interleaved by pipeline stage (stage it of split s: rows (it * splits + s) * KS ..), so all CTAs
    // stream rows from one narrow window of the block (better DRAM locality than contiguous splits)
    const int splits = (int)gridDim.y;
    const int n_it = split < args.steps ? (int)((args.steps - split + splits - 1) / splits) : 0;
    const int n_cta = min(KC_CTA, args.kmma - kh * KC_CTA);   // MMA N rows of this CTA (multiple of 16)
    if (n_it <= 0 || n_cta <= 0) return;
    const int nh = (n_cta + MMA_N - 1) / MMA_N;
    const int n_last = n_cta - (nh - 1) * MMA_N;
    const int kc_cta = min(KC_CTA, (args.k + 31) / 32 * 32 - kh * KC_CTA);   // drained columns

    const int tile = blockIdx.x;
    const bool on_b = tile >= args.tiles_a;
    const int64_t col0 = on_b ? (int64_t)(tile - args.tiles_a) * TILE_M : (int64_t)tile * TILE_M;
    const int64_t ncols_src = on_b ? args.n2 : args.n1;
    const int valid = (int)(ncols_src - col0 < TILE_M ? ncols_src - col0 : TILE_M);
    const int64_t cbase = on_b ? args.n1 + col0 : col0;
    const CUtensorMap* tm_data = on_b ? &tm_b : &tm_a;

    // carve shared memory (1024-byte aligned): data ring, Pi ring, barriers
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* base_ptr = smem_raw + (base - raw);
    const uint32_t dring = base;
    const uint32_t pring = base + DRING_BYTES;
    const uint32_t bar_base = pring + PRING_BYTES;
    uint64_t* bars = (uint64_t*)(base_ptr + DRING_BYTES + PRING_BYTES);
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * (DSTAGES + PSTAGES) + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    auto dfull_bar = [&](int d) { return bar_base + 8u * d; };
    auto dempty_bar = [&](int d) { return bar_base + 8u * (DSTAGES + d); };
    auto pfull_bar = [&](int s) { return bar_base + 8u * (2 * DSTAGES + s); };
    auto pempty_bar = [&](int s) { return bar_base + 8u * (2 * DSTAGES + PSTAGES + s); };
    const uint32_t acc_bar = bar_base + 8u * (2 * DSTAGES + 2 * PSTAGES);
    // norm warps: compensated sums of squares of their two columns (the two lanes of packed f32x2 registers)
    uint64_t hi2 = 0ull, lo2 = 0ull;

    if (threadIdx.x == 0) {
        for (int d = 0; d < DSTAGES; ++d) {
            mbar_init(dfull_bar(d), 1);
            mbar_init(dempty_bar(d), 1 + NNORM);   // the MMA commit and the norm warps
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
        // ---------------- data producer (lane 0 issues)
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
                for (int g = 0; g < KS / BOX_ROWS; ++g)
#pragma unroll
                    for (int b = 0; b < TILE_M / BOX_COLS; ++b)
                        tma_load_2d(dst + grp_off(g * (BOX_ROWS / 8), b), tm_data, (int)col0 + BOX_COLS * b,
                                    t + BOX_ROWS * g, dfull_bar(d));
            }
            issued = it + 1;
            __syncwarp();
        }
        // the CTA may not finish while a load it issued is still landing (even after an abort)
        for (int it = max(0, issued - DSTAGES); it < issued; ++it)
            mbar_wait_landed(dfull_bar(it % DSTAGES), (uint32_t)(it / DSTAGES) & 1u, WAIT_NS);
    } else if (warp == 2) {
        // ---------------- Pi producer: this CTA's sketch rows kh * 512 ...
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
                    tma_load_2d(pring + s * PI_STAGE_BYTES + h * PI_BOX_BYTES, &tm_pi, t,
                                kh * KC_CTA + h * MMA_N, pfull_bar(s));
            }
            issued = it + 1;
            __syncwarp();
        }
        for (int it = max(0, issued - PSTAGES); it < issued; ++it)
            mbar_wait_landed(pfull_bar(it % PSTAGES), (uint32_t)(it / PSTAGES) & 1u, WAIT_NS);
    } else if (warp == 1) {
        // ---------------- MMA issuer (the whole warp waits; lane 0 issues)
        const uint32_t id_full = idesc_bf16(TILE_M, MMA_N, true);
        const uint32_t id_last = idesc_bf16(TILE_M, n_last, true);
        bool ok = true;
        for (int it = 0; it < n_it; ++it) {
            const int sd = it % DSTAGES, sp = it % PSTAGES;
            const uint32_t dph = (uint32_t)(it / DSTAGES) & 1u, pph = (uint32_t)(it / PSTAGES) & 1u;
            ok = __all_sync(0xffffffffu,
                            mbar_wait(pfull_bar(sp), pph, abort_flag) && mbar_wait(dfull_bar(sd), dph, abort_flag));
            if (!ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    set_error(args.err, DEVERR_TIMEOUT | (1 << 9));
                }
                break;
            }
            tc_fence_after();
            if (lane == 0) {
                const uint32_t dbase = dring + sd * DATA_STAGE_BYTES, pbase = pring + sp * PI_STAGE_BYTES;
#pragma unroll
                for (int kk = 0; kk < KS / 16; ++kk) {
                    // A (data) MN-major, 128B swizzle: 64-column atoms 1 KB apart (LBO), 8-row groups 2 KB apart
                    // (SBO), the next 16 rows two groups on; B (Pi) K-major, 64B swizzle, the next 16 rows at +32 B
                    const uint64_t ad = smem_desc(dbase + grp_off(2 * kk, 0), A_LBO, A_SBO, SWZ_128B);
                    for (int h = 0; h < nh; ++h) {
                        const uint64_t bd = smem_desc(pbase + h * PI_BOX_BYTES + kk * 32, 16, 512, SWZ_64B);
                        mma_bf16(tmem + h * MMA_N, ad, bd, h == nh - 1 ? id_last : id_full,
                                 (it > 0 || kk > 0) ? 1u : 0u);
                    }
                }
                mma_commit(dempty_bar(sd));
                mma_commit(pempty_bar(sp));
            }
            __syncwarp();
        }
        if (ok && lane == 0) mma_commit(acc_bar);
        __syncwarp();
    } else if (norm_index(warp) >= 0) {
        // ---------------- norm warps: box ni % 2 (64 columns), 8-row groups 2 (ni / 2), 2 (ni / 2) + 1 of every
        // stage; lane l reads columns 2l, 2l + 1 of each row (one 4-byte word, conflict-free under the swizzle)
        const int ni = norm_index(warp);
        const int box = ni & 1, g0 = 2 * (ni >> 1);
        const bool do_norms = kh == 0;   // the other sketch-row half reads the same data
        for (int it = 0; it < n_it; ++it) {
            const int d = it % DSTAGES;
            const uint32_t ph = (uint32_t)(it / DSTAGES) & 1u;
            const bool ok = __all_sync(0xffffffffu, mbar_wait(dfull_bar(d), ph, abort_flag));
            if (!ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    set_error(args.err, DEVERR_TIMEOUT | (1 << 10));
                }
                break;
            }
            if (do_norms) {
                const uint8_t* stage = base_ptr + d * DATA_STAGE_BYTES;
#pragma unroll
                for (int gg = 0; gg < 2; ++gg) {
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        // 128B swizzle: the 16-byte chunk c of box row t sits at chunk c ^ (t & 7)
                        const uint32_t wv = *(const uint32_t*)(stage + grp_off(g0 + gg, box) + t * 128 +
                                                               (((lane >> 2) ^ t) << 4) + ((lane & 3) << 2));
                        two_sum_square_x2(pack2(__uint_as_float(wv << 16), __uint_as_float(wv & 0xFFFF0000u)),
                                          hi2, lo2);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(dempty_bar(d));
        }
    }
    __syncthreads();   // every role has left its loop
    const bool acc_ok = __all_sync(0xffffffffu, !*abort_flag && mbar_wait(acc_bar, 0, abort_flag));
    tc_fence_after();
    // every MMA has completed: the data ring is free for the norm hand-off
    double* nsum = (double*)base_ptr;   // [group half][128 columns]
    if (norm_index(warp) >= 0) {
        const int ni = norm_index(warp);
        float h0, h1, l0, l1;
        unpack2(hi2, h0, h1);
        unpack2(lo2, l0, l1);
        const int m = (ni & 1) * BOX_COLS + 2 * lane;
        nsum[(ni >> 1) * TILE_M + m] = (double)h0 + (double)l0;
        nsum[(ni >> 1) * TILE_M + m + 1] = (double)h1 + (double)l1;
    }
    __syncthreads();
    {
        // ---------------- TMEM drain by the 8 warps: warp w reads TMEM lanes 32 (w % 4) ... and half w / 4 of the
        // accumulator columns, and adds them into the split's partial sketch (sketch rows kh * 512 ...)
        const int q = warp & 3;
        const int m = q * 32 + lane;
        const int half = ((kc_cta / 32 + 1) / 2) * 32;
        const int cbeg = (warp >> 2) * half, cend = min(kc_cta, cbeg + half);
        if (acc_ok) {
            const int64_t c = cbase + m;
            float* dst = args.part + ((int64_t)split * args.ntot + c) * args.ldk + kh * KC_CTA;
            const int kmax = args.k - kh * KC_CTA;   // valid sketch rows of this half
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
                                o.x += v[i];
                                o.y += v[i + 1];
                                o.z += v[i + 2];
                                o.w += v[i + 3];
                                *p4 = o;
                            }
                    } else {
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            if (cc + i < kmax) dst[cc + i] += v[i];
                    }
                }
            }
            if (kh == 0 && warp < 4 && m < valid)
                args.nsq[(int64_t)split * args.ntot + c] += nsum[m] + nsum[TILE_M + m];
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

bool bf16_tc_supported(const smp_ctx* c) {
    return c->p.dtype == SMP_BF16 && c->p.k <= MAX_K && encode_fn() != nullptr;
}

bool bf16_block_ok(const smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb) {
    return bf16_tc_supported(c) && aligned_bf16(A, lda) && (c->p.same_ab || aligned_bf16(B, ldb));
}

cudaError_t launch_sketch_bf16(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                               int64_t nrows, const float* Pi, int64_t ldp) {
    static std::atomic<bool> attr{false};
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(sketch_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int k = c->p.k;
    const int kmma = (int)round_up(k, 16);
    const int khalves = (kmma + KC_CTA - 1) / KC_CTA;
    const int64_t tpad = round_up(nrows, KS);
    cudaStream_t st = c->stream;
    int buf = -1;
    cudaError_t e = Pi ? pi_import(c, Pi, ldp, nrows, &buf) : pi_acquire(c, row0, nrows, &buf);
    if (e != cudaSuccess) return e;
    const PiGeom gm = pi_geom(c);
    CUtensorMap ma, mb, mp;
    const void* Bp = c->p.same_ab ? A : B;
    const int64_t n2 = c->p.same_ab ? 0 : c->p.n2;
    // data boxes: 64 bf16 columns (128 B) x 8 rows, matching the kernel's expect_tx; Pi boxes: 32 x 256
    if (!make_map(&ma, A, (uint64_t)c->p.n1, (uint64_t)nrows, (uint64_t)lda, BOX_COLS, BOX_ROWS,
                  CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2) ||
        !make_map(&mb, Bp, (uint64_t)(c->p.same_ab ? c->p.n1 : c->p.n2), (uint64_t)nrows,
                  (uint64_t)(c->p.same_ab ? lda : ldb), BOX_COLS, BOX_ROWS, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2) ||
        !make_map(&mp, c->pi_buf[buf], (uint64_t)tpad, (uint64_t)gm.kpad, (uint64_t)gm.ld, KS, MMA_N,
                  CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2))
        return cudaErrorInvalidValue;
    Bf16Args a;
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
    a.err = c->dev_err;
    sketch_bf16_kernel<<<smp::counted(dim3((unsigned)tiles, (unsigned)splits, (unsigned)khalves)), THREADS,
                         SMEM_BYTES, st>>>(ma, mb, mp, a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (Pi) {   // a caller's Pi: the buffer only becomes free again, nothing is generated ahead
        c->pi_last = buf;
        return cudaEventRecord(c->pi_free[buf], st);
    }
    return pi_release(c, buf, row0, nrows);
}

}  // namespace smp
