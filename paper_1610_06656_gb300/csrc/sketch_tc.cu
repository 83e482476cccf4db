// Tensor-core sketch engine for sm_103a (Algorithm 1, step 2; Section 2.1 "Step 1"): At += Pi[:, rows] A_blk and
// Bt += Pi[:, rows] B_blk with TF32 operands and FP32 accumulation in TMEM, fused with the compensated column sums
// of squares, so each element of A and B is read from HBM once.
//
// Two kernels per row block:
//  1. pi_gen_kernel writes Pi[a][t] (t contiguous, rounded to TF32) for the block's rows into a context buffer.
//     Generating Pi once per block and letting every column tile read it (through L2) costs one Gaussian per
//     (sketch row, data row); regenerating it inside each column tile would cost (n1 + n2) / 128 times more.
//  2. sketch_tc_kernel: one CTA per (128-column tile, row split; the splits interleaved by pipeline stage). Warp 0
//     issues one TMA load per stage of the data tile (rows of A are contiguous along the columns, so the tile lands
//     column-major: one 128-column x KS-row box, no swizzle) into a staging ring; warp 2 issues the TMA loads of
//     the stage's Pi tile (K-major, swizzled, up to 256-row boxes) into a Pi ring, all guarded by mbarriers. kind::tf32 takes K-major operands only, so eight copy warps (a 32-column
//     box and two 8-row groups each) read every staged element once, fold x^2 into compensated (TwoSum + FMA
//     residual) column sums, round x to TF32 (cvt.rna) and write it back K-major (swizzled, conflict-free 16-byte
//     stores). Warp 1 (one thread) issues tcgen05.mma kind::tf32 with M = 128 data columns and N = up to 256 sketch
//     rows per instruction into a TMEM accumulator of 128 lanes x up to 512 columns. All 16 warps then drain TMEM
//     with tcgen05.ld and add the tile into the split's partial sketch. Every wait is bounded (%globaltimer, the
//     limit a kernel argument): a timeout sets the device error word and raises the CTA's abort flag; every role
//     leaves its loop, the producers wait (bounded) until the loads they issued have landed, the MMA warp commits
//     the accumulator barrier anyway so the MMAs in flight are waited for, the drain is skipped and TMEM is freed.
#include <cuda.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace smp {
namespace {
using namespace tc;

constexpr int TILE_M = 128;        // data columns per CTA (MMA M)
// Three rings: staged data tiles (TMA target, freed by the copy warps), K-major operand copies (written by the copy
// warps, freed by the MMA) and Pi tiles (TMA target, freed by the MMA); their depths per operand variant are in Geo.
constexpr int PI_BOX_ROWS = 256;   // sketch rows per Pi box (MMA N)
constexpr int MAX_KC = 512;        // sketch rows per CTA (TMEM columns)
// One TMA load moves a whole stage of data: a 128-column x KS-row box without swizzle (row t of the stage: 512
// contiguous bytes), landing column-major. A CTA completes about four TMA loads per microsecond however many are in
// flight (a TMA-only stream on this part: 33 GB/s per CTA with 8 KB boxes at 4 to 24 in flight, 55 GB/s with 16 KB
// boxes, where 128 CTAs reach 7 TB/s), so the box count per byte bounds one CTA's stream.
constexpr int DATA_ROW_BYTES = 128 * 4;
// Operand variants. K-major operand rows hold the KS values of a stage (TF32 in 32-bit containers or BF16): 64-byte
// rows take the 64-byte swizzle (8-row groups 512 B apart), 128-byte rows the 128-byte swizzle (groups 1,024 B apart);
// an MMA K slice is 32 B of the row (8 TF32 or 16 BF16 values).
//  - TF32, k > SMALL_KC: 16-row stages (8 KB of data, a 32 KB Pi stage at k = 512 in two 256-row boxes), rings of
//    data / copies / Pi 4 / 3 / 5: a Pi stage takes ~1-2 us from L2, and 32-row stages (64 KB of Pi each) leave room
//    for only two in flight (0.52 against 0.50 ms per 65,536 x 4,000 block).
//  - TF32, k <= SMALL_KC (the batched and serving sizes, k = 8 r <= 160): 32-row stages (one 16 KB data box, a Pi box
//    of round_up(k, 16) rows, four MMA slices), rings 4 / 3 / 4. Against 16-row stages: 0.31 against 0.42 ms per
//    65,536-row block at n = 2,048, k = 40; 3.75 against 2.9 TB/s over 24 concurrent mixed blocks.
//  - BF16 operands of binary32 inputs: 32-row stages of 64-byte rows, rings 4 / 4 / 4 (k > SMALL_KC) or 6 / 4 / 8.
constexpr int SMALL_KC = 160;
template <bool B16, bool SMALL = false>
struct Geo {
    static constexpr int KS = (B16 || SMALL) ? 32 : 16;      // data rows per pipeline stage
    static constexpr int ROWB = KS * (B16 ? 2 : 4);           // bytes of one K-major operand row
    static constexpr uint32_t SWZ = ROWB == 128 ? SWZ_128B : SWZ_64B;
    static constexpr uint32_t SBO = 8 * ROWB;                // 8-row group stride of the operand layouts
    static constexpr int KSLICES = ROWB / 32;                // MMA K slices per stage
    static constexpr int DSTAGES = B16 ? (SMALL ? 6 : 4) : 4;
    static constexpr int ASTAGES = B16 ? 4 : 3;
    static constexpr int PSTAGES = B16 ? (SMALL ? 8 : 4) : (SMALL ? 4 : 5);
    static constexpr int DATA_STAGE_BYTES = 4 * KS * 32 * 4; // 128 columns x KS rows: [8-row group][32-col box]
    static constexpr int A_SLOT_BYTES = TILE_M * ROWB;
    static constexpr int PI_BOX_BYTES = PI_BOX_ROWS * ROWB;  // a full 256-row box
    static constexpr int PI_SLOT_BYTES = SMALL ? SMALL_KC * ROWB : (MAX_KC / PI_BOX_ROWS) * PI_BOX_BYTES;
    static constexpr int DRING_BYTES = DSTAGES * DATA_STAGE_BYTES;
    static constexpr int ARING_BYTES = ASTAGES * A_SLOT_BYTES;
    static constexpr int PRING_BYTES = PSTAGES * PI_SLOT_BYTES;
    static constexpr int BAR_BYTES = 8 * (2 * (DSTAGES + ASTAGES + PSTAGES) + 1) + 8;   // mbarriers, TMEM address, abort
    static constexpr int SMEM_BYTES = DRING_BYTES + ARING_BYTES + PRING_BYTES + 1024 /* alignment */ + BAR_BYTES;
    static_assert(SMEM_BYTES <= 232448, "shared memory budget");
    static_assert(PI_SLOT_BYTES % 1024 == 0 && A_SLOT_BYTES % 1024 == 0, "slots keep the swizzle atoms aligned");
};
constexpr int PI_GEN_SMEM = 8192;  // see generate_pi
constexpr int PI_ROW_PAD = 64;     // Pi buffers: rows padded to a multiple of 64 (every engine's stage height)
constexpr int THREADS = 512;       // 16 warps: producers 0 and 2, MMA 1, copy warps on schedulers 0, 2, 3
constexpr int NCOPY = 8;           // copy warps: (32-column box, 8-row group) pairs
// copy warp c (0..7) is warp COPY_WARP[c]: warp ids 4, 6, 7, 8, 10, 11, 12, 14 live on schedulers 0, 2, 3 (id % 4),
// leaving scheduler 1 to the MMA issuer (warp 1); tcgen05.mma issue slows down when a busy warp shares it
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
// ------------------------------------------------------------------------------------------------ Pi generation
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return __uint_as_float(y);
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return y;
}
// Two values rounded to BF16 (nearest, ties to even), the first in the low half (the lower K index).
__device__ __forceinline__ uint32_t bf16_pair(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void store_pi(float* p, float z) { *p = to_tf32(z); }
__device__ __forceinline__ void store_pi(__nv_bfloat16* p, float z) { *p = __float2bfloat16_rn(z); }
__device__ __forceinline__ void store_pi(__nv_fp8_e4m3* p, float z) { *p = __nv_fp8_e4m3(z); }

// pi[a][t] (ld = ldp) = Pi(a, row0 + t) rounded to the operand type (TF32 in a binary32 container, or BF16) for
// a < k, t < nrows; 0 for k <= a < kpad or nrows <= t < tpad. One thread per (t, group of four sketch rows): one
// Philox block feeds four rows.
template <typename TP>
__global__ void __launch_bounds__(256) pi_gen_kernel(TP* __restrict__ pi, int64_t ldp, int k, int kpad,
                                                     int64_t row0, int64_t nrows, int64_t tpad, uint32_t k0,
                                                     uint32_t k1, float scale) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int g = blockIdx.y;
    if (t >= tpad) return;
    float z[4] = {0.f, 0.f, 0.f, 0.f};
    if (t < nrows && 4 * g < k) {
        const uint64_t row = (uint64_t)(row0 + t);
        const U32x4 x = philox4x32_10((uint32_t)row, (uint32_t)(row >> 32), (uint32_t)g, TAG_PI, k0, k1);
        box_muller_f32(x.x, x.y, z[0], z[1]);
        box_muller_f32(x.z, x.w, z[2], z[3]);
#pragma unroll
        for (int q = 0; q < 4; ++q) z[q] = (4 * g + q < k) ? z[q] * scale : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (4 * g + q < kpad) store_pi(pi + (int64_t)(4 * g + q) * ldp + t, z[q]);
}

// ------------------------------------------------------------------------------------------------ main kernel
struct TcArgs {
    int64_t n1, n2, ntot;
    int tiles_a;            // column tiles over A; tiles over B follow
    int k, kc, nh;          // sketch rows, TMEM columns used (multiple of 32), Pi boxes per stage
    int n_last;             // N of the last Pi box's MMA (multiple of 16)
    int pbox;               // sketch rows per Pi box: 256, or round_up(k, 16) when one box covers k
    uint32_t tmem_cols;     // power of two >= kc
    int64_t nrows;
    int64_t steps;          // KS-row stages of the block (split s takes stages s, s + splits, ...)
    int64_t ldk;
    float* part;            // [splits][ntot][ldk]
    double* nsq;            // [splits][ntot]
    int* err;
    unsigned long long wait_ns;   // limit of every mbarrier wait
    int skip_stage;               // test hook: the data producer issues nothing from this stage on (-1: never)
};

template <bool B16, bool SMALL>
__global__ void __launch_bounds__(THREADS, 1) sketch_tc_kernel(const __grid_constant__ CUtensorMap tm_a,
                                                               const __grid_constant__ CUtensorMap tm_b,
                                                               const __grid_constant__ CUtensorMap tm_pi,
                                                               const TcArgs args) {
    using G = Geo<B16, SMALL>;
    constexpr int KS = G::KS;
    constexpr int DATA_STAGE_BYTES = G::DATA_STAGE_BYTES;
    constexpr int DSTAGES = G::DSTAGES;
    constexpr int ASTAGES = G::ASTAGES;
    constexpr int PSTAGES = G::PSTAGES;
    constexpr int DRING_BYTES = G::DRING_BYTES;
    constexpr int ARING_BYTES = G::ARING_BYTES;
    constexpr int PRING_BYTES = G::PRING_BYTES;
    constexpr int PI_SLOT_BYTES = G::PI_SLOT_BYTES;
    constexpr int A_SLOT_BYTES = G::A_SLOT_BYTES;
    constexpr int PI_BOX_BYTES = G::PI_BOX_BYTES;
    extern __shared__ uint8_t smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int split = blockIdx.y;
    // row splits interleaved by stage: stage it of split s covers rows (it * splits + s) * KS .. + KS, so at any time
    // all CTAs stream rows from one narrow window of the block (the TMA-only probe: 2.4 against 1.9 TB/s with the
    // splits' rows contiguous)
    const int splits = (int)gridDim.y;
    const int n_it = split < args.steps ? (int)((args.steps - split + splits - 1) / splits) : 0;
    if (n_it <= 0) return;
    auto stage_row = [&](int it) { return (int)(((int64_t)it * splits + split) * KS); };

    const int tile = blockIdx.x;
    const bool on_b = tile >= args.tiles_a;
    const int64_t col0 = on_b ? (int64_t)(tile - args.tiles_a) * TILE_M : (int64_t)tile * TILE_M;
    const int64_t ncols_src = on_b ? args.n2 : args.n1;
    const int valid = (int)(ncols_src - col0 < TILE_M ? ncols_src - col0 : TILE_M);
    const int64_t cbase = on_b ? args.n1 + col0 : col0;
    const CUtensorMap* tm_data = on_b ? &tm_b : &tm_a;

    // carve shared memory (1024-byte aligned): data ring, copy ring, Pi ring, then barriers
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* base_ptr = smem_raw + (base - raw);
    const uint32_t dring = base;                        // DSTAGES x DATA_STAGE_BYTES
    const uint32_t aring = base + DRING_BYTES;          // ASTAGES x A_SLOT_BYTES
    const uint32_t pring = aring + ARING_BYTES;         // PSTAGES x PI_SLOT_BYTES
    const uint32_t bar_base = pring + PRING_BYTES;
    uint64_t* bars = (uint64_t*)(base_ptr + DRING_BYTES + ARING_BYTES + PRING_BYTES);
    // bars: data full / empty [D], copy full / empty [A], Pi full / empty [P]; then the accumulator-ready barrier,
    // the TMEM address word and the abort flag
    uint32_t* tmem_slot = (uint32_t*)(bars + 2 * (DSTAGES + ASTAGES + PSTAGES) + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    // copy warps: compensated sums of squares of their column and row group, even and odd rows in the two lanes of
    // packed f32x2 accumulators (two short dependency chains, half the instructions)
    uint64_t hi2 = 0ull, lo2 = 0ull;
    auto dfull_bar = [&](int d) { return bar_base + 8u * d; };
    auto dempty_bar = [&](int d) { return bar_base + 8u * (DSTAGES + d); };
    auto afull_bar = [&](int s) { return bar_base + 8u * (2 * DSTAGES + s); };
    auto aempty_bar = [&](int s) { return bar_base + 8u * (2 * DSTAGES + ASTAGES + s); };
    auto pfull_bar = [&](int s) { return bar_base + 8u * (2 * DSTAGES + 2 * ASTAGES + s); };
    auto pempty_bar = [&](int s) { return bar_base + 8u * (2 * DSTAGES + 2 * ASTAGES + PSTAGES + s); };
    const uint32_t acc_bar = bar_base + 8u * (2 * DSTAGES + 2 * ASTAGES + 2 * PSTAGES);

    if (threadIdx.x == 0) {
        for (int d = 0; d < DSTAGES; ++d) {
            mbar_init(dfull_bar(d), 1);
            mbar_init(dempty_bar(d), NCOPY);
        }
        for (int s = 0; s < ASTAGES; ++s) {
            mbar_init(afull_bar(s), NCOPY);
            mbar_init(aempty_bar(s), 1);      // the MMA commit
        }
        for (int s = 0; s < PSTAGES; ++s) {
            mbar_init(pfull_bar(s), 1);
            mbar_init(pempty_bar(s), 1);      // the MMA commit
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
        // ---------------- data producer: column-major data tiles into the staging ring (lane 0 issues)
        if (lane == 0) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)tm_data) : "memory");
        int issued = 0;
        // the data is read once: keep it from pushing Pi (read by 32 column tiles) out of L2; with both policies the
        // per-launch times stopped spreading (median 0.505 ms against 0.55-0.59 ms, the minimum unchanged)
        const uint64_t pol_data = policy_evict_first();
        for (int it = 0; it < n_it; ++it) {
            if (it == args.skip_stage) break;   // test hook: the loads of this stage never come
            const int d = it % DSTAGES;
            const uint32_t ph = (uint32_t)(it / DSTAGES) & 1u;
            bool ok = true;
            if (it >= DSTAGES)
                ok = __all_sync(0xffffffffu, mbar_wait_for(dempty_bar(d), ph ^ 1u, abort_flag, args.wait_ns));
            if (!ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    set_error(args.err, DEVERR_TIMEOUT | (1 << 8));
                }
                break;
            }
            if (lane == 0) {
                mbar_arrive_expect_tx(dfull_bar(d), DATA_STAGE_BYTES);
                tma_load_2d_hint(dring + d * DATA_STAGE_BYTES, tm_data, (int)col0, stage_row(it), dfull_bar(d),
                                 pol_data);
            }
            issued = it + 1;
            __syncwarp();
        }
        // the TMEM drain reads and rewrites this tile's slice of the split's partial sketch: bring it into L2 while
        // the last stages are still in flight
        {
            const int nlines = (int)((args.ldk * 4 + 127) / 128);   // 128-byte lines per partial row (may overhang)
            for (int e = lane; e < valid * nlines; e += 32) {
                const int m = e / nlines, l = e - m * nlines;
                const char* pr = (const char*)(args.part + ((int64_t)split * args.ntot + cbase + m) * args.ldk) + l * 128;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(pr));
            }
        }
        // the CTA may not finish while a load it issued is still landing in its shared memory (even after an abort)
        for (int it = max(0, issued - DSTAGES); it < issued; ++it)
            mbar_wait_landed(dfull_bar(it % DSTAGES), (uint32_t)(it / DSTAGES) & 1u, args.wait_ns);
    } else if (warp == 2) {
        // ---------------- Pi producer: Pi tiles into the ring once the MMA has released the slot (splitting a stage's
        // two boxes over two issuing warps measured slower: 0.54 against 0.50 ms per 65,536 x 4,000 block)
        if (lane == 0) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_pi) : "memory");
        const uint32_t bytes = (uint32_t)(args.nh * args.pbox * G::ROWB);
        const uint64_t pol_pi = policy_evict_last();
        int issued = 0;
        for (int it = 0; it < n_it; ++it) {
            const int s = it % PSTAGES;
            const uint32_t ph = (uint32_t)(it / PSTAGES) & 1u;
            bool ok = true;
            if (it >= PSTAGES)
                ok = __all_sync(0xffffffffu, mbar_wait_for(pempty_bar(s), ph ^ 1u, abort_flag, args.wait_ns));
            if (!ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    set_error(args.err, DEVERR_TIMEOUT | (1 << 12));
                }
                break;
            }
            if (lane == 0) {
                mbar_arrive_expect_tx(pfull_bar(s), bytes);
                const int t = stage_row(it);
                for (int h = 0; h < args.nh; ++h)
                    tma_load_2d_hint(pring + s * PI_SLOT_BYTES + h * PI_BOX_BYTES, &tm_pi, t, h * PI_BOX_ROWS,
                                     pfull_bar(s), pol_pi);
            }
            issued = it + 1;
            __syncwarp();
        }
        // the CTA may not finish while a load it issued is still landing (even after an abort)
        for (int it = max(0, issued - PSTAGES); it < issued; ++it)
            mbar_wait_landed(pfull_bar(it % PSTAGES), (uint32_t)(it / PSTAGES) & 1u, args.wait_ns);
    } else if (warp == 1) {
        // ---------------- MMA issuer (the whole warp waits; lane 0 issues)
        const uint32_t id_full = B16 ? idesc_bf16(TILE_M, PI_BOX_ROWS, false) : idesc_tf32(TILE_M, PI_BOX_ROWS);
        const uint32_t id_last = B16 ? idesc_bf16(TILE_M, args.n_last, false) : idesc_tf32(TILE_M, args.n_last);
        bool ok = true;
        for (int it = 0; it < n_it; ++it) {
            const int sp = it % PSTAGES, sa = it % ASTAGES;
            const uint32_t pph = (uint32_t)(it / PSTAGES) & 1u, aph = (uint32_t)(it / ASTAGES) & 1u;
            ok = __all_sync(0xffffffffu, mbar_wait_for(pfull_bar(sp), pph, abort_flag, args.wait_ns) &&
                                             mbar_wait_for(afull_bar(sa), aph, abort_flag, args.wait_ns));
            if (!ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    set_error(args.err, DEVERR_TIMEOUT | (1 << 9));
                }
                break;
            }
            tc_fence_after();
            if (lane == 0) {
                const uint32_t abase = aring + sa * A_SLOT_BYTES, pbase = pring + sp * PI_SLOT_BYTES;
#pragma unroll
                for (int kb = 0; kb < G::KSLICES; ++kb) {
                    // both operands K-major and swizzled (TF32: 128-byte rows, BF16: 64-byte rows; 8-row groups SBO
                    // apart); K slice kb (8 TF32 or 16 BF16 values) at +32 kb bytes of the row
                    const uint64_t ad = smem_desc(abase + kb * 32, 16, G::SBO, G::SWZ);
                    for (int h = 0; h < args.nh; ++h) {
                        const uint64_t bd = smem_desc(pbase + h * PI_BOX_BYTES + kb * 32, 16, G::SBO, G::SWZ);
                        if (B16)
                            mma_bf16(tmem + h * PI_BOX_ROWS, ad, bd, h == args.nh - 1 ? id_last : id_full,
                                     (it > 0 || kb > 0) ? 1u : 0u);
                        else
                            mma_tf32(tmem + h * PI_BOX_ROWS, ad, bd, h == args.nh - 1 ? id_last : id_full,
                                     (it > 0 || kb > 0) ? 1u : 0u);
                    }
                }
                mma_commit(aempty_bar(sa));
                mma_commit(pempty_bar(sp));
            }
            __syncwarp();
        }
        // always: the accumulator commit also tells the drain when the MMAs in flight have finished
        if (lane == 0) mma_commit(acc_bar);
        __syncwarp();
    } else if (copy_index(warp) >= 0) {
        // ---------------- copy warps: a 32-column box and the 8-row groups ci / 4, ci / 4 + 2 of the stage: column sums
        // of squares and the K-major operand copy of their rows (TF32: 16 B per 4 rows; BF16: 16 B per 8 rows)
        const int ci = copy_index(warp);
        const int box = ci & 3, grp0 = ci >> 2;
        const int m = box * 32 + lane;   // data column within the tile
        constexpr int NG = KS / 16;      // 8-row groups per copy warp
        for (int it = 0; it < n_it; ++it) {
            const int d = it % DSTAGES;
            const uint32_t dph = (uint32_t)(it / DSTAGES) & 1u;
            const int s = it % ASTAGES;
            const uint32_t ph = (uint32_t)(it / ASTAGES) & 1u;
            bool ok = mbar_wait_for(dfull_bar(d), dph, abort_flag, args.wait_ns);
            if (ok && it >= ASTAGES) ok = mbar_wait_for(aempty_bar(s), ph ^ 1u, abort_flag, args.wait_ns);   // slot free
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) {
                    *abort_flag = 1;
                    set_error(args.err, DEVERR_TIMEOUT | (1 << 10));
                }
                break;
            }
            // staged stage: row t at t * 512 B, the warp's 32 columns (128 contiguous bytes: conflict-free) per row
            float x[NG][8];
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                const float* grp_p = (const float*)(base_ptr + d * DATA_STAGE_BYTES +
                                                    (grp0 + 2 * g) * 8 * DATA_ROW_BYTES) + box * 32 + lane;
#pragma unroll
                for (int t = 0; t < 8; ++t) x[g][t] = grp_p[t * 128];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(dempty_bar(d));   // staging read: the producer may refill it
            // K-major copy: data column m is operand row m (ROWB bytes); the swizzle puts 16-byte chunk q at q ^ sw
            // (128-byte rows: sw = m % 8; 64-byte rows: sw = (m / 2) % 4)
            uint4* arow = (uint4*)(base_ptr + DRING_BYTES + s * A_SLOT_BYTES + m * G::ROWB);
            const int sw = G::ROWB == 128 ? m & 7 : (m >> 1) & 3;
#pragma unroll
            for (int g = 0; g < NG; ++g) {
#pragma unroll
                for (int t = 0; t < 8; t += 2) two_sum_square_x2(pack2(x[g][t], x[g][t + 1]), hi2, lo2);
                if (B16) {   // rows 8 gg .. 8 gg + 7 as BF16 (round to nearest even) in chunk gg
                    const int gg = grp0 + 2 * g;
                    uint4 v;
                    v.x = bf16_pair(x[g][0], x[g][1]);
                    v.y = bf16_pair(x[g][2], x[g][3]);
                    v.z = bf16_pair(x[g][4], x[g][5]);
                    v.w = bf16_pair(x[g][6], x[g][7]);
                    arow[gg ^ sw] = v;
                } else {     // rows 8 gg .. 8 gg + 7 as TF32 in chunks 2 gg, 2 gg + 1
                    const int q0 = 2 * (grp0 + 2 * g);
                    arow[q0 ^ sw] = make_uint4(tf32_bits(x[g][0]), tf32_bits(x[g][1]), tf32_bits(x[g][2]),
                                               tf32_bits(x[g][3]));
                    arow[(q0 + 1) ^ sw] = make_uint4(tf32_bits(x[g][4]), tf32_bits(x[g][5]), tf32_bits(x[g][6]),
                                                     tf32_bits(x[g][7]));
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(afull_bar(s));
        }
    }
    __syncthreads();   // every role has left its loop: the staging ring is free
    double* nsum = (double*)base_ptr;   // per column: the two 8-row groups' compensated sums of squares
    if (copy_index(warp) >= 0) {
        const int ci = copy_index(warp);
        float hi0, hi1, lo0, lo1;
        unpack2(hi2, hi0, hi1);
        unpack2(lo2, lo0, lo1);
        nsum[(ci >> 2) * TILE_M + (ci & 3) * 32 + lane] = ((double)hi0 + (double)lo0) + ((double)hi1 + (double)lo1);
    }
    __syncthreads();
    {
        // ---------------- TMEM drain by all 16 warps: warp w reads TMEM lanes 32 (w % 4) ... and the column quarter
        // w / 4 of the accumulator, and adds it into the split's partial sketch
        const int q = warp & 3;
        const int m = q * 32 + lane;
        const int cq = ((args.kc / 32 + 3) / 4) * 32;   // accumulator columns per warp (multiple of 32)
        const int cbeg = (warp >> 2) * cq, cend = min(args.kc, cbeg + cq);
        const bool landed = __all_sync(0xffffffffu, mbar_wait_for(acc_bar, 0, abort_flag, args.wait_ns));
        const bool acc_ok = landed && !*abort_flag;
        if (acc_ok) {
            tc_fence_after();
            const int64_t c = cbase + m;
            float* dst = args.part + ((int64_t)split * args.ntot + c) * args.ldk;
            for (int cc = cbeg; cc < cend; cc += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)cc, v);
                if (m < valid) {
                    if (args.ldk % 4 == 0) {
#pragma unroll
                        for (int i = 0; i < 32; i += 4)
                            if (cc + i < args.ldk) {
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
                            if (cc + i < args.k) dst[cc + i] += v[i];
                    }
                }
            }
            if (warp < 4 && m < valid) args.nsq[(int64_t)split * args.ntot + c] += nsum[m] + nsum[TILE_M + m];
        } else if (!landed && lane == 0) {
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

// ------------------------------------------------------------------------------------------------ host side
bool aligned16(const void* p, int64_t ld) { return ((uintptr_t)p % 16 == 0) && (ld % 4 == 0); }

template <typename K>
cudaError_t set_smem(K* kernel, int bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Pi buffers, side stream and events of the tensor-core engine (created on first use).
cudaError_t ensure_pi_buffers(smp_ctx* c, size_t bytes) {
    if (!c->gen_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->gen_stream, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaEventCreateWithFlags(&c->pi_ready[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->pi_free[b], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return e;
    }
    if (c->pi_buf_bytes >= bytes) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(c->gen_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);   // no sketch still reads the old buffers
    if (e != cudaSuccess) return e;
    for (int b = 0; b < 2; ++b) {
        free_idle(c->pi_buf[b]);   // both streams were synchronised above
        c->pi_buf[b] = nullptr;
        c->pi_row0[b] = -1;
        c->pi_nrows[b] = 0;
    }
    c->pi_buf_bytes = 0;
    for (int b = 0; b < 2; ++b) {
        // stream-ordered on the context's stream; the side stream's first generation into the buffer waits for
        // pi_free[b], recorded here after the allocation
        e = dev_malloc(&c->pi_buf[b], bytes, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(c->pi_free[b], c->stream);
        if (e != cudaSuccess) return e;
    }
    c->pi_buf_bytes = bytes;
    return cudaSuccess;
}

// Pi for rows [row0, row0 + nrows) into buffer b on the side stream, once the last sketch that read b has ended.
// The kernel asks for PI_GEN_SMEM bytes of shared memory it does not use: a sketch CTA leaves less than that free
// on its SM, so the generator only runs on SMs the sketch grid leaves idle instead of slowing its CTAs down.
cudaError_t generate_pi(smp_ctx* c, int b, int64_t row0, int64_t nrows) {
    cudaError_t e = cudaStreamWaitEvent(c->gen_stream, c->pi_free[b], 0);
    if (e != cudaSuccess) return e;
    const PiGeom gm = pi_geom(c);
    const int k = c->p.k;
    const int64_t tpad = round_up(nrows, PI_ROW_PAD);
    const dim3 g((unsigned)((tpad + 255) / 256), (unsigned)(gm.kpad / 4));
    const uint32_t k0 = (uint32_t)c->p.seed, k1 = (uint32_t)(c->p.seed >> 32);
    const float scale = (float)(1.0 / std::sqrt((double)k));
    if (gm.esize == 1)   // E4M3 of the N(0, 1) normals; the sketch kernel applies 1 / sqrt(k)
        pi_gen_kernel<__nv_fp8_e4m3><<<smp::counted(g), 256, PI_GEN_SMEM, c->gen_stream>>>(
            (__nv_fp8_e4m3*)c->pi_buf[b], gm.ld, k, gm.kpad, row0, nrows, tpad, k0, k1, 1.f);
    else if (gm.esize == 2)
        pi_gen_kernel<__nv_bfloat16><<<smp::counted(g), 256, PI_GEN_SMEM, c->gen_stream>>>(
            (__nv_bfloat16*)c->pi_buf[b], gm.ld, k, gm.kpad, row0, nrows, tpad, k0, k1, scale);
    else
        pi_gen_kernel<float><<<smp::counted(g), 256, PI_GEN_SMEM, c->gen_stream>>>(
            (float*)c->pi_buf[b], gm.ld, k, gm.kpad, row0, nrows, tpad, k0, k1, scale);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(c->pi_ready[b], c->gen_stream);
    if (e != cudaSuccess) return e;
    c->pi_row0[b] = row0;
    c->pi_nrows[b] = nrows;
    return cudaSuccess;
}

}  // namespace

PiGeom pi_geom(const smp_ctx* c) {
    PiGeom g;
    // binary32 row blocks go to sketch_tc_kernel, whose Pi box is round_up(k, 16) rows when that is at most 256;
    // the BF16-input engines read 256-row boxes
    const int k16 = (int)round_up(c->p.k, 16);
    g.kpad = (c->p.dtype == SMP_F32 && k16 <= PI_BOX_ROWS) ? k16 : (int)round_up(k16, 256);
    g.ld = round_up(c->max_rows, PI_ROW_PAD);
    g.esize = c->p.engine == SMP_ENGINE_TC_FP8 ? 1
              : (c->p.dtype == SMP_BF16 || c->p.engine == SMP_ENGINE_TC_BF16) ? 2 : 4;
    return g;
}

cudaError_t pi_acquire(smp_ctx* c, int64_t row0, int64_t nrows, int* buf) {
    const PiGeom gm = pi_geom(c);
    cudaError_t e = ensure_pi_buffers(c, (size_t)gm.kpad * gm.ld * gm.esize);
    if (e != cudaSuccess) return e;
    int b = -1;
    for (int b2 = 0; b2 < 2 && b < 0; ++b2)
        if (c->pi_row0[b2] == row0 && c->pi_nrows[b2] >= nrows) b = b2;
    if (b < 0) {
        b = c->pi_row0[0] < 0 ? 0 : (c->pi_row0[1] < 0 ? 1 : (c->pi_nrows[0] <= c->pi_nrows[1] ? 0 : 1));
        e = generate_pi(c, b, row0, nrows);
        if (e != cudaSuccess) return e;
    }
    e = cudaStreamWaitEvent(c->stream, c->pi_ready[b], 0);
    *buf = b;
    return e;
}

cudaError_t pi_release(smp_ctx* c, int b, int64_t row0, int64_t nrows) {
    cudaError_t e = cudaEventRecord(c->pi_free[b], c->stream);
    c->pi_last = b;
    c->pi_last_rows = std::max(c->pi_last_rows, nrows);
    const int other = 1 - b;
    const int64_t next0 = row0 + nrows;
    if (e == cudaSuccess && !(c->pi_row0[other] == next0 && c->pi_nrows[other] >= nrows))
        e = generate_pi(c, other, next0, nrows);
    return e;
}

namespace {
// dst[a][t] (ld) = src[a][t] (ldp) rounded to the operand type (BF16 or E4M3) for a < k, t < nrows; zeros
// elsewhere up to kpad x tpad.
template <typename TP>
__global__ void pi_import_kernel(const float* __restrict__ src, int64_t ldp, int k, int64_t nrows, TP* dst,
                                 int64_t ld, int kpad, int64_t tpad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (t >= tpad || a >= kpad) return;
    const float v = (a < k && t < nrows) ? src[(int64_t)a * ldp + t] : 0.f;
    store_pi(dst + (int64_t)a * ld + t, v);
}
}  // namespace

cudaError_t pi_import(smp_ctx* c, const float* Pi, int64_t ldp, int64_t nrows, int* buf) {
    const PiGeom gm = pi_geom(c);
    cudaError_t e = ensure_pi_buffers(c, (size_t)gm.kpad * gm.ld * gm.esize);
    if (e != cudaSuccess) return e;
    const int b = c->pi_last < 0 ? 0 : 1 - c->pi_last;
    // the caller's Pi replaces whatever the buffer held; the stream waits for the buffer's generator and readers
    e = cudaStreamWaitEvent(c->stream, c->pi_ready[b], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->pi_free[b], 0);
    if (e != cudaSuccess) return e;
    c->pi_row0[b] = -1;
    c->pi_nrows[b] = 0;
    const int64_t tpad = round_up(nrows, PI_ROW_PAD);
    const dim3 grid((unsigned)((tpad + 255) / 256), (unsigned)gm.kpad);
    if (gm.esize == 2)
        pi_import_kernel<__nv_bfloat16><<<smp::counted(grid), 256, 0, c->stream>>>(
            Pi, ldp, c->p.k, nrows, (__nv_bfloat16*)c->pi_buf[b], gm.ld, gm.kpad, tpad);
    else if (gm.esize == 1)
        pi_import_kernel<__nv_fp8_e4m3><<<smp::counted(grid), 256, 0, c->stream>>>(
            Pi, ldp, c->p.k, nrows, (__nv_fp8_e4m3*)c->pi_buf[b], gm.ld, gm.kpad, tpad);
    else
        return cudaErrorInvalidValue;
    *buf = b;
    return cudaGetLastError();
}

cudaError_t tc_speculate_first_block(smp_ctx* c) {
    if (!c->gen_stream || c->pi_last < 0 || c->pi_last_rows <= 0) return cudaSuccess;
    const int other = 1 - c->pi_last;
    if (c->pi_row0[other] == 0 && c->pi_nrows[other] >= c->pi_last_rows) return cudaSuccess;
    return generate_pi(c, other, 0, c->pi_last_rows);
}

void release_tc(smp_ctx* c) {
    if (c->gen_stream) cudaStreamSynchronize(c->gen_stream);   // the side stream is done with the buffers
    release_after(c->stream);
    free_idle(c->fp8_ws);
    c->fp8_ws = nullptr;
    for (int b = 0; b < 2; ++b) {
        free_idle(c->pi_buf[b]);
        if (c->pi_ready[b]) cudaEventDestroy(c->pi_ready[b]);
        if (c->pi_free[b]) cudaEventDestroy(c->pi_free[b]);
        c->pi_buf[b] = nullptr;
        c->pi_ready[b] = c->pi_free[b] = nullptr;
    }
    if (c->gen_stream) cudaStreamDestroy(c->gen_stream);
    c->gen_stream = nullptr;
    c->pi_buf_bytes = 0;
}

bool tc_supported(const smp_ctx* c) { return c->p.dtype == SMP_F32 && c->p.k <= MAX_KC && encode_fn() != nullptr; }

bool tc_block_ok(const smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb) {
    return tc_supported(c) && aligned16(A, lda) && (c->p.same_ab || aligned16(B, ldb));
}

cudaError_t launch_sketch_tc_pi(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                                int64_t nrows, const float* Pi, int64_t ldp) {
    // SMP_ENGINE_TC_BF16: BF16 operands (32 rows per stage, Pi in BF16); otherwise TF32 operands
    const bool b16 = c->p.engine == SMP_ENGINE_TC_BF16;
    const int k = c->p.k;
    const int kc = (int)round_up(k, 32);                 // TMEM columns drained (multiple of 32)
    const int kmma = (int)round_up(k, 16);               // MMA N coverage
    const int nh = (kmma + PI_BOX_ROWS - 1) / PI_BOX_ROWS;
    const int n_last = kmma - (nh - 1) * PI_BOX_ROWS;
    const int pbox = nh == 1 ? kmma : PI_BOX_ROWS;
    const bool small = kmma <= SMALL_KC;
    const int variant = (b16 ? 1 : 0) + (small ? 2 : 0);
    static std::atomic<bool> attr[4] = {{false}, {false}, {false}, {false}};
    if (!attr[variant]) {
        cudaError_t e = cudaSuccess;
        switch (variant) {
            case 0: e = set_smem(sketch_tc_kernel<false, false>, Geo<false, false>::SMEM_BYTES); break;
            case 1: e = set_smem(sketch_tc_kernel<true, false>, Geo<true, false>::SMEM_BYTES); break;
            case 2: e = set_smem(sketch_tc_kernel<false, true>, Geo<false, true>::SMEM_BYTES); break;
            default: e = set_smem(sketch_tc_kernel<true, true>, Geo<true, true>::SMEM_BYTES); break;
        }
        if (e != cudaSuccess) return e;
        attr[variant] = true;
    }
    const int ks = (b16 || small) ? 32 : 16;
    const CUtensorMapSwizzle pi_swz = (!b16 && small) ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    const int64_t tpad = round_up(nrows, ks);
    cudaStream_t st = c->stream;
    const void* pi = Pi;
    int64_t pld = ldp;
    int64_t pi_rows = k;
    int64_t pi_inner = nrows;
    int buf = -1;
    if (!pi || b16) {
        // generated Pi (kpad rows, zero beyond k; double-buffered, generated one block ahead on a side stream), or
        // the caller's Pi rounded to BF16 into a Pi buffer
        cudaError_t e = pi ? pi_import(c, Pi, ldp, nrows, &buf) : pi_acquire(c, row0, nrows, &buf);
        if (e != cudaSuccess) return e;
        const PiGeom gm = pi_geom(c);
        pi = c->pi_buf[buf];
        pld = gm.ld;
        pi_rows = gm.kpad;
        pi_inner = tpad;
    }
    CUtensorMap ma, mb, mp;
    const void* Bp = c->p.same_ab ? A : B;
    const int64_t n2 = c->p.same_ab ? 0 : c->p.n2;
    // data boxes: 128 columns x ks rows, no swizzle = the kernel's DATA_STAGE_BYTES per stage (its expect_tx);
    // Pi boxes: ks values per sketch row (TF32: 128 B, 128-byte swizzle; BF16: 64 B, 64-byte swizzle) x pbox rows
    if (!make_map(&ma, A, (uint64_t)c->p.n1, (uint64_t)nrows, (uint64_t)lda, TILE_M, ks, CU_TENSOR_MAP_SWIZZLE_NONE) ||
        !make_map(&mb, Bp, (uint64_t)(c->p.same_ab ? c->p.n1 : c->p.n2), (uint64_t)nrows,
                  (uint64_t)(c->p.same_ab ? lda : ldb), TILE_M, ks, CU_TENSOR_MAP_SWIZZLE_NONE) ||
        !(b16 ? make_map(&mp, pi, (uint64_t)pi_inner, (uint64_t)pi_rows, (uint64_t)pld, ks, pbox,
                         CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2)
              : make_map(&mp, pi, (uint64_t)pi_inner, (uint64_t)pi_rows, (uint64_t)pld, ks, pbox, pi_swz)))
        return cudaErrorInvalidValue;
    TcArgs a;
    a.n1 = c->p.n1;
    a.n2 = n2;
    a.ntot = c->ntot;
    a.tiles_a = (int)((c->p.n1 + TILE_M - 1) / TILE_M);
    const int tiles = a.tiles_a + (int)((n2 + TILE_M - 1) / TILE_M);
    a.k = k;
    a.kc = kc;
    a.nh = nh;
    a.n_last = n_last;
    a.pbox = pbox;
    uint32_t cols = 32;
    while ((int)cols < kc) cols <<= 1;
    a.tmem_cols = cols;
    a.nrows = nrows;
    const int64_t steps = tpad / ks;
    int splits = std::max(1, std::min(c->splits, c->sm_count / std::max(1, tiles)));
    splits = (int)std::min<int64_t>(splits, steps);
    a.steps = steps;
    a.ldk = c->ldk;
    a.part = (float*)c->part;
    a.nsq = c->nsq;
    a.err = c->dev_err;
    const int64_t wait = g_tc_wait_ns.load(std::memory_order_relaxed);
    a.wait_ns = wait > 0 ? (unsigned long long)wait : WAIT_NS;
    a.skip_stage = g_tc_skip_stage.exchange(-1, std::memory_order_relaxed);
    const dim3 grid = smp::counted(dim3((unsigned)tiles, (unsigned)splits));
    switch (variant) {
        case 0: sketch_tc_kernel<false, false><<<grid, THREADS, Geo<false, false>::SMEM_BYTES, st>>>(ma, mb, mp, a); break;
        case 1: sketch_tc_kernel<true, false><<<grid, THREADS, Geo<true, false>::SMEM_BYTES, st>>>(ma, mb, mp, a); break;
        case 2: sketch_tc_kernel<false, true><<<grid, THREADS, Geo<false, true>::SMEM_BYTES, st>>>(ma, mb, mp, a); break;
        default: sketch_tc_kernel<true, true><<<grid, THREADS, Geo<true, true>::SMEM_BYTES, st>>>(ma, mb, mp, a); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || buf < 0) return e;
    if (Pi) {   // a caller's Pi: the buffer only becomes free again, nothing is generated ahead
        c->pi_last = buf;
        return cudaEventRecord(c->pi_free[buf], st);
    }
    // the sketch reads buffer `buf` until it ends; meanwhile the other buffer gets Pi of the next row block
    return pi_release(c, buf, row0, nrows);
}

cudaError_t launch_sketch_tc(smp_ctx* c, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t row0,
                             int64_t nrows) {
    return launch_sketch_tc_pi(c, A, lda, B, ldb, row0, nrows, nullptr, 0);
}

}  // namespace smp
