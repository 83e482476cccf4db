/*
 * smp.h -- C ABI of libsmp, a GB300 (sm_103a) implementation of SMP-PCA, the single-pass rank-r approximation of
 * A^T B from "Single Pass PCA of Matrix Products" (Wu, Bhojanapalli, Sanghavi, Dimakis; arXiv 1610.06656).
 *
 * The path (Algorithm 1):
 *   smp_sketch_begin / smp_sketch_accumulate / smp_sketch_finalize   step 2: At = Pi A, Bt = Pi B, ||A_i||, ||B_j||
 *   smp_sample                                                       step 3: Omega by Eq. (1)
 *   smp_estimate                                                     step 4: M~ over Omega by Eq. (2)
 *   smp_waltmin                                                      step 5: Algorithm 2 (Appendix A)
 *   smp_sketch_svd                     the baseline SVD(At^T Bt) of Section 4, from the same finalized sketches
 *
 * LELA, the two-pass method of Section 4 (Table 1) that SMP-PCA is compared with, on the same context:
 *   smp_norms_accumulate + smp_sketch_finalize   pass 1: ||A_i||, ||B_j|| alone (no sketch)
 *   smp_sample                                   Omega by Eq. (1), the sampling SMP-PCA takes over from LELA
 *   smp_exact_accumulate / smp_exact_values      pass 2: the exact entries A_i^T B_j of A^T B over Omega
 *   smp_waltmin                                  Algorithm 2 on the exact entries
 *
 * Conventions shared by every call:
 *   - Pointers named *_dev are CUDA device pointers owned by the caller unless stated otherwise. Pointers
 *     returned by the *_view calls are borrowed from the context and stay valid until smp_destroy (or until the
 *     next call that rebuilds them, as stated).
 *   - Every call is issued on the context's stream (the cudaStream_t given to smp_sketch_begin, passed as void*).
 *     Calls are asynchronous unless stated; smp_sample and smp_waltmin synchronise the stream before returning.
 *   - Every call returns an smp_status and never aborts the process. smp_last_error gives a one-line reason.
 *     A kernel that detects a numerical failure records it in a device error word that the next synchronising
 *     call reports (SMP_ENUMERIC / SMP_ETIMEOUT).
 *   - Matrices are row-major. A row block holds data rows [row0, row0 + nrows) of A (nrows x n1, leading
 *     dimension lda elements) and of B (nrows x n2, ldb). Blocks may arrive in any order; a block that overlaps
 *     rows already accumulated is rejected (smp_sketch_coverage reports what has been seen).
 *   - Randomness: Pi, the sampling coins, the optional Omega split and the start block of the initial subspace
 *     iteration come from Philox4x32-10 (Salmon et al., SC'11) with the counter layouts documented with each
 *     call, so results are a function of (inputs, seeds) only.
 */
#ifndef SMP_H
#define SMP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SMP_OK = 0,
    SMP_EINVAL = 1,        /* bad argument: null pointer, size out of range, misaligned leading dimension */
    SMP_ENOMEM = 2,        /* a device allocation failed */
    SMP_ECUDA = 3,         /* a CUDA runtime call failed (see smp_last_error) */
    SMP_ESTATE = 4,        /* call out of order (e.g. accumulate after finalize, estimate before sample) */
    SMP_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    SMP_ENUMERIC = 6,      /* a factorisation broke down (non-positive pivot) */
    SMP_EUNSUPPORTED = 7,  /* valid request this build does not implement (e.g. dtype/engine pair) */
    SMP_EBUSY = 8          /* serving: the job does not fit in what is left of the memory budget; retry later */
} smp_status;

typedef enum {
    SMP_F32 = 0,           /* row blocks are float */
    SMP_BF16 = 1,          /* row blocks are bfloat16 */
    SMP_F64 = 2            /* row blocks are double; the sketch accumulates in double */
} smp_dtype;

typedef enum {
    SMP_ENGINE_AUTO = 0,   /* tensor-core sketch where the dtype has one, else SIMT */
    SMP_ENGINE_SIMT = 1,   /* CUDA-core sketch: FP32 FMA (FP64 for SMP_F64); the exact-arithmetic reference */
    SMP_ENGINE_TC = 2,     /* tcgen05 sketch, FP32 accumulation: SMP_F32 as TF32 operands with k <= 512 (row
                              blocks 16-byte aligned, lda, ldb multiples of 4); SMP_BF16 as BF16 operands with
                              k <= 1024 (row blocks 16-byte aligned, lda, ldb multiples of 8) */
    SMP_ENGINE_TC_FP8 = 3, /* tcgen05 sketch of SMP_BF16 row blocks with FP8 E4M3 operands: each block is scaled by
                              one power of two per matrix, 2^ceil(log2(max |x| / 448)), Pi is E4M3 of the normals,
                              FP32 accumulation; column norms of the stored BF16 values. k <= 1024, alignment as for
                              SMP_BF16. Never chosen by SMP_ENGINE_AUTO. */
    SMP_ENGINE_SRHT = 4,   /* block SRHT as Pi (Section 4: the Spark implementation's sketch) instead of the Gaussian:
                              data rows in blocks of R = max_rows rows (a power of two in [256, 2^16]; block b =
                              rows [bR, (b+1)R)), Pi_b = k^-1/2 S_b H_R D_b with D_b the signs of Philox counter
                              (t mod 2^32, t >> 32, 0, 6) (bit 0 of word 0 set: -1), H_R the unnormalised Sylvester
                              Walsh-Hadamard matrix and S_b k rows of H_R drawn with replacement (row a: the top
                              log2(R) bits of word 0 of counter (a, b mod 2^32, b >> 32, 7)). SMP_F32 only; every
                              accumulate call covers one block (row0 % max_rows == 0); binary32 arithmetic, norms
                              compensated as in the other engines. Never chosen by SMP_ENGINE_AUTO. */
    SMP_ENGINE_TC_BF16 = 5 /* tcgen05 sketch of SMP_F32 row blocks with BF16 operands: the kernel rounds each input
                              to BF16 (nearest, ties to even) on its way to the tensor cores, Pi is generated in
                              BF16, accumulation in FP32 (kind::f16), column norms compensated from the binary32
                              inputs; k <= 512, alignment as SMP_ENGINE_TC's SMP_F32 case. Never chosen by
                              SMP_ENGINE_AUTO. */
} smp_engine;

/* smp_waltmin flags */
#define SMP_SPLIT_OMEGA 1u   /* Algorithm 2 step 3: each sample joins subset floor(u (2T+1)), u its split coin  */
#define SMP_NO_TRIM     2u   /* skip Algorithm 2 step 6                                                          */
#define SMP_INIT_GIVEN  4u   /* use the caller's U_init (n1 x r, double) instead of steps 4-6                    */
#define SMP_FP64_ALS    8u   /* Gram matrices and iterates in double (default: float Gram, double Cholesky)     */

typedef struct {
    int64_t n1;            /* columns of A (>= 1)                                                             */
    int64_t n2;            /* columns of B (>= 1); must equal n1 when same_ab                                  */
    int32_t k;             /* sketch size, 1 <= k <= 4096 (tensor-core engines: k <= 512 TF32, 1024 BF16 / FP8) */
    int32_t dtype;         /* smp_dtype of the row blocks                                                      */
    uint64_t seed;         /* Pi seed: Philox key (seed mod 2^32, seed >> 32)                                  */
    int32_t same_ab;       /* 1: B is A (PCA, Section 3 Remark 3); B pointers are ignored and Bt aliases At     */
    int32_t engine;        /* smp_engine                                                                       */
    int64_t max_rows;      /* largest nrows any accumulate call will pass (sizes scratch); 0 means 65,536      */
} smp_params;

typedef struct smp_ctx smp_ctx;

/* Create a context and its resident device accumulators (Algorithm 1, step 2: the sketch state At, Bt and the
 * column sums of squares). stream is a cudaStream_t (NULL = legacy default stream); the context uses the device
 * current at this call. On success *out owns about 4 * (n1 + n2) * (k + 4) * S bytes of device memory, S the
 * number of row splits the sketch engine uses (at most 8). Errors: SMP_EINVAL, SMP_ENOMEM, SMP_ECUDA. */
smp_status smp_sketch_begin(const smp_params* params, void* stream, smp_ctx** out);

/* Add the contribution of data rows [row0, row0 + nrows): At += Pi[:, rows] A_blk, Bt += Pi[:, rows] B_blk and the
 * squares of every entry to the column sums (Algorithm 1, step 2; Section 2.1 "Step 1"). Pi(a, t) ~ N(0, 1/k) is
 * generated from Philox counter (t mod 2^32, t >> 32, a / 4, 1) with a Box-Muller map (words 0,1 -> rows 4g, 4g+1;
 * words 2,3 -> rows 4g+2, 4g+3; u1 = ((x>>8)+1) 2^-24, u2 = (x>>8) 2^-24, rho = sqrt(-2 ln u1),
 * z = rho cos(2 pi u2), rho sin(2 pi u2), Pi = z / sqrt(k)) and never kept beyond the block: the CUDA-core engine
 * generates it in registers; the tensor-core engines generate the block's k x nrows slice once, in the operand
 * type, into a context buffer that every column tile of the block reads (and that the next block overwrites).
 * A_blk_dev / B_blk_dev: device, row-major, element type from params.dtype, lda >= n1, ldb >= n2; B ignored when
 * same_ab. 0 <= nrows <= max_rows; nrows = 0 is a no-op. Blocks may arrive in any order; a block overlapping
 * rows already accumulated since the context was created or reset is rejected (SMP_EINVAL) before anything is
 * launched, since it would be summed twice. Asynchronous. Errors: SMP_EINVAL, SMP_ESTATE (after finalize),
 * SMP_ECUDA. */
smp_status smp_sketch_accumulate(smp_ctx* ctx, const void* A_blk_dev, int64_t lda, const void* B_blk_dev,
                                 int64_t ldb, int64_t row0, int64_t nrows);

/* smp_sketch_accumulate for a row block held in HOST memory: A_blk_host (nrows x n1, leading dimension lda) and
 * B_blk_host (nrows x n2, ldb; ignored when same_ab) are copied into one of two context-owned device staging
 * buffers (max_rows x (n1 + n2) elements, rows padded to 16 bytes, allocated on the first call) on a copy stream of
 * the context, and the block is then sketched from there on the context's stream exactly as smp_sketch_accumulate
 * would (same engines, checks and results). Consecutive calls alternate between the two buffers, so the copy of one
 * block overlaps the sketch of the previous one. The copy overlaps the caller's host work only for page-locked
 * (pinned) host memory; pageable memory is staged by the CUDA runtime. The host block must stay valid and unchanged
 * until the context's stream has been synchronised (smp_sync, smp_sample, smp_waltmin). Asynchronous. Errors: as
 * smp_sketch_accumulate; SMP_ENOMEM (staging buffers). */
smp_status smp_sketch_accumulate_host(smp_ctx* ctx, const void* A_blk_host, int64_t lda, const void* B_blk_host,
                                      int64_t ldb, int64_t row0, int64_t nrows);

/* Same as smp_sketch_accumulate but with Pi[:, row0:row0+nrows] supplied by the caller (test hook: Pi = I, or
 * the oracle's Pi). Pi_blk_dev is k x nrows row-major with leading dimension ldp, element type float (double for
 * SMP_F64). Runs the context's engine; the SMP_F32 tensor-core engine reads Pi through TMA and needs a 16-byte
 * aligned Pi_blk_dev and ldp % 4 == 0 (SMP_ENGINE_AUTO falls back to the SIMT engine otherwise); the SMP_BF16 one
 * rounds Pi to BF16 into its own buffer first. */
smp_status smp_sketch_accumulate_pi(smp_ctx* ctx, const void* Pi_blk_dev, int64_t ldp, const void* A_blk_dev,
                                    int64_t lda, const void* B_blk_dev, int64_t ldb, int64_t row0, int64_t nrows);

/* Start a new single pass on an existing context: clears the accumulators, the finalized sketch and Omega, keeps
 * every allocation (so a serving loop or a benchmark reuses one context per problem shape). Asynchronous. */
smp_status smp_sketch_reset(smp_ctx* ctx);

/* Close the single pass: reduce the row-split partials in a fixed order (bitwise reproducible), form
 * ||A_i||^2 in double, ||A||_F^2 = sum_i ||A_i||^2 summed left to right, ||At_i|| and the rescale factors
 * (D_A)_ii = ||A_i|| / ||At_i|| (0 when ||At_i|| = 0), the compact form of Eq. (2) (Appendix B). Same for B.
 * Asynchronous. Errors: SMP_ESTATE (twice), SMP_ECUDA. */
smp_status smp_sketch_finalize(smp_ctx* ctx);

/* Borrow the finalized sketch (valid until smp_destroy). At_dev: n1 x ldk row-major (row i = sketch column At_i,
 * k values then padding), Bt_dev: n2 x ldk (== At_dev when same_ab); float, or double for SMP_F64.
 * sA_dev/sB_dev: ||A_i||^2, ||B_j||^2 (double, device). F_host: {||A||_F^2, ||B||_F^2} copied to the host
 * (synchronises). Any output pointer may be NULL. Errors: SMP_ESTATE before finalize. */
smp_status smp_sketch_view(smp_ctx* ctx, const void** At_dev, const void** Bt_dev, int64_t* ldk,
                           const double** sA_dev, const double** sB_dev, double* F_host);

/* Replace the sketch state with caller data (stage-parity and resume hook); marks the context finalized.
 * At_dev: n1 x k row-major, Bt_dev: n2 x k (ignored when same_ab), float (double for SMP_F64); sA_dev, sB_dev:
 * double column sums of squares. Copies; asynchronous. */
smp_status smp_sketch_import(smp_ctx* ctx, const void* At_dev, const void* Bt_dev, const double* sA_dev,
                             const double* sB_dev);

/* Draw Omega (Algorithm 1, step 3): (i, j) is kept iff u_ij < q^_ij = min{1, q_ij}, q_ij = alpha_i + beta_j,
 * alpha_i = m * (||A_i||^2 / ((2 n2) ||A||_F^2)), beta_j = m * (||B_j||^2 / ((2 n1) ||B||_F^2)) (Eq. (1); every
 * step one IEEE binary64 operation in this order, so given the same norms Omega is bit-identical to any
 * implementation that follows it). u_ij = ((x0 >> 5) 2^26 + (x1 >> 6)) 2^-53 from Philox counter (i, j, 0, 2) under
 * key (seed mod 2^32, seed >> 32). m > 0 is the sample budget as a double (no rounding). Builds the context-owned
 * CSR (row-major canonical order) and CSC views of Omega. Synchronises; *nnz_out receives |Omega|.
 * Errors: SMP_ESTATE (before finalize), SMP_EINVAL (m <= 0, both Frobenius norms zero), SMP_ENOMEM. */
smp_status smp_sample(smp_ctx* ctx, double m, uint64_t seed, int64_t* nnz_out);

/* Row-wise multinomial sampling of Omega (Appendix, "Sampling"), the alternative to smp_sample's Bernoulli coins.
 * With alpha_i, beta_j of Eq. (1) as in smp_sample (unclipped q_ij = alpha_i + beta_j): Bcum = inclusive prefix sums
 * of beta (1,024-element blocks summed left to right, each block offset by the left-to-right sum of the earlier
 * blocks' totals); row i has S_i = n2 alpha_i + Bcum_{n2-1} (= the Appendix's m_i) and draws c_i = floor(S_i + 1/2)
 * columns; draw s takes u = the 53-bit Philox uniform of counter (i, s, 0, 5) under key seed, t = u S_i, and the
 * smallest j with t < (j + 1) alpha_i + Bcum_j (j = n2 - 1 if none), i.e. column j with probability q_ij / S_i.
 * Omega is the set of distinct drawn pairs (CSR / CSC exactly as smp_sample builds them); the q^ stored with each
 * pair is (c_i ((alpha_i + beta_j) / S_i)) / count_ij (count_ij = its draws), so smp_waltmin's weight 1/q^ is the
 * unbiased importance weight. Every step is one round-to-nearest binary64 operation in the order written.
 * Synchronises (twice: the draw total, then nnz). Errors: SMP_ESTATE (before finalize), SMP_EINVAL (m <= 0, both
 * Frobenius norms zero), SMP_ENOMEM. */
smp_status smp_sample_multinomial(smp_ctx* ctx, double m, uint64_t seed, int64_t* nnz);

/* smp_sample with caller-supplied column sums of squares (double device arrays of n1 and n2 entries) in place of
 * the sketch's: the stage-parity hook for bit-exact Omega. Does not need a finalized sketch. */
smp_status smp_sample_from_norms(smp_ctx* ctx, const double* sA_dev, const double* sB_dev, double m,
                                 uint64_t seed, int64_t* nnz_out);

/* Borrow Omega (valid until the next smp_sample* or smp_destroy). CSR: row_ptr[n1+1] (int64), col[nnz] (int32,
 * increasing within a row), qhat[nnz] (double q^_ij). CSC: col_ptr[n2+1] (int64), csc_row[nnz] (int32,
 * increasing within a column), csc_pos[nnz] (int64, position of the entry in the CSR arrays). Any output may be
 * NULL. Errors: SMP_ESTATE before sampling. */
smp_status smp_omega_view(const smp_ctx* ctx, int64_t* nnz, const int64_t** row_ptr, const int32_t** col,
                          const double** qhat, const int64_t** col_ptr, const int32_t** csc_row,
                          const int64_t** csc_pos);

/* M~(i, j) = ||A_i|| ||B_j|| <At_i, Bt_j> / (||At_i|| ||Bt_j||) for every (i, j) in Omega, in CSR order
 * (Algorithm 1, step 4; Eq. (2)); 0 when a sketch column is zero. vals_dev: caller device buffer of nnz floats
 * (doubles for SMP_F64). Asynchronous. Errors: SMP_ESTATE (before sampling). */
smp_status smp_estimate(smp_ctx* ctx, void* vals_dev);

/* WAltMin(P_Omega(M~), Omega, r, q^, T) (Algorithm 2) followed by the canonical form of U^ V^T:
 * w_ij = 1/q^_ij; U0 = top-r left singular subspace of R_Omega0(M~) by block subspace iteration (Philox start
 * block, counter (i, 0, c/4, 4) under key seed) with a Rayleigh-Ritz step; trim: row i of U0 is zeroed when
 * ||U0^i|| > 8 sqrt(r) ||A_i|| / ||A||_F; then T rounds of the weighted least-squares V- and U-updates, each row
 * solving (G + lambda I) x = b with G = sum w f f^T, b = sum w M~ f, lambda = 1e-10 tr(G)/r (x = 0 when tr(G) = 0),
 * by a double-precision Cholesky. Finally QR(U^) = Qu Ru, QR(V^) = Qv Rv, SVD(Ru Rv^T) = W S Z^T, U = Qu W,
 * V = Qv Z, the largest-magnitude entry of each U column made positive.
 * vals_dev: P_Omega(M~) in CSR order (float; double for SMP_F64), e.g. from smp_estimate. 1 <= r <= 32,
 * r <= min(n1, n2); T >= 0. flags: SMP_* above. seed: split and start-block key. U_init_dev: n1 x r double,
 * read only with SMP_INIT_GIVEN. Outputs (device, double, row-major): U_dev n1 x r, S_dev r, V_dev n2 x r.
 * Synchronises. Errors: SMP_ESTATE, SMP_EINVAL, SMP_ENUMERIC, SMP_ENOMEM. */
smp_status smp_waltmin(smp_ctx* ctx, const void* vals_dev, int32_t r, int32_t T, uint32_t flags, uint64_t seed,
                       const double* U_init_dev, double* U_dev, double* S_dev, double* V_dev);

/* Baseline SVD(At^T Bt) (Section 4, the comparison of SMP-PCA with the SVD of the sketched product): the top-r
 * singular triplets of M = At^T Bt (At = Pi A: k x n1, Bt = Pi B: k x n2, the finalized sketches), by block power
 * iteration through the factors without forming the n1 x n2 product (the footnote there). Block of b =
 * min(2r + 8, 64, n1, n2, k) columns, Philox start block on the right (counter (j, 0, c/4, 4) under key seed),
 * orthonormalised by Cholesky-QR; each iteration Y = M Z, Y orthonormalised, Z = M^T Y. Every second (binary32
 * sketches) or fourth (binary64) iteration the top-r Ritz vectors U = Y E_r (E: eigenvectors of Z^T Z, binary64
 * Jacobi) and their values (eigenvalues of Z^T Z) are compared with the previous check's; the iteration stops when
 * the vectors move by less than 2e-5 (1e-11) in sqrt(r - ||U^T U_prev||_F^2), when no value changes by more than
 * 2e-7 (1e-14) of the largest, or after 200 (400) iterations. Output: U = Y E_r, S = sqrt(eigenvalues),
 * V = Z E_r / S, the largest-magnitude entry of each U column made positive. Products in the sketch precision
 * (binary32 or binary64), reductions over the long dimension finished in binary64.
 * 1 <= r <= 32, r <= min(n1, n2, k). Outputs (device, double, row-major): U_dev n1 x r, S_dev r, V_dev n2 x r.
 * Synchronises. Errors: SMP_ESTATE (sketch not finalized), SMP_EINVAL, SMP_ENOMEM. */
smp_status smp_sketch_svd(smp_ctx* ctx, int32_t r, uint64_t seed, double* U_dev, double* S_dev, double* V_dev);

/* ---------------------------------------------------------------------------------------------------------------
 * Serving form: a request loop with continuous batching. Each admitted job owns a context (resident sketch state,
 * Omega, scratch) on a CUDA stream of its own; row blocks of many jobs arrive interleaved and sketch concurrently;
 * when a job is closed, one of solve_workers host threads runs finalize, sample (Bernoulli, Eq. (1)), estimate and
 * WAltMin for it on its stream while other jobs keep sketching. Admission is gated by a device-memory budget:
 * a job is admitted only if smp_serve_job_bytes of it fits in the budget left, else SMP_EBUSY. A job's results do
 * not depend on what else runs (its kernels touch only its context; every reduction has a fixed order).
 * Threading: admit / block / close for one job come from one host thread at a time; collect, poll, cancel and
 * stats may come from any thread. The caller keeps each pushed block's memory valid until the job is collected
 * or cancelled.
 * ------------------------------------------------------------------------------------------------------------- */
typedef struct smp_server smp_server;

typedef struct {
    int64_t hbm_budget_bytes;   /* device memory the admitted jobs may hold together (> 0)                       */
    int32_t solve_workers;      /* host threads running the solve chain of closed jobs, 1..64                     */
} smp_server_params;

typedef struct {
    smp_params sketch;          /* the job's sketch context (smp_sketch_begin), stream chosen by the server        */
    int32_t r, T;               /* rank and WAltMin iterations (smp_waltmin)                                      */
    uint32_t flags;             /* smp_waltmin flags                                                              */
    double m;                   /* expected samples (smp_sample)                                                  */
    uint64_t sample_seed, walt_seed;
} smp_job_params;

/* Upper bound on the device bytes a job's context, Omega, scratch and results can hold (the admission charge).
 * Host only. Errors: SMP_EINVAL. */
smp_status smp_serve_job_bytes(const smp_job_params* job, int64_t* bytes);

/* Start a server on the current device with its worker threads. Errors: SMP_EINVAL, SMP_ENOMEM, SMP_ECUDA. */
smp_status smp_serve_create(const smp_server_params* params, smp_server** out);

/* Admit a job: reserve its bytes, create its stream and context. *job_id identifies it until collected or
 * cancelled. Errors: SMP_EBUSY (over budget), SMP_EINVAL, SMP_ENOMEM, SMP_ECUDA, SMP_ESTATE (server stopping). */
smp_status smp_serve_admit(smp_server* server, const smp_job_params* job, int64_t* job_id);

/* Sketch one row block of a streaming job (smp_sketch_accumulate on its context and stream). Asynchronous.
 * Errors: as smp_sketch_accumulate; SMP_EINVAL (unknown job), SMP_ESTATE (job already closed). */
smp_status smp_serve_block(smp_server* server, int64_t job_id, const void* A_blk_dev, int64_t lda,
                           const void* B_blk_dev, int64_t ldb, int64_t row0, int64_t nrows);

/* The job's last block has been pushed: queue its solve chain; its latency clock starts here. */
smp_status smp_serve_close(smp_server* server, int64_t job_id);

/* *done = 1 once the job's solve chain has finished (successfully or not). */
smp_status smp_serve_poll(smp_server* server, int64_t job_id, int32_t* done);

/* Wait for a closed job (timeout_s < 0: no limit; SMP_ETIMEOUT when it runs out, the job stays), copy its factors
 * (U n1 x r, S r, V n2 x r, binary64, canonical form as smp_waltmin) to the caller's device buffers (any may be
 * NULL), report |Omega| and the latency from close to the end of WAltMin, and release the job and its budget.
 * Returns the job's own status when its chain failed. */
smp_status smp_serve_collect(smp_server* server, int64_t job_id, double timeout_s, double* U_dev, double* S_dev,
                             double* V_dev, int64_t* nnz, double* latency_ms);

/* Drop a job in any state (a running solve is allowed to finish first) and release its budget. */
smp_status smp_serve_cancel(smp_server* server, int64_t job_id);

/* Bytes currently charged to admitted jobs and their number. */
smp_status smp_serve_stats(smp_server* server, int64_t* used_bytes, int32_t* live_jobs);

/* Stop the workers (queued jobs are not solved), release every job, free the server. NULL is a no-op. */
smp_status smp_serve_destroy(smp_server* server);

/* Block until the context's stream is idle and report any device-side error word. */
smp_status smp_sync(smp_ctx* ctx);

/* Free the context and everything it owns. NULL is a no-op. */
smp_status smp_destroy(smp_ctx* ctx);

/* One-line description of the last failure on ctx (or of the last failed smp_sketch_begin when ctx is NULL). */
const char* smp_last_error(const smp_ctx* ctx);

/* Name of a status code. */
const char* smp_status_string(smp_status s);

/* Library version, major * 10000 + minor * 100 + patch. */
int32_t smp_version(void);

/* Allocation-free sketch of one row range. The paper has no counterpart: this call exists for callers that hold
 * device buffers but may not allocate device memory themselves, e.g. a plug-in inside a host framework that owns
 * the whole device-memory budget through its own pool, or a latency-critical loop where cudaMalloc / cudaFree would
 * synchronise the device and stall other streams.
 * It computes what smp_sketch_begin + one smp_sketch_accumulate(row0, nrows) + smp_sketch_finalize would (same
 * Philox Pi, same SIMT kernel) and writes it to the caller's device buffers: At_dev (n1 x k row-major, row i =
 * sketch column At_i), Bt_dev (n2 x k), sA_dev (n1 doubles, ||A_i||^2 over the range) and sB_dev (n2 doubles).
 * A_dev / B_dev: nrows x n1 / nrows x n2 row-major, lda >= n1, ldb >= n2, dtype SMP_F32 or SMP_BF16 (others:
 * SMP_EUNSUPPORTED). 1 <= n1, n2 <= 2^30, 1 <= k <= 1024. Asynchronous on stream (a cudaStream_t).
 * Scratch: a fixed array of SMP_NOALLOC_SCRATCH_BYTES (16 MiB) compiled into the library, held on every GPU that
 * loads it until the process exits. The partials need (n1 + n2) * (round_up(k, 4) * 4 + 8) bytes (each part rounded
 * up to 256 bytes); larger shapes are rejected with SMP_EINVAL before anything is launched. The call performs no
 * cudaMalloc / cudaFree. The first call in a CUDA context looks up the array's device address
 * (cudaGetSymbolAddress) in that context and caches it under the context's unique id (so a device reset or a second
 * context on the same device gets a lookup of its own): make that first call before any stream capture. Every call
 * on a device shares the one array and clears the part it uses, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller. */
#define SMP_NOALLOC_SCRATCH_BYTES (16u << 20)
smp_status smp_sketch_noalloc(const void* A_dev, int64_t lda, const void* B_dev, int64_t ldb, int64_t n1,
                              int64_t n2, int32_t k, int32_t dtype, uint64_t seed, int64_t row0, int64_t nrows,
                              float* At_dev, float* Bt_dev, double* sA_dev, double* sB_dev, void* stream);

/* Number of CUDA kernels this library has launched since it was loaded (all contexts, all threads). */
int64_t smp_launch_count(void);

/* Rows accumulated since the context was created or reset: their number, the first row not covered by a
 * contiguous run from row 0 (0 if row 0 is missing), and the number of disjoint ranges (1 for a complete prefix).
 * Host only. */
smp_status smp_sketch_coverage(const smp_ctx* ctx, int64_t* rows, int64_t* first_missing, int64_t* ranges);

/* ---------------------------------------------------------------------------------------------------------------
 * LELA (Section 4, Table 1: the two-pass comparison method). */

/* Pass 1: fold the row block's column sums of squares into the norm accumulators, without a sketch (the
 * compensated binary32 sums of the sketch engines for SMP_F32 and SMP_BF16 blocks, binary64 for SMP_F64, reduced
 * over row splits in a fixed order by smp_sketch_finalize). Same block conventions, checks and row tracking as
 * smp_sketch_accumulate. One pass holds either sketch rows or norms-only rows: mixing them is SMP_ESTATE, and after a
 * norms-only pass smp_estimate and smp_sketch_svd return SMP_ESTATE. Asynchronous. Errors: SMP_EINVAL, SMP_ESTATE,
 * SMP_ECUDA. */
smp_status smp_norms_accumulate(smp_ctx* ctx, const void* A_blk_dev, int64_t lda, const void* B_blk_dev,
                                int64_t ldb, int64_t row0, int64_t nrows);

/* Pass 2: add sum_{t in block} A[t][i] B[t][j] into the exact entry M_ij = A_i^T B_j of every (i, j) in the
 * context's Omega (after smp_sample; drawing a new Omega starts the pass afresh). The blocks must cover the same
 * rows as pass 1 (smp_exact_coverage reports them); a block overlapping rows already added is SMP_EINVAL.
 * SMP_F32 blocks that are 16-byte aligned with lda, ldb % 4 == 0 run on tensor cores (SMP_ENGINE_AUTO or _TC):
 * the block of A is transposed into a context buffer of n1 x max_rows floats (allocated on first use), both operands
 * are rounded to TF32 (round to nearest, ties away), products accumulate in binary32 over a row split of the block
 * and in binary64 across splits and blocks; |error| <= (2^-10 + rows * 2^-23) sum_t |A[t][i] B[t][j]| with rows
 * the block's row count. Other blocks (SMP_F64, SMP_BF16, unaligned, SMP_ENGINE_SIMT) run on the CUDA cores in the
 * context's precision (binary64 for SMP_F64, binary32 otherwise). SMP_ENGINE_TC with a block the tensor-core path
 * cannot take is SMP_EUNSUPPORTED. Asynchronous. Errors: SMP_ESTATE (before sampling), SMP_EINVAL,
 * SMP_EUNSUPPORTED, SMP_ENOMEM, SMP_ECUDA. */
smp_status smp_exact_accumulate(smp_ctx* ctx, const void* A_blk_dev, int64_t lda, const void* B_blk_dev,
                                int64_t ldb, int64_t row0, int64_t nrows);

/* The exact entries in CSR order (the order of smp_estimate's output, ready for smp_waltmin): the row splits
 * summed in a fixed order. vals_dev: caller device buffer of nnz floats (doubles for SMP_F64). Asynchronous.
 * Errors: SMP_ESTATE (no Omega, or no smp_exact_accumulate since it was drawn), SMP_EINVAL. */
smp_status smp_exact_values(smp_ctx* ctx, void* vals_dev);

/* Rows added by smp_exact_accumulate since Omega was drawn, as smp_sketch_coverage. Host only. */
smp_status smp_exact_coverage(const smp_ctx* ctx, int64_t* rows, int64_t* first_missing, int64_t* ranges);

/* Fault injection for tests: the next n device allocations made by the library fail (the calls that made them
 * return SMP_ENOMEM and leave the context usable or destroyable). n <= 0 clears it. Process-wide. */
void smp_debug_fail_allocs(int32_t n);

/* Test hook of the bounded device-side waits (failure detection; the paper has no counterpart):
 * every mbarrier wait of the TF32 / BF16-operand tensor-core sketch kernel (SMP_ENGINE_TC with SMP_F32 blocks,
 * SMP_ENGINE_TC_BF16) gives up after wait_ns nanoseconds (<= 0: the default of 2 s); if skip_stage >= 0, the next
 * such launch issues no data loads from pipeline stage skip_stage on, so the waits on that stage run out: the
 * kernel then records DEVERR_TIMEOUT in the context's error word, lets its loads and MMAs in flight finish, frees
 * its tensor memory and returns, the next synchronising call returns SMP_ETIMEOUT, and the context stays usable
 * (smp_sketch_reset, then accumulate again). The skip applies to one launch; the limit stays until changed.
 * Process-wide. */
void smp_debug_tc_wait(int64_t wait_ns, int32_t skip_stage);

#ifdef __cplusplus
}
#endif
#endif /* SMP_H */
