"""Plain CPU binary64 oracle for SMP-PCA (Wu, Bhojanapalli, Sanghavi, Dimakis, "Single Pass PCA of Matrix
Products", arXiv 1610.06656).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or links this module; only `tests/`,
`__graft_entry__.smoke()` and the `cpu_baseline` / `--impl reference` legs of `bench.py` use it. It shares no
code with the CUDA path: the only common module is the seeded input generator, which holds none of the method's
arithmetic.

Each function follows one step of Algorithm 1 (SMP-PCA) or Algorithm 2 (WAltMin, Appendix A) in the paper's
order and notation, in binary64, with Pi materialised explicitly block by block. Library primitives used as
steps: numpy matmul, numpy/LAPACK SVD, QR and linear solve. Where the paper is silent the reading is stated in
the docstring; the same reading binds the CUDA path.

Parity pins live in tests/test_oracle_*.py; every function here is pinned there (none is "parity unpinned").
"""
import math

import numpy as np

from . import philox

SPLIT_NONE = 0
SPLIT_OMEGA = 1


# --------------------------------------------------------------------------------------------------------------
# Step 1 (Algorithm 1, step 2; Section 2.1 "Step 1"): one pass forming Pi A, Pi B and the column norms.
# --------------------------------------------------------------------------------------------------------------
class SketchState:
    """Accumulators of the single pass: At = Pi A (k x n1), Bt = Pi B (k x n2), sA_i = ||A_i||^2, sB_j = ||B_j||^2."""

    def __init__(self, n1, n2, k, seed, same_ab=False):
        self.n1, self.n2, self.k, self.seed, self.same_ab = n1, n2, k, seed, same_ab
        self.At = np.zeros((k, n1))
        self.Bt = self.At if same_ab else np.zeros((k, n2))
        self.sA = np.zeros(n1)
        self.sB = self.sA if same_ab else np.zeros(n2)
        self.rows_seen = 0

    def accumulate(self, A_blk, B_blk, row0, pi_blk=None):
        """Add the contribution of data rows [row0, row0 + R): At += Pi[:, rows] A[rows, :], and the squares.

        The rows may arrive in any order (Section 1, last contribution; Section 5): row0 selects Pi's columns.
        pi_blk (k x R), when given, replaces the Philox Pi (explicit-Pi test mode, e.g. Pi = I).
        """
        A_blk = np.asarray(A_blk, dtype=np.float64)
        R = A_blk.shape[0]
        P = philox.pi_block(self.seed, self.k, row0, R) if pi_blk is None else np.asarray(pi_blk, np.float64)
        self.At += P @ A_blk
        self.sA += np.sum(A_blk * A_blk, axis=0)
        if not self.same_ab:
            B_blk = np.asarray(B_blk, dtype=np.float64)
            self.Bt += P @ B_blk
            self.sB += np.sum(B_blk * B_blk, axis=0)
        self.rows_seen += R


def fwht(X):
    """Unnormalised fast Walsh-Hadamard transform along axis 0 (length a power of two), Sylvester order:
    Y[s] = sum_t (-1)^popcount(s & t) X[t]. Butterflies of span 1, 2, 4, ... in binary64."""
    Y = np.array(X, dtype=np.float64, copy=True)
    n = Y.shape[0]
    h = 1
    while h < n:
        Y = Y.reshape((n // (2 * h), 2, h) + Y.shape[1:])
        a = Y[:, 0].copy()
        Y[:, 0] = a + Y[:, 1]
        Y[:, 1] = a - Y[:, 1]
        Y = Y.reshape((n,) + Y.shape[3:])
        h *= 2
    return Y


def srht_signs(seed, t0, nrows):
    """D_tt = +-1 for data rows t0 .. t0 + nrows - 1 (bit 0 of the Philox word x0 set: -1)."""
    k0, k1 = philox.seed_key(seed)
    t = np.arange(t0, t0 + nrows, dtype=np.uint64)
    x0, _, _, _ = philox.philox4x32_10(t & np.uint64(philox.MASK32), t >> np.uint64(32), np.uint64(0),
                                       np.uint64(philox.TAG_SRHT_SIGN), k0, k1)
    return np.where((x0 & np.uint64(1)) != 0, -1.0, 1.0)


def srht_rows(seed, b, k, p):
    """The k Hadamard rows block b samples (uniformly, with replacement): the top p bits of x0."""
    k0, k1 = philox.seed_key(seed)
    a = np.arange(k, dtype=np.uint64)
    x0, _, _, _ = philox.philox4x32_10(a, np.uint64(b & philox.MASK32), np.uint64(b >> 32),
                                       np.uint64(philox.TAG_SRHT_ROW), k0, k1)
    return (x0 >> np.uint64(32 - p)).astype(np.int64)


def sketch_srht(A, B, k, seed, block_log2, same_ab=False):
    """Step 1 with a block subsampled randomized Hadamard transform as Pi (Section 4: the Spark implementation's
    sketch; its footnote: O(nd log d) time and O(d) space instead of O(ndk) and O(dk)).

    Reading (the paper cites the SRHT without a streaming form): the data rows are cut into blocks of R = 2^p rows
    (block b = rows [bR, (b+1)R), the last one zero-padded) and Pi = [Pi_0, Pi_1, ...] with independent
    Pi_b = k^-1/2 S_b H_R D_b: D_b the random signs of srht_signs, H_R the unnormalised Walsh-Hadamard matrix, S_b
    k rows of H_R drawn uniformly with replacement (srht_rows); E[Pi^T Pi] = I. So
    At = sum_b k^-1/2 (H_R D_b A_b)[S_b, :], each block through fwht. Norms as in sketch(). Returns a SketchState.
    """
    A = np.asarray(A, dtype=np.float64)
    d, n1 = A.shape
    B = A if same_ab else np.asarray(B, dtype=np.float64)
    n2 = B.shape[1]
    R = 1 << block_log2
    st = SketchState(n1, n2, k, seed, same_ab)
    inv = 1.0 / np.sqrt(float(k))
    for b, t0 in enumerate(range(0, d, R)):
        rows = min(R, d - t0)
        D = srht_signs(seed, t0, rows)[:, None]
        S = srht_rows(seed, b, k, block_log2)
        XA = np.zeros((R, n1))
        XA[:rows] = D * A[t0:t0 + rows]
        st.At += inv * fwht(XA)[S]
        st.sA += np.sum(A[t0:t0 + rows] ** 2, axis=0)
        if not same_ab:
            XB = np.zeros((R, n2))
            XB[:rows] = D * B[t0:t0 + rows]
            st.Bt += inv * fwht(XB)[S]
            st.sB += np.sum(B[t0:t0 + rows] ** 2, axis=0)
        st.rows_seen += rows
    return st


def frobenius_sq(s):
    """||A||_F^2 = sum_i ||A_i||^2, summed strictly left to right (the order the sampler's reading fixes)."""
    total = 0.0
    for v in np.asarray(s, dtype=np.float64):
        total = total + float(v)
    return total


def sketch(A, B, k, seed, block_rows=65536, same_ab=False, pi=None):
    """Run the whole single pass over A (d x n1) and B (d x n2) in row blocks; returns the SketchState."""
    A = np.asarray(A)
    d, n1 = A.shape
    n2 = n1 if same_ab else np.asarray(B).shape[1]
    st = SketchState(n1, n2, k, seed, same_ab)
    for r0 in range(0, d, block_rows):
        r1 = min(d, r0 + block_rows)
        st.accumulate(A[r0:r1], None if same_ab else B[r0:r1], r0, None if pi is None else pi[:, r0:r1])
    return st


def rescale_factors(Xt, s):
    """(D_X)_ii = ||X_i|| / ||Xt_i||: the compact form M~ = D_A At^T Bt D_B (Appendix B, stated just before the
    lemma that bounds |M~_ij - A_i^T B_j|).

    Reading: a column whose sketch is exactly zero gets D = 0, so its estimates are 0.
    """
    norm_true = np.sqrt(np.asarray(s, dtype=np.float64))
    norm_sk = np.sqrt(np.sum(Xt * Xt, axis=0))
    D = np.zeros_like(norm_true)
    nz = norm_sk > 0
    D[nz] = norm_true[nz] / norm_sk[nz]
    return D


# --------------------------------------------------------------------------------------------------------------
# Step 2a (Algorithm 1, step 3; Eq. (1)): biased Bernoulli sampling of Omega.
# --------------------------------------------------------------------------------------------------------------
def sampling_terms(sA, sB, m):
    """alpha_i = m * (||A_i||^2 / (2 n2 ||A||_F^2)), beta_j = m * (||B_j||^2 / (2 n1 ||B||_F^2)), so q_ij = alpha_i + beta_j.

    Eq. (1) exactly as printed (the A-term normalised by n2, the B-term by n1). Every step is one IEEE binary64
    operation in this order. Reading: if ||A||_F = 0 the A-term is 0 (likewise B).
    """
    sA = np.asarray(sA, dtype=np.float64)
    sB = np.asarray(sB, dtype=np.float64)
    n1, n2 = sA.shape[0], sB.shape[0]
    FA, FB = frobenius_sq(sA), frobenius_sq(sB)
    m = float(m)
    alpha = m * (sA / (float(2 * n2) * FA)) if FA > 0 else np.zeros(n1)
    beta = m * (sB / (float(2 * n1) * FB)) if FB > 0 else np.zeros(n2)
    return alpha, beta


def q_matrix(sA, sB, m):
    """Dense q_ij (unclipped) and q^_ij = min{1, q_ij} (Algorithm 1, step 3)."""
    alpha, beta = sampling_terms(sA, sB, m)
    q = alpha[:, None] + beta[None, :]
    return q, np.minimum(1.0, q)


def sample_omega(sA, sB, m, seed):
    """Keep (i, j) independently iff u_ij < q^_ij (strict), u_ij the 53-bit Philox uniform of (i, j).

    Returns Omega in canonical row-major order as (rows, cols, qhat) arrays (int64, int64, float64).
    """
    sA = np.asarray(sA, dtype=np.float64)
    sB = np.asarray(sB, dtype=np.float64)
    n1, n2 = sA.shape[0], sB.shape[0]
    _, qhat = q_matrix(sA, sB, m)
    rows_out, cols_out, q_out = [], [], []
    jj = np.arange(n2, dtype=np.uint64)
    for i in range(n1):
        u = philox.coin_uniforms(seed, philox.TAG_SAMPLE, np.uint64(i), jj)
        keep = np.nonzero(u < qhat[i])[0]
        rows_out.append(np.full(keep.shape[0], i, dtype=np.int64))
        cols_out.append(keep.astype(np.int64))
        q_out.append(qhat[i, keep])
    return np.concatenate(rows_out), np.concatenate(cols_out), np.concatenate(q_out)


PREFIX_BLOCK = 1024


def blocked_prefix(x):
    """Inclusive prefix sums of x in the order both sides of the parity tests follow (a reading: the paper fixes no
    order): sequential left-to-right sums within blocks of PREFIX_BLOCK elements, each block's sums then offset by the
    sequential sum of the earlier blocks' totals (one binary64 addition per element; the first block's offset is 0)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    offset = 0.0
    for b0 in range(0, x.shape[0], PREFIX_BLOCK):
        w = np.cumsum(x[b0:b0 + PREFIX_BLOCK])        # np.add.accumulate: strictly left to right
        out[b0:b0 + PREFIX_BLOCK] = offset + w
        offset = offset + float(w[-1])
    return out


def sample_omega_multinomial(sA, sB, m, seed):
    """Row-wise multinomial sampling of Omega (Appendix, "Sampling"), the O(m log n) alternative to the Bernoulli
    coins. Row i expects m_i = sum_j q_ij draws (q_ij = alpha_i + beta_j of Eq. (1), unclipped) and draws column j
    with probability q~_ij = q_ij / m_i, located by binary search on the row's CDF, whose entries are a linear
    shift and scale of one shared prefix sum of beta.

    Readings (binding for both sides):
      * S_i = n2 alpha_i + Bcum_{n2-1} with Bcum = blocked_prefix(beta); draws per row c_i = floor(S_i + 1/2);
      * draw s of row i: u = the 53-bit Philox uniform of counter (i, s, 0, TAG_MULTI), t = u S_i, and the column
        is the smallest j with t < (j + 1) alpha_i + Bcum_j (the last column if none);
      * Omega is the set of distinct drawn pairs, count_ij the number of draws of (i, j); the effective probability
        stored with each pair is q^_ij = (c_i ((alpha_i + beta_j) / S_i)) / count_ij, so the WAltMin weight
        1 / q^_ij = count_ij / (c_i q~_ij) has expectation 1 per entry, as 1 / q^ does for the Bernoulli coins.
    Every step is one IEEE binary64 operation in the order written. Returns (rows, cols, qhat, counts) in
    canonical row-major order.
    """
    alpha, beta = sampling_terms(sA, sB, m)
    n1, n2 = alpha.shape[0], beta.shape[0]
    Bcum = blocked_prefix(beta)
    jp1 = np.arange(1, n2 + 1, dtype=np.float64)
    rows_out, cols_out, q_out, c_out = [], [], [], []
    for i in range(n1):
        S = float(n2) * alpha[i] + Bcum[-1]
        c = int(np.floor(S + 0.5))
        if c == 0:
            continue
        u = philox.coin_uniforms(seed, philox.TAG_MULTI, np.uint64(i), np.arange(c, dtype=np.uint64))
        t = u * S
        cdf = jp1 * alpha[i] + Bcum                    # non-decreasing: (j + 1) alpha_i + Bcum_j
        j = np.minimum(np.searchsorted(cdf, t, side="right"), n2 - 1)
        counts = np.bincount(j, minlength=n2)
        keep = np.nonzero(counts)[0]
        cnt = counts[keep]
        rows_out.append(np.full(keep.shape[0], i, dtype=np.int64))
        cols_out.append(keep.astype(np.int64))
        q_out.append((float(c) * ((alpha[i] + beta[keep]) / S)) / cnt.astype(np.float64))
        c_out.append(cnt.astype(np.int64))
    if not rows_out:
        e = np.zeros(0, dtype=np.int64)
        return e, e, np.zeros(0), e
    return np.concatenate(rows_out), np.concatenate(cols_out), np.concatenate(q_out), np.concatenate(c_out)


# --------------------------------------------------------------------------------------------------------------
# Step 2b (Algorithm 1, step 4; Eq. (2)): rescaled JL estimate over Omega.
# --------------------------------------------------------------------------------------------------------------
def estimate(rows, cols, At, Bt, sA, sB):
    """M~(i, j) = ||A_i|| ||B_j|| <At_i, Bt_j> / (||At_i|| ||Bt_j||) for (i, j) in Omega (Eq. (2)).

    Reading: if ||At_i|| = 0 or ||Bt_j|| = 0 the estimate is 0.
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    nA = np.sqrt(np.asarray(sA, dtype=np.float64))
    nB = np.sqrt(np.asarray(sB, dtype=np.float64))
    nAt = np.sqrt(np.sum(At * At, axis=0))
    nBt = np.sqrt(np.sum(Bt * Bt, axis=0))
    dots = np.einsum('ke,ke->e', At[:, rows], Bt[:, cols])
    den = nAt[rows] * nBt[cols]
    out = np.zeros(rows.shape[0])
    ok = den > 0
    out[ok] = nA[rows[ok]] * nB[cols[ok]] * (dots[ok] / den[ok])
    return out


# --------------------------------------------------------------------------------------------------------------
# Step 3 (Algorithm 1, step 5; Algorithm 2, Appendix A): WAltMin.
# --------------------------------------------------------------------------------------------------------------
def weights(qhat):
    """w_ij = 1/q^_ij when q^_ij > 0, else 0 (Algorithm 2, step 2)."""
    qhat = np.asarray(qhat, dtype=np.float64)
    w = np.zeros_like(qhat)
    pos = qhat > 0
    w[pos] = 1.0 / qhat[pos]
    return w


def split_subsets(rows, cols, T, seed):
    """Subset id in [0, 2T] of each sample (Algorithm 2, step 3).

    Reading: "equal uniformly random subsets" is taken as each sample joining subset floor(u * (2T+1)) with
    u the 53-bit Philox split uniform of (i, j): every subset is uniformly random and equal in expected size.
    """
    u = philox.coin_uniforms(seed, philox.TAG_SPLIT, np.asarray(rows, np.uint64), np.asarray(cols, np.uint64))
    sub = np.floor(u * float(2 * T + 1)).astype(np.int64)
    return np.minimum(sub, 2 * T)


def trim(U0, sA, FA):
    """Zero row i of U0 when ||U0^i|| > 8 sqrt(r) ||A_i|| / ||A||_F (Algorithm 2, step 6).

    The paper leaves the threshold to the LELA paper; the reading takes the row-norm bound the analysis states
    for the initial iterate (Appendix C, the corollary quoted after the proof of the Initialization lemma).
    """
    r = U0.shape[1]
    thr = 8.0 * math.sqrt(r) * np.sqrt(np.asarray(sA, np.float64)) / math.sqrt(FA) if FA > 0 else np.zeros(U0.shape[0])
    rn = np.sqrt(np.sum(U0 * U0, axis=1))
    out = U0.copy()
    out[rn > thr] = 0.0
    return out


RIDGE = 1e-10


def weighted_ls(n_out, idx_out, idx_in, vals, w, F):
    """x_o = argmin_x sum_{e : idx_out[e] = o} w_e (F[idx_in[e]] . x - vals_e)^2 for every output index o.

    One half-step of Algorithm 2 (steps 8 / 9) written as its per-row normal equations
    (sum_e w_e f_e f_e^T) x = sum_e w_e vals_e f_e. Reading for rows the paper leaves undefined: a ridge
    lambda = 1e-10 * trace(G) / r is added, and a row with trace(G) = 0 (no samples, or all-zero factors)
    gets x = 0.
    """
    r = F.shape[1]
    X = np.zeros((n_out, r))
    idx_out = np.asarray(idx_out, dtype=np.int64)
    order = np.argsort(idx_out, kind='stable')
    bounds = np.searchsorted(idx_out[order], np.arange(n_out + 1))
    for o in range(n_out):
        sel = order[bounds[o]:bounds[o + 1]]
        if sel.shape[0] == 0:
            continue
        Fo = F[idx_in[sel]]
        we = w[sel]
        G = (Fo * we[:, None]).T @ Fo
        b = Fo.T @ (we * vals[sel])
        tr = float(np.trace(G))
        if tr == 0.0:
            continue
        X[o] = np.linalg.solve(G + (RIDGE * tr / r) * np.eye(r), b)
    return X


def waltmin(n1, n2, rows, cols, vals, qhat, r, T, sA, split=SPLIT_NONE, split_seed=0, U_init=None):
    """WAltMin(P_Omega(M~), Omega, r, q^, T) -> (U^(T), V^(T)) (Algorithm 2).

    split = SPLIT_NONE (default reading): every half-step and the initial SVD use all of Omega, as the paper's
    Spark implementation's ALS did (Section 4). split = SPLIT_OMEGA divides Omega into 2T+1 subsets as step 3
    says. U_init (n1 x r), when given, replaces the trimmed initial SVD (stage-parity hook).
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    w = weights(qhat)
    if split == SPLIT_OMEGA:
        sub = split_subsets(rows, cols, T, split_seed)
        subset = lambda s: sub == s  # noqa: E731
    else:
        everything = np.ones(rows.shape[0], dtype=bool)
        subset = lambda s: everything  # noqa: E731
    if U_init is None:
        s0 = subset(0)
        R0 = np.zeros((n1, n2))
        R0[rows[s0], cols[s0]] = w[s0] * vals[s0]           # R_Omega0(M~) = w .* P_Omega0(M~) (step 4)
        Usvd, _, _ = np.linalg.svd(R0, full_matrices=False)  # SVD(R_Omega0(M~), r) (step 5)
        U = trim(Usvd[:, :r], sA, frobenius_sq(sA))          # step 6
    else:
        U = np.asarray(U_init, dtype=np.float64).copy()
    V = np.zeros((n2, r))
    for t in range(T):                                       # steps 7-10
        s = subset(2 * t + 1)
        V = weighted_ls(n2, cols[s], rows[s], vals[s], w[s], U)
        s = subset(2 * t + 2)
        U = weighted_ls(n1, rows[s], cols[s], vals[s], w[s], V)
    return U, V


def sign_rule(U, V):
    """Sign reading of the canonical form: the largest-magnitude entry of each column of U is positive (ties: the
    lowest row index); the matching column of V flips with it. In place; returns (U, V)."""
    for c in range(U.shape[1]):
        i = int(np.argmax(np.abs(U[:, c])))
        if U[i, c] < 0:
            U[:, c] = -U[:, c]
            V[:, c] = -V[:, c]
    return U, V


def canonical(U, V):
    """Canonical form of U V^T: QR(U) = Qu Ru, QR(V) = Qv Rv, SVD(Ru Rv^T) = W S Z^T -> (Qu W, S, Qv Z), with the
    sign reading of sign_rule."""
    Qu, Ru = np.linalg.qr(U)
    Qv, Rv = np.linalg.qr(V)
    W, S, Zt = np.linalg.svd(Ru @ Rv.T)
    Uc, Vc = sign_rule(Qu @ W, Qv @ Zt.T)
    return Uc, S, Vc


def sketch_svd(At, Bt, r):
    """Baseline SVD(A~^T B~) (Section 4, the comparison of SMP-PCA with the SVD of the sketched product): the top-r
    singular triplets of A~^T B~ (A~ = At: k x n1, B~ = Bt: k x n2). The paper computes them by power iteration
    without forming the n1 x n2 product (footnote there); power iteration converges to this plain definition, which
    is written out here: the dense product in binary64, its LAPACK SVD truncated to r, the sign reading of
    sign_rule."""
    M = np.asarray(At, dtype=np.float64).T @ np.asarray(Bt, dtype=np.float64)
    W, S, Zt = np.linalg.svd(M, full_matrices=False)
    U, V = sign_rule(W[:, :r].copy(), Zt[:r].T.copy())
    return U, S[:r].copy(), V


def spectral_error(M, U, S, V):
    """||M - U diag(S) V^T|| / ||M|| in the spectral norm (Section 4, the y-axis of Fig. 4(b))."""
    return float(np.linalg.norm(M - (U * S) @ V.T, 2) / np.linalg.norm(M, 2))


def optimal_error(M, r):
    """Eckart-Young: the best rank-r spectral error sigma_{r+1} / sigma_1 ("Optimal" in Table 1)."""
    s = np.linalg.svd(M, compute_uv=False)
    return float(s[r] / s[0]) if s.shape[0] > r else 0.0


def default_m(n1, n2, r):
    """m = 4 n r log n with n = max(n1, n2) and the natural log (Section 4, default parameters)."""
    n = max(n1, n2)
    return 4.0 * n * r * math.log(n)


def smp_pca(A, B, r, k, m, T, seed, sample_seed, block_rows=65536, same_ab=False, split=SPLIT_NONE,
            split_seed=0, pi=None, sampler="bernoulli", srht_log2=None):
    """Algorithm 1 end to end. Returns a dict with every intermediate and the canonical (U, S, V). sampler:
    "bernoulli" (Eq. (1) coins, step 3) or "multinomial" (the Appendix's row-wise sampling). srht_log2: sketch
    with the block SRHT of 2^srht_log2-row blocks instead of the Gaussian Pi."""
    if srht_log2 is not None:
        st = sketch_srht(A, B, k, seed, srht_log2, same_ab)
    else:
        st = sketch(A, B, k, seed, block_rows, same_ab, pi)
    if sampler == "multinomial":
        rows, cols, qhat, _ = sample_omega_multinomial(st.sA, st.sB, m, sample_seed)
    else:
        rows, cols, qhat = sample_omega(st.sA, st.sB, m, sample_seed)
    vals = estimate(rows, cols, st.At, st.Bt, st.sA, st.sB)
    Uh, Vh = waltmin(st.n1, st.n2, rows, cols, vals, qhat, r, T, st.sA, split, split_seed)
    U, S, V = canonical(Uh, Vh)
    return dict(state=st, rows=rows, cols=cols, qhat=qhat, vals=vals, Uhat=Uh, Vhat=Vh, U=U, S=S, V=V)


# --------------------------------------------------------------------------------------------------------------
# LELA, the two-pass method SMP-PCA is compared with (Section 1; Section 4, Table 1 and Fig. 5(a)): a first pass
# for the column norms, Omega drawn from the same q_ij (Eq. (1), which SMP-PCA takes over from LELA), a second pass
# for the exact entries of A^T B on Omega, then the same WAltMin (Algorithm 2).
# --------------------------------------------------------------------------------------------------------------
def column_norms_sq(A, B, same_ab=False):
    """Pass 1: ||A_i||^2 and ||B_j||^2 over all d rows (the norms alone, no sketch)."""
    A = np.asarray(A, dtype=np.float64)
    sA = np.einsum("ti,ti->i", A, A)
    if same_ab:
        return sA, sA
    B = np.asarray(B, dtype=np.float64)
    return sA, np.einsum("tj,tj->j", B, B)


def exact_entries(rows, cols, A, B, chunk=1 << 14):
    """Pass 2: M_ij = A_i^T B_j for every (i, j) of Omega, in the order of rows / cols."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    out = np.empty(len(rows))
    for s in range(0, len(rows), chunk):
        r, c = rows[s:s + chunk], cols[s:s + chunk]
        out[s:s + chunk] = np.einsum("te,te->e", A[:, r], B[:, c])
    return out


def lela(A, B, r, m, T, sample_seed, same_ab=False, split=SPLIT_NONE, split_seed=0, sampler="bernoulli"):
    """LELA end to end: pass 1 norms, Omega (Bernoulli coins of Eq. (1), or the Appendix's row-wise multinomial
    draws), pass 2 exact entries, WAltMin on them. Returns the same dict layout as smp_pca (no sketch state)."""
    A = np.asarray(A, dtype=np.float64)
    Bm = A if same_ab else np.asarray(B, dtype=np.float64)
    sA, sB = column_norms_sq(A, Bm, same_ab)
    if sampler == "multinomial":
        rows, cols, qhat, _ = sample_omega_multinomial(sA, sB, m, sample_seed)
    else:
        rows, cols, qhat = sample_omega(sA, sB, m, sample_seed)
    vals = exact_entries(rows, cols, A, Bm)
    Uh, Vh = waltmin(A.shape[1], Bm.shape[1], rows, cols, vals, qhat, r, T, sA, split, split_seed)
    U, S, V = canonical(Uh, Vh)
    return dict(sA=sA, sB=sB, rows=rows, cols=cols, qhat=qhat, vals=vals, Uhat=Uh, Vhat=Vh, U=U, S=S, V=V)
