"""Algorithm 1 end to end through libsmp on device tensors (a sequence of C-ABI calls; no host compute)."""
import math

import torch

from . import smp as S

_DTYPES = {torch.float32: S.SMP_F32, torch.bfloat16: S.SMP_BF16, torch.float64: S.SMP_F64}


def default_m(n1, n2, r):
    """m = 4 n r ln n, n = max(n1, n2) (Section 4 default sampling budget)."""
    n = max(n1, n2)
    return 4.0 * n * r * math.log(n)


class Solver:
    """One reusable context for problems of a fixed shape (n1, n2, k, dtype): each solve() is one full pass of
    Algorithm 1 over the row blocks it is given."""

    def __init__(self, n1, n2, k, dtype=torch.float32, seed=1, same_ab=False, engine=S.SMP_ENGINE_AUTO,
                 max_rows=65536, stream=None):
        self.n1, self.n2, self.k, self.same_ab = n1, n2, k, same_ab
        self.dtype = dtype
        self.stream = stream
        self.ctx = S.smp_sketch_begin(n1, n2, k, seed, _DTYPES[dtype], same_ab, engine, max_rows, stream)
        self.val_dtype = torch.float64 if dtype == torch.float64 else torch.float32

    def close(self):
        if self.ctx:
            S.smp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sketch(self, A, B=None, block_rows=65536, reset=True, order=None):
        """Stream A, B (d x n, row-major device tensors) through smp_sketch_accumulate in row blocks."""
        if reset:
            S.smp_sketch_reset(self.ctx)
        d = A.shape[0]
        starts = list(range(0, d, block_rows)) if order is None else order
        for r0 in starts:
            r1 = min(d, r0 + block_rows)
            a = A[r0:r1]
            b = None if self.same_ab else B[r0:r1]
            S.smp_sketch_accumulate(self.ctx, a, A.stride(0), b, 0 if b is None else B.stride(0), r0, r1 - r0)
        S.smp_sketch_finalize(self.ctx)

    def sample(self, m, seed=2, sampler="bernoulli"):
        """Omega by the Bernoulli coins of Eq. (1) (smp_sample) or row-wise multinomial draws (Appendix)."""
        if sampler == "multinomial":
            return S.smp_sample_multinomial(self.ctx, m, seed)
        return S.smp_sample(self.ctx, m, seed)

    def estimate(self, nnz):
        vals = torch.empty(max(nnz, 1), dtype=self.val_dtype, device="cuda")
        S.smp_estimate(self.ctx, vals)
        return vals[:nnz]

    def waltmin(self, vals, r, T, flags=0, seed=3, U_init=None):
        U = torch.empty(self.n1, r, dtype=torch.float64, device="cuda")
        Sv = torch.empty(r, dtype=torch.float64, device="cuda")
        V = torch.empty(self.n2, r, dtype=torch.float64, device="cuda")
        S.smp_waltmin(self.ctx, vals, r, T, flags, seed, U_init, U, Sv, V)
        return U, Sv, V

    def sketch_svd(self, r, seed=4):
        """Baseline SVD(At^T Bt) of the finalized sketches (smp_sketch_svd): U (n1 x r), S (r), V (n2 x r)."""
        U = torch.empty(self.n1, r, dtype=torch.float64, device="cuda")
        Sv = torch.empty(r, dtype=torch.float64, device="cuda")
        V = torch.empty(self.n2, r, dtype=torch.float64, device="cuda")
        S.smp_sketch_svd(self.ctx, r, seed, U, Sv, V)
        return U, Sv, V

    def solve(self, A, B, r, T, m=None, sample_seed=2, walt_seed=3, flags=0, block_rows=65536, sampler="bernoulli"):
        m = default_m(self.n1, self.n2, r) if m is None else m
        self.sketch(A, B, block_rows)
        nnz = self.sample(m, sample_seed, sampler)
        vals = self.estimate(nnz)
        U, Sv, V = self.waltmin(vals, r, T, flags, walt_seed)
        return dict(U=U, S=Sv, V=V, nnz=nnz, vals=vals)

    def norms(self, A, B=None, block_rows=65536, reset=True):
        """LELA's first pass: stream A, B through smp_norms_accumulate (column norms only), then finalize."""
        if reset:
            S.smp_sketch_reset(self.ctx)
        for r0 in range(0, A.shape[0], block_rows):
            r1 = min(A.shape[0], r0 + block_rows)
            b = None if self.same_ab else B[r0:r1]
            S.smp_norms_accumulate(self.ctx, A[r0:r1], A.stride(0), b, 0 if b is None else B.stride(0), r0, r1 - r0)
        S.smp_sketch_finalize(self.ctx)

    def exact(self, A, B=None, block_rows=65536):
        """LELA's second pass over the drawn Omega: the exact entries A_i^T B_j in CSR order."""
        for r0 in range(0, A.shape[0], block_rows):
            r1 = min(A.shape[0], r0 + block_rows)
            b = None if self.same_ab else B[r0:r1]
            S.smp_exact_accumulate(self.ctx, A[r0:r1], A.stride(0), b, 0 if b is None else B.stride(0), r0, r1 - r0)
        nnz = S.smp_omega_view(self.ctx)["nnz"]
        vals = torch.empty(max(nnz, 1), dtype=self.val_dtype, device="cuda")
        S.smp_exact_values(self.ctx, vals)
        return vals[:nnz]

    def lela(self, A, B, r, T, m=None, sample_seed=2, walt_seed=3, flags=0, block_rows=65536, sampler="bernoulli"):
        """LELA end to end (Section 4): norms pass, Omega, exact-entry pass, WAltMin."""
        m = default_m(self.n1, self.n2, r) if m is None else m
        self.norms(A, B, block_rows)
        nnz = self.sample(m, sample_seed, sampler)
        vals = self.exact(A, B, block_rows)
        U, Sv, V = self.waltmin(vals, r, T, flags, walt_seed)
        return dict(U=U, S=Sv, V=V, nnz=nnz, vals=vals)

    def omega(self):
        """Omega as torch tensors copied from the context's device arrays (CSR and CSC)."""
        v = S.smp_omega_view(self.ctx)
        nnz = v["nnz"]
        return dict(
            nnz=nnz,
            row_ptr=_wrap(v["row_ptr"], self.n1 + 1, torch.int64),
            col=_wrap(v["col"], nnz, torch.int32),
            qhat=_wrap(v["qhat"], nnz, torch.float64),
            col_ptr=_wrap(v["col_ptr"], self.n2 + 1, torch.int64),
            csc_row=_wrap(v["csc_row"], nnz, torch.int32),
            csc_pos=_wrap(v["csc_pos"], nnz, torch.int64),
        )

    def sketch_state(self):
        At, Bt, ldk, sA, sB, F = S.smp_sketch_view(self.ctx)
        el = torch.float64 if self.dtype == torch.float64 else torch.float32
        At_t = _wrap(At, self.n1 * ldk, el).view(self.n1, ldk)[:, :self.k]
        Bt_t = _wrap(Bt, self.n2 * ldk, el).view(self.n2, ldk)[:, :self.k]
        return dict(At=At_t, Bt=Bt_t, sA=_wrap(sA, self.n1, torch.float64), sB=_wrap(sB, self.n2, torch.float64),
                    F=F)


def _wrap(ptr, n, dtype):
    """Copy n elements at a device pointer into a new torch tensor (device-to-device memcpy in torch)."""
    out = torch.empty(max(n, 0), dtype=dtype, device="cuda")
    if n > 0:
        import ctypes
        cudart = _cudart()
        nbytes = n * out.element_size()
        err = cudart.cudaMemcpy(ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ptr), ctypes.c_size_t(nbytes), 3)
        if err != 0:
            raise RuntimeError("cudaMemcpy failed: %d" % err)
    return out


_CUDART = None


def _cudart():
    global _CUDART
    if _CUDART is None:
        import ctypes
        import ctypes.util
        for name in ("libcudart.so", "libcudart.so.13", ctypes.util.find_library("cudart")):
            if not name:
                continue
            try:
                _CUDART = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if _CUDART is None:
            raise RuntimeError("libcudart not found")
    return _CUDART
