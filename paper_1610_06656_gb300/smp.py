"""ctypes binding of libsmp (include/smp.h): the same call names, argument marshalling only.

Device buffers are passed as torch CUDA tensors (or raw integer device pointers); streams as torch.cuda.Stream,
a raw cudaStream_t integer, or None for torch's current stream. Every compute step runs inside libsmp's kernels;
this module never computes on the host. Importing it does not need a GPU, but loading the library needs
libsmp.so to have been built (`__graft_entry__.build()`); a missing library raises instead of falling back.
"""
import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsmp.so")

SMP_OK, SMP_EINVAL, SMP_ENOMEM, SMP_ECUDA, SMP_ESTATE, SMP_ETIMEOUT, SMP_ENUMERIC, SMP_EUNSUPPORTED, SMP_EBUSY = range(9)
SMP_F32, SMP_BF16, SMP_F64 = 0, 1, 2
SMP_ENGINE_AUTO, SMP_ENGINE_SIMT, SMP_ENGINE_TC, SMP_ENGINE_TC_FP8, SMP_ENGINE_SRHT, SMP_ENGINE_TC_BF16 = 0, 1, 2, 3, 4, 5
SMP_SPLIT_OMEGA, SMP_NO_TRIM, SMP_INIT_GIVEN, SMP_FP64_ALS = 1, 2, 4, 8

_c = ctypes
_vp = _c.c_void_p
_i32, _i64, _u32, _u64, _f64 = _c.c_int32, _c.c_int64, _c.c_uint32, _c.c_uint64, _c.c_double


class smp_params(_c.Structure):
    _fields_ = [("n1", _i64), ("n2", _i64), ("k", _i32), ("dtype", _i32), ("seed", _u64), ("same_ab", _i32),
                ("engine", _i32), ("max_rows", _i64)]


class smp_server_params(_c.Structure):
    _fields_ = [("hbm_budget_bytes", _i64), ("solve_workers", _i32)]


class smp_job_params(_c.Structure):
    _fields_ = [("sketch", smp_params), ("r", _i32), ("T", _i32), ("flags", _u32), ("m", _f64),
                ("sample_seed", _u64), ("walt_seed", _u64)]


# name -> (restype, argtypes), mirroring include/smp.h
SIGNATURES = {
    "smp_sketch_coverage": (_i32, [_vp, _c.POINTER(_i64), _c.POINTER(_i64), _c.POINTER(_i64)]),
    "smp_norms_accumulate": (_i32, [_vp, _vp, _i64, _vp, _i64, _i64, _i64]),
    "smp_exact_accumulate": (_i32, [_vp, _vp, _i64, _vp, _i64, _i64, _i64]),
    "smp_exact_values": (_i32, [_vp, _vp]),
    "smp_exact_coverage": (_i32, [_vp, _c.POINTER(_i64), _c.POINTER(_i64), _c.POINTER(_i64)]),
    "smp_debug_fail_allocs": (None, [_i32]),
    "smp_debug_tc_wait": (None, [_i64, _i32]),
    "smp_serve_job_bytes": (_i32, [_c.POINTER(smp_job_params), _c.POINTER(_i64)]),
    "smp_serve_create": (_i32, [_c.POINTER(smp_server_params), _c.POINTER(_vp)]),
    "smp_serve_admit": (_i32, [_vp, _c.POINTER(smp_job_params), _c.POINTER(_i64)]),
    "smp_serve_block": (_i32, [_vp, _i64, _vp, _i64, _vp, _i64, _i64, _i64]),
    "smp_serve_close": (_i32, [_vp, _i64]),
    "smp_serve_poll": (_i32, [_vp, _i64, _c.POINTER(_i32)]),
    "smp_serve_collect": (_i32, [_vp, _i64, _f64, _vp, _vp, _vp, _c.POINTER(_i64), _c.POINTER(_f64)]),
    "smp_serve_cancel": (_i32, [_vp, _i64]),
    "smp_serve_stats": (_i32, [_vp, _c.POINTER(_i64), _c.POINTER(_i32)]),
    "smp_serve_destroy": (_i32, [_vp]),
    "smp_sketch_begin": (_i32, [_c.POINTER(smp_params), _vp, _c.POINTER(_vp)]),
    "smp_sketch_accumulate": (_i32, [_vp, _vp, _i64, _vp, _i64, _i64, _i64]),
    "smp_sketch_accumulate_host": (_i32, [_vp, _vp, _i64, _vp, _i64, _i64, _i64]),
    "smp_sketch_accumulate_pi": (_i32, [_vp, _vp, _i64, _vp, _i64, _vp, _i64, _i64, _i64]),
    "smp_sketch_reset": (_i32, [_vp]),
    "smp_sketch_finalize": (_i32, [_vp]),
    "smp_sketch_view": (_i32, [_vp, _c.POINTER(_vp), _c.POINTER(_vp), _c.POINTER(_i64), _c.POINTER(_vp),
                               _c.POINTER(_vp), _c.POINTER(_f64)]),
    "smp_sketch_import": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "smp_sample": (_i32, [_vp, _f64, _u64, _c.POINTER(_i64)]),
    "smp_sample_multinomial": (_i32, [_vp, _f64, _u64, _c.POINTER(_i64)]),
    "smp_sample_from_norms": (_i32, [_vp, _vp, _vp, _f64, _u64, _c.POINTER(_i64)]),
    "smp_omega_view": (_i32, [_vp, _c.POINTER(_i64), _c.POINTER(_vp), _c.POINTER(_vp), _c.POINTER(_vp),
                              _c.POINTER(_vp), _c.POINTER(_vp), _c.POINTER(_vp)]),
    "smp_estimate": (_i32, [_vp, _vp]),
    "smp_waltmin": (_i32, [_vp, _vp, _i32, _i32, _u32, _u64, _vp, _vp, _vp, _vp]),
    "smp_sketch_svd": (_i32, [_vp, _i32, _u64, _vp, _vp, _vp]),
    "smp_sync": (_i32, [_vp]),
    "smp_destroy": (_i32, [_vp]),
    "smp_last_error": (_c.c_char_p, [_vp]),
    "smp_status_string": (_c.c_char_p, [_i32]),
    "smp_version": (_i32, []),
    "smp_launch_count": (_i64, []),
    "smp_sketch_noalloc": (_i32, [_vp, _i64, _vp, _i64, _i64, _i64, _i32, _i32, _u64, _i64, _i64, _vp, _vp, _vp,
                                  _vp, _vp]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libsmp.so (once) and declare every exported call's signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libsmp.so is not built (%s); run __graft_entry__.build() first" % path)
    lib = _c.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SmpError(RuntimeError):
    def __init__(self, status, call, msg):
        self.status = status
        super().__init__("%s -> %s: %s" % (call, status_string(status), msg))


def status_string(s):
    return load().smp_status_string(int(s)).decode()


def _ptr(x):
    """Device pointer of a torch tensor, an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status, call, ctx=None):
    if status != SMP_OK:
        msg = load().smp_last_error(ctx).decode(errors="replace")
        raise SmpError(status, call, msg)


# ---- the C calls, one wrapper each ------------------------------------------------------------------------------
def smp_sketch_begin(n1, n2, k, seed, dtype=SMP_F32, same_ab=False, engine=SMP_ENGINE_AUTO, max_rows=0,
                     stream=None):
    p = smp_params(n1=n1, n2=n2, k=k, dtype=dtype, seed=seed & 0xFFFFFFFFFFFFFFFF, same_ab=int(bool(same_ab)),
                   engine=engine, max_rows=max_rows)
    out = _vp()
    _check(load().smp_sketch_begin(_c.byref(p), _stream(stream), _c.byref(out)), "smp_sketch_begin")
    return out.value


def smp_sketch_accumulate(ctx, A_blk, lda, B_blk, ldb, row0, nrows):
    _check(load().smp_sketch_accumulate(ctx, _ptr(A_blk), lda, _ptr(B_blk), ldb, row0, nrows),
           "smp_sketch_accumulate", ctx)


def smp_sketch_accumulate_host(ctx, A_blk, lda, B_blk, ldb, row0, nrows):
    """A_blk / B_blk: host buffers (CPU torch tensors, pinned for overlap, or raw host addresses)."""
    _check(load().smp_sketch_accumulate_host(ctx, _ptr(A_blk), lda, _ptr(B_blk), ldb, row0, nrows),
           "smp_sketch_accumulate_host", ctx)


def smp_sketch_accumulate_pi(ctx, Pi_blk, ldp, A_blk, lda, B_blk, ldb, row0, nrows):
    _check(load().smp_sketch_accumulate_pi(ctx, _ptr(Pi_blk), ldp, _ptr(A_blk), lda, _ptr(B_blk), ldb, row0,
                                           nrows), "smp_sketch_accumulate_pi", ctx)


def smp_sketch_reset(ctx):
    _check(load().smp_sketch_reset(ctx), "smp_sketch_reset", ctx)


def smp_sketch_finalize(ctx):
    _check(load().smp_sketch_finalize(ctx), "smp_sketch_finalize", ctx)


def smp_sketch_view(ctx):
    """Returns (At_ptr, Bt_ptr, ldk, sA_ptr, sB_ptr, (FA, FB))."""
    At, Bt, sA, sB = _vp(), _vp(), _vp(), _vp()
    ldk = _i64()
    F = (_f64 * 2)()
    _check(load().smp_sketch_view(ctx, _c.byref(At), _c.byref(Bt), _c.byref(ldk), _c.byref(sA), _c.byref(sB), F),
           "smp_sketch_view", ctx)
    return At.value, Bt.value, ldk.value, sA.value, sB.value, (F[0], F[1])


def smp_sketch_import(ctx, At, Bt, sA, sB):
    _check(load().smp_sketch_import(ctx, _ptr(At), _ptr(Bt), _ptr(sA), _ptr(sB)), "smp_sketch_import", ctx)


def smp_sample(ctx, m, seed):
    nnz = _i64()
    _check(load().smp_sample(ctx, float(m), seed & 0xFFFFFFFFFFFFFFFF, _c.byref(nnz)), "smp_sample", ctx)
    return nnz.value


def smp_sample_multinomial(ctx, m, seed):
    nnz = _i64()
    _check(load().smp_sample_multinomial(ctx, float(m), seed & 0xFFFFFFFFFFFFFFFF, _c.byref(nnz)),
           "smp_sample_multinomial", ctx)
    return nnz.value


def smp_sample_from_norms(ctx, sA, sB, m, seed):
    nnz = _i64()
    _check(load().smp_sample_from_norms(ctx, _ptr(sA), _ptr(sB), float(m), seed & 0xFFFFFFFFFFFFFFFF,
                                        _c.byref(nnz)), "smp_sample_from_norms", ctx)
    return nnz.value


def smp_omega_view(ctx):
    """Returns dict(nnz, row_ptr, col, qhat, col_ptr, csc_row, csc_pos) of device pointers."""
    nnz = _i64()
    ptrs = [_vp() for _ in range(6)]
    _check(load().smp_omega_view(ctx, _c.byref(nnz), *[_c.byref(p) for p in ptrs]), "smp_omega_view", ctx)
    names = ["row_ptr", "col", "qhat", "col_ptr", "csc_row", "csc_pos"]
    d = {n: p.value for n, p in zip(names, ptrs)}
    d["nnz"] = nnz.value
    return d


def smp_estimate(ctx, vals):
    _check(load().smp_estimate(ctx, _ptr(vals)), "smp_estimate", ctx)


def smp_sketch_svd(ctx, r, seed, U, S, V):
    _check(load().smp_sketch_svd(ctx, r, seed & 0xFFFFFFFFFFFFFFFF, _ptr(U), _ptr(S), _ptr(V)), "smp_sketch_svd",
           ctx)


def smp_waltmin(ctx, vals, r, T, flags, seed, U_init, U, S, V):
    _check(load().smp_waltmin(ctx, _ptr(vals), r, T, flags, seed & 0xFFFFFFFFFFFFFFFF, _ptr(U_init), _ptr(U),
                              _ptr(S), _ptr(V)), "smp_waltmin", ctx)


def smp_sync(ctx):
    _check(load().smp_sync(ctx), "smp_sync", ctx)


def smp_destroy(ctx):
    load().smp_destroy(ctx)


def smp_last_error(ctx=None):
    return load().smp_last_error(ctx).decode(errors="replace")


def smp_version():
    return load().smp_version()


def smp_sketch_noalloc(A, lda, B, ldb, n1, n2, k, dtype, seed, row0, nrows, At, Bt, sA, sB, stream=None):
    """Allocation-free sketch of one row range into caller buffers (see include/smp.h)."""
    _check(load().smp_sketch_noalloc(_ptr(A), lda, _ptr(B), ldb, n1, n2, k, dtype, seed & 0xFFFFFFFFFFFFFFFF, row0,
                                     nrows, _ptr(At), _ptr(Bt), _ptr(sA), _ptr(sB), _stream(stream)),
           "smp_sketch_noalloc")


def smp_launch_count():
    return load().smp_launch_count()


# ------------------------------------------------------------------------------------------------ serving form
def job_params(n1, n2, k, r, T, m, seed, sample_seed, walt_seed, dtype=SMP_F32, same_ab=False,
               engine=SMP_ENGINE_AUTO, max_rows=0, flags=0):
    sk = smp_params(n1=n1, n2=n2, k=k, dtype=dtype, seed=seed & 0xFFFFFFFFFFFFFFFF, same_ab=int(bool(same_ab)),
                    engine=engine, max_rows=max_rows)
    return smp_job_params(sketch=sk, r=r, T=T, flags=flags, m=float(m), sample_seed=sample_seed & 0xFFFFFFFFFFFFFFFF,
                          walt_seed=walt_seed & 0xFFFFFFFFFFFFFFFF)


def smp_serve_job_bytes(jp):
    b = _i64()
    _check(load().smp_serve_job_bytes(_c.byref(jp), _c.byref(b)), "smp_serve_job_bytes")
    return b.value


def smp_serve_create(hbm_budget_bytes, solve_workers=4):
    p = smp_server_params(hbm_budget_bytes=int(hbm_budget_bytes), solve_workers=solve_workers)
    out = _vp()
    _check(load().smp_serve_create(_c.byref(p), _c.byref(out)), "smp_serve_create")
    return out.value


def smp_serve_admit(server, jp):
    """Job id, or None when the budget is full (SMP_EBUSY)."""
    jid = _i64()
    st = load().smp_serve_admit(server, _c.byref(jp), _c.byref(jid))
    if st == SMP_EBUSY:
        return None
    _check(st, "smp_serve_admit")
    return jid.value


def smp_serve_block(server, job, A_blk, lda, B_blk, ldb, row0, nrows):
    _check(load().smp_serve_block(server, job, _ptr(A_blk), lda, _ptr(B_blk), ldb, row0, nrows), "smp_serve_block")


def smp_serve_close(server, job):
    _check(load().smp_serve_close(server, job), "smp_serve_close")


def smp_serve_poll(server, job):
    d = _i32()
    _check(load().smp_serve_poll(server, job, _c.byref(d)), "smp_serve_poll")
    return bool(d.value)


def smp_serve_collect(server, job, U=None, S=None, V=None, timeout_s=-1.0):
    """(nnz, latency_ms) after copying the factors into U, S, V (device tensors or None)."""
    nnz, lat = _i64(), _f64()
    _check(load().smp_serve_collect(server, job, float(timeout_s), _ptr(U), _ptr(S), _ptr(V), _c.byref(nnz),
                                    _c.byref(lat)), "smp_serve_collect")
    return nnz.value, lat.value


def smp_serve_cancel(server, job):
    _check(load().smp_serve_cancel(server, job), "smp_serve_cancel")


def smp_serve_stats(server):
    used, live = _i64(), _i32()
    _check(load().smp_serve_stats(server, _c.byref(used), _c.byref(live)), "smp_serve_stats")
    return used.value, live.value


def smp_serve_destroy(server):
    _check(load().smp_serve_destroy(server), "smp_serve_destroy")


def smp_sketch_coverage(ctx):
    """(rows accumulated, first row missing from the run that starts at 0, number of disjoint ranges)."""
    rows, first, ranges = _i64(), _i64(), _i64()
    _check(load().smp_sketch_coverage(ctx, _c.byref(rows), _c.byref(first), _c.byref(ranges)), "smp_sketch_coverage",
           ctx)
    return rows.value, first.value, ranges.value


def smp_norms_accumulate(ctx, A_blk, lda, B_blk, ldb, row0, nrows):
    _check(load().smp_norms_accumulate(ctx, _ptr(A_blk), lda, _ptr(B_blk), ldb, row0, nrows),
           "smp_norms_accumulate", ctx)


def smp_exact_accumulate(ctx, A_blk, lda, B_blk, ldb, row0, nrows):
    _check(load().smp_exact_accumulate(ctx, _ptr(A_blk), lda, _ptr(B_blk), ldb, row0, nrows),
           "smp_exact_accumulate", ctx)


def smp_exact_values(ctx, vals):
    _check(load().smp_exact_values(ctx, _ptr(vals)), "smp_exact_values", ctx)


def smp_exact_coverage(ctx):
    """(rows of the exact pass, first row missing from the run that starts at 0, number of disjoint ranges)."""
    rows, first, ranges = _i64(), _i64(), _i64()
    _check(load().smp_exact_coverage(ctx, _c.byref(rows), _c.byref(first), _c.byref(ranges)), "smp_exact_coverage",
           ctx)
    return rows.value, first.value, ranges.value


def smp_debug_fail_allocs(n):
    load().smp_debug_fail_allocs(int(n))


def smp_debug_tc_wait(wait_ns=0, skip_stage=-1):
    load().smp_debug_tc_wait(int(wait_ns), int(skip_stage))
