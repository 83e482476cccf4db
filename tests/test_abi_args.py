"""Host-side argument checks of the C ABI (no GPU): smp_sketch_begin validates its parameters before it touches
the device, and the calls that take a context reject a null one."""
import pytest

from paper_1610_06656_gb300 import build
from paper_1610_06656_gb300 import smp as S


@pytest.fixture(scope="module")
def lib():
    S.load(build.build())
    return S


@pytest.mark.parametrize("kw,status", [
    (dict(n1=0, n2=10, k=8), "SMP_EINVAL"),                                   # empty A
    (dict(n1=10, n2=10, k=0), "SMP_EINVAL"),                                  # k below 1
    (dict(n1=10, n2=10, k=4097), "SMP_EINVAL"),                               # k above 4,096
    (dict(n1=10, n2=12, k=8, same_ab=True), "SMP_EINVAL"),                    # A = B needs n1 == n2
    (dict(n1=10, n2=10, k=8, engine=6), "SMP_EINVAL"),                        # unknown engine
    (dict(n1=10, n2=10, k=8, dtype=7), "SMP_EINVAL"),                         # unknown dtype
    (dict(n1=10, n2=10, k=8, dtype=0, engine=3), "SMP_EUNSUPPORTED"),         # FP8 engine takes BF16 blocks
    (dict(n1=10, n2=10, k=8, dtype=1, engine=5), "SMP_EUNSUPPORTED"),         # BF16-operand engine takes FP32
    (dict(n1=10, n2=10, k=8, dtype=1, engine=4), "SMP_EUNSUPPORTED"),         # SRHT takes FP32 blocks
    (dict(n1=10, n2=10, k=8, engine=4, max_rows=1000), "SMP_EINVAL"),         # SRHT block not a power of two
    (dict(n1=10, n2=10, k=8, engine=4, max_rows=1 << 17), "SMP_EINVAL"),      # SRHT block above 2^16
    (dict(n1=10, n2=10, k=8, max_rows=-1), "SMP_EINVAL"),
])
def test_begin_rejects_bad_parameters(lib, kw, status):
    args = dict(seed=1, stream=0)   # stream 0: no torch CUDA call on a machine without a GPU
    args.update(kw)
    with pytest.raises(lib.SmpError) as e:
        lib.smp_sketch_begin(**args)
    assert lib.status_string(e.value.status) == status
    assert lib.load().smp_last_error(None)   # a one-line reason is left for the caller


@pytest.mark.parametrize("name,args", [
    ("smp_sketch_finalize", ()), ("smp_sketch_reset", ()), ("smp_estimate", (None,)),
    ("smp_exact_values", (None,)), ("smp_norms_accumulate", (None, 0, None, 0, 0, 0)),
    ("smp_exact_accumulate", (None, 0, None, 0, 0, 0)), ("smp_sync", ()),
])
def test_null_context_is_einval(lib, name, args):
    with pytest.raises(lib.SmpError) as e:
        getattr(lib, name)(None, *args)
    assert e.value.status == lib.SMP_EINVAL


def test_destroy_null_is_a_noop(lib):
    lib.smp_destroy(None)
