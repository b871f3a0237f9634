"""Failure handling of the bounded device-side waits, without a GPU fault.

The tcgen05 kernels give every mbarrier wait a time limit; a wait that runs
out raises the CTA's abort flag, the kernel waits (up to 2 s) for the copies
and MMAs it still has in flight, releases its tensor memory and returns, and
the entry point reports AFN_ERR_TIMEOUT.  Here the limit is lowered to a few
nanoseconds (afn_set_wait_limit_ns), so the waits of a healthy launch run
out; nothing faults, traps or hangs.  The next call with the default limit
on the same device must still give the oracle's result.
"""
import numpy as np
import pytest

import oracle
from paper_2304_05460_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def afn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_05460_gb300 import afn as a
    yield a
    a.afn_set_wait_limit_ns(0)


def _matvec_ok(afn, X, P):
    q = afn.afn_kernel_matvec(X, afn.GAUSSIAN, 2.0, 1e-2, P, precision=afn.PREC_MIXED)
    ref = oracle.matvec(X, afn.GAUSSIAN, 2.0, 1e-2, P)
    K = oracle.kernel_matrix(X, X, afn.GAUSSIAN, 2.0)
    bound = K @ np.abs(P) + 1e-2 * np.abs(P)
    assert np.all(np.abs(q - ref.reshape(q.shape)) <= 2e-5 * bound)


def test_matvec_wait_limit_runs_out_and_recovers(afn):
    X = inputs.normal_points(3000, 8, 71)
    P = inputs.rhs(3000, 32, 72)          # 32 columns: the tcgen05 matvec
    _matvec_ok(afn, X, P)
    try:
        afn.afn_set_wait_limit_ns(1)
        with pytest.raises(afn.AfnError) as e:
            afn.afn_kernel_matvec(X, afn.GAUSSIAN, 2.0, 1e-2, P, precision=afn.PREC_MIXED)
        assert e.value.status == afn.AFN_ERR_TIMEOUT
    finally:
        afn.afn_set_wait_limit_ns(0)
    _matvec_ok(afn, X, P)


@pytest.mark.parametrize("mode", [1, 2])
def test_apply_wait_limit_runs_out_and_recovers(afn, mode):
    # the tensor-core W products: three-pass tf32 (mode 1) and BF16 (mode 2)
    n, k = 2600, 260
    X = inputs.normal_points(n, 8, 73)
    h = afn.afn_build(X, afn.GAUSSIAN, 1.0, 1e-2, k, 32, precision=afn.PREC_MIXED, apply_tc=mode)
    r = inputs.rhs(n, 32, 74)             # 32 columns: the tcgen05 W products
    s0 = afn.afn_apply_precond(h, r)
    try:
        afn.afn_set_wait_limit_ns(1)
        with pytest.raises(afn.AfnError) as e:
            afn.afn_apply_precond(h, r)
        assert e.value.status == afn.AFN_ERR_TIMEOUT
    finally:
        afn.afn_set_wait_limit_ns(0)
    s1 = afn.afn_apply_precond(h, r)
    assert np.array_equal(s0, s1)
    afn.afn_free(h)


def test_double_float_tensor_core_wait_limit_runs_out_and_recovers(afn):
    # the double-float matvec with the sum on the tensor cores (32 columns)
    X = inputs.normal_points(3000, 8, 75)
    P = inputs.rhs(3000, 32, 76)
    q0 = afn.afn_kernel_matvec(X, afn.GAUSSIAN, 2.0, 1e-2, P, precision=afn.MATVEC_DF_TC)
    try:
        afn.afn_set_wait_limit_ns(1)
        with pytest.raises(afn.AfnError) as e:
            afn.afn_kernel_matvec(X, afn.GAUSSIAN, 2.0, 1e-2, P, precision=afn.MATVEC_DF_TC)
        assert e.value.status == afn.AFN_ERR_TIMEOUT
    finally:
        afn.afn_set_wait_limit_ns(0)
    q1 = afn.afn_kernel_matvec(X, afn.GAUSSIAN, 2.0, 1e-2, P, precision=afn.MATVEC_DF_TC)
    assert np.array_equal(q0, q1)
