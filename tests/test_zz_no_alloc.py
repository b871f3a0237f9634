"""afn_kernel_matvec_noalloc: the FP64 kernel matvec for callers that cannot
allocate device memory (for example a service whose device memory is planned
up front and handed out by its own pool, or a plug-in that must not grow its
host process's device footprint).  Its scratch is a
fixed array inside the library, so the test checks that two calls in a row --
which share and reuse that array -- each give the same result as the
allocating entry point afn_kernel_matvec, within the FP64 matvec tolerance
used by the parity tests, and that a size the array cannot hold is refused.

This file is named so that pytest collects it last."""
import ctypes as C

import numpy as np
import pytest

from paper_2304_05460_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_05460_gb300 import afn
    return torch, afn


def _call(afn, torch, Xd, kernel, l, mu, Pt, Qt):
    """Call the C entry point directly; Pt/Qt hold n x nrhs column-major."""
    n, d = Xd.shape
    nrhs = Pt.shape[0]
    f = afn.lib().afn_kernel_matvec_noalloc
    return f(C.c_void_p(Xd.data_ptr()), n, d, kernel, float(l), float(mu),
             C.c_void_p(Pt.data_ptr()), nrhs, C.c_void_p(Qt.data_ptr()), None)


def _bound(X, kernel, l, mu, P):
    import oracle
    K = oracle.kernel_matrix(X, X, kernel, l)
    A = np.abs(P)
    return K @ A + mu * A


@pytest.mark.parametrize("n,d,kernel,nrhs", [(3001, 8, 0, 11), (1777, 3, 1, 3)])
def test_noalloc_matches_allocating_entry_twice(env, n, d, kernel, nrhs):
    torch, afn = env
    X = inputs.normal_points(n, d, 10 + n)
    l, mu = 0.8 * np.sqrt(d), 1e-2
    Xd = torch.tensor(X, device="cuda")
    for call in range(2):
        P = inputs.rhs(n, nrhs, 20 + n + call)
        ref = afn.afn_kernel_matvec(X, kernel, l, mu, P, precision=afn.PREC_FP64)
        Pt = torch.tensor(np.ascontiguousarray(P.T), device="cuda")
        Qt = torch.full((nrhs, n), float("nan"), dtype=torch.float64, device="cuda")
        st = _call(afn, torch, Xd, kernel, l, mu, Pt, Qt)
        assert st == afn.AFN_OK, afn.last_error()
        q = Qt.cpu().numpy().T
        bound = _bound(X, kernel, l, mu, P)
        assert np.all(np.abs(q - ref) <= 1e-12 * bound + 1e-300)


def test_noalloc_rejects_oversized_problem(env):
    torch, afn = env
    n = 2_200_000
    Xd = torch.zeros((n, 1), dtype=torch.float64, device="cuda")
    Pt = torch.zeros((1, n), dtype=torch.float64, device="cuda")
    Qt = torch.zeros((1, n), dtype=torch.float64, device="cuda")
    st = _call(afn, torch, Xd, 0, 1.0, 1e-2, Pt, Qt)
    assert st == afn.AFN_ERR_ARG
    assert "scratch" in afn.last_error()


def test_noalloc_rejects_host_memory(env):
    torch, afn = env
    X = np.zeros((10, 2))
    P = np.zeros((1, 10))
    Q = np.zeros((1, 10))
    f = afn.lib().afn_kernel_matvec_noalloc
    st = f(X.ctypes.data_as(C.c_void_p), 10, 2, 0, 1.0, 1e-2, P.ctypes.data_as(C.c_void_p), 1,
           Q.ctypes.data_as(C.c_void_p), None)
    assert st == afn.AFN_ERR_ARG
