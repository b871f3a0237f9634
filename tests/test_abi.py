"""The C-ABI library loads and exports every symbol include/afn.h declares
(no compute: this runs without a GPU), and the binding refuses bad input
before any device work."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def _declared():
    names = set()
    for f in os.listdir(HEADER_DIR):
        if f.endswith(".h"):
            txt = open(os.path.join(HEADER_DIR, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(afn_[A-Za-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2304_05460_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("afn_build", "afn_solve", "afn_free", "afn_last_error", "afn_kernel_matvec",
                 "afn_fps", "afn_knn_pattern", "afn_rank_estimate", "afn_apply_precond"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_exports_are_c_symbols():
    from paper_2304_05460_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.build()], capture_output=True,
                         text=True).stdout
    syms = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for n in _declared():
        assert n in syms, n          # unmangled extern "C"


def test_argument_checks_without_gpu():
    from paper_2304_05460_gb300 import afn
    X = np.zeros((4, 3))
    with pytest.raises(afn.AfnError) as e:
        afn.afn_build(X, afn.GAUSSIAN, -1.0, 1e-3, 2, 2)        # l <= 0
    assert e.value.status == afn.AFN_ERR_ARG
    with pytest.raises(afn.AfnError) as e:
        afn.afn_build(X, afn.GAUSSIAN, 1.0, 0.0, 2, 2)         # mu <= 0
    assert e.value.status == afn.AFN_ERR_ARG
    with pytest.raises(afn.AfnError) as e:
        afn.afn_build(np.zeros((4, 17)), afn.GAUSSIAN, 1.0, 1e-3, 2, 2)   # d > 16
    assert e.value.status == afn.AFN_ERR_ARG
    with pytest.raises(afn.AfnError) as e:
        afn.afn_build(X, 5, 1.0, 1e-3, 2, 2)                  # unknown kernel
    assert e.value.status == afn.AFN_ERR_ARG
    for w in (0, 129):                                       # FSAI width outside 1..128
        with pytest.raises(afn.AfnError) as e:
            afn.afn_build(X, afn.GAUSSIAN, 1.0, 1e-3, 2, w)
        assert e.value.status == afn.AFN_ERR_ARG


def test_default_options():
    from paper_2304_05460_gb300 import afn
    o = afn.options()
    assert (o.precision, o.landmarks, o.rank_mode, o.max_iter, o.max_outer) == (0, 0, 0, 500, 10)
    assert o.inner_tol == 0.01 and o.fps_start == 0
    # Alg. 5 fields sit after the stream pointer; AFN is the default preconditioner
    assert (o.precond, o.precond_threshold) == (afn.PRECOND_AFN, 0)
    assert (o.factors, o.apply_tc, o.flexible, o.schur_order) == (afn.FACTORS_FP32, 2, 0, 0)
    assert (o.krylov, o.auto_rho) == (afn.KRYLOV_FP32, 0.0)
    assert ctypes.sizeof(afn.afn_options) == 104
    assert ctypes.sizeof(afn.afn_build_info) == 96


def test_bad_matvec_precision_rejected_without_gpu():
    from paper_2304_05460_gb300 import afn
    X = np.zeros((4, 3))
    p = np.ones(4)
    for prec in (3, 6, -1):
        with pytest.raises(afn.AfnError) as e:
            afn.afn_kernel_matvec(X, afn.GAUSSIAN, 1.0, 1e-3, p, precision=prec)
        assert e.value.status == afn.AFN_ERR_ARG


def test_bad_krylov_and_auto_rho_rejected_without_gpu():
    from paper_2304_05460_gb300 import afn
    X = np.zeros((4, 3))
    for kw in (dict(krylov=4), dict(krylov=-1), dict(auto_rho=-0.5), dict(auto_rho=float("nan"))):
        with pytest.raises(afn.AfnError) as e:
            afn.afn_build(X, afn.GAUSSIAN, 1.0, 1e-3, 2, 2, **kw)
        assert e.value.status == afn.AFN_ERR_ARG


def test_bad_precond_rejected_without_gpu():
    from paper_2304_05460_gb300 import afn
    X = np.zeros((4, 3))
    for kw in (dict(precond=3), dict(precond=-1), dict(precond=afn.PRECOND_AUTO, precond_threshold=-5)):
        with pytest.raises(afn.AfnError) as e:
            afn.afn_build(X, afn.GAUSSIAN, 1.0, 1e-3, 2, 2, **kw)
        assert e.value.status == afn.AFN_ERR_ARG


def test_bad_factor_and_apply_options_rejected_without_gpu():
    from paper_2304_05460_gb300 import afn
    X = np.zeros((4, 3))
    for kw in (dict(factors=2), dict(factors=-1), dict(apply_tc=3), dict(apply_tc=-1),
               dict(flexible=3), dict(schur_order=2)):
        with pytest.raises(afn.AfnError) as e:
            afn.afn_build(X, afn.GAUSSIAN, 1.0, 1e-3, 2, 2, **kw)
        assert e.value.status == afn.AFN_ERR_ARG


def test_noalloc_binding_refuses_bad_tensors_before_any_launch():
    # the binding checks type, dtype, contiguity, shape and device before it calls the
    # library, so a mis-shaped (n, nrhs) block never reaches the kernels
    torch = pytest.importorskip("torch")
    from paper_2304_05460_gb300 import afn
    n, d = 10, 3
    X = torch.zeros((n, d), dtype=torch.float64)
    good = torch.zeros((2, n), dtype=torch.float64)
    cases = [
        (np.zeros((n, d)), good, good, "torch tensor"),
        (X.float(), good, good, "float64"),
        (X, torch.zeros((n, 2), dtype=torch.float64), torch.zeros((n, 2), dtype=torch.float64),
         "shape (nrhs, n)"),
        (X, good, torch.zeros((3, n), dtype=torch.float64), "one shape"),
        (X, torch.zeros((4, n), dtype=torch.float64)[:, ::2].t(), good, "contiguous"),
        (X[:, :2], good, good, None),
        (X, good, good, "CUDA memory"),
    ]
    for pts, p, q, msg in cases:
        with pytest.raises(ValueError) as e:
            afn.afn_kernel_matvec_noalloc(pts, afn.GAUSSIAN, 1.0, 1e-2, p, q)
        if msg:
            assert msg in str(e.value), (msg, str(e.value))


def test_binding_refuses_blocks_of_the_wrong_size_before_any_launch():
    # the library reads n x nrhs values from a right-hand-side block and cannot see the
    # buffer's size, so the binding refuses a block whose rows differ from n (and
    # points or blocks that are not 2-D / 1-D) before calling it
    from paper_2304_05460_gb300 import afn
    X = np.zeros((10, 3))
    for p in (np.zeros(9), np.zeros((11, 2)), np.zeros((10, 2, 2))):
        with pytest.raises(ValueError):
            afn.afn_kernel_matvec(X, afn.GAUSSIAN, 1.0, 1e-2, p)
    with pytest.raises(ValueError):
        afn.afn_kernel_matvec(np.zeros(10), afn.GAUSSIAN, 1.0, 1e-2, np.zeros(10))
    with pytest.raises(ValueError):
        afn.afn_build(np.zeros((2, 5, 3)), afn.GAUSSIAN, 1.0, 1e-2, 2, 2)

    class FakeHandle:
        ptr, n = None, 10
    for r in (np.zeros(9), np.zeros((12, 1))):
        with pytest.raises(ValueError):
            afn.afn_solve(FakeHandle(), r, 1e-6)
        with pytest.raises(ValueError):
            afn.afn_apply_precond(FakeHandle(), r)

    class FakeBatch:
        ptr, nsys, n = None, 2, [10, 20]
    with pytest.raises(ValueError):
        afn.afn_solve_batched(FakeBatch(), [np.zeros(10), np.zeros(19)], 1e-6)


def test_header_is_c99_and_the_library_links_from_c(tmp_path):
    # a C caller: the header compiles as strict C99, the program links against the
    # library by name, and an argument error comes back as a status (no GPU work)
    import shutil
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2304_05460_gb300 import build
    libdir = os.path.dirname(build.build())
    src = tmp_path / "caller.c"
    src.write_text(
        '#include <stdio.h>\n#include "afn.h"\n'
        "int main(void) {\n"
        "    afn_options o;\n"
        "    afn_handle *h = 0;\n"
        "    double pts[6] = {0};\n"
        "    afn_status st;\n"
        "    afn_default_options(&o);\n"
        "    st = afn_build(pts, 2, 3, AFN_GAUSSIAN, -1.0, 1e-2, 1, 1, &o, &h);\n"
        '    printf("%d %d %s\\n", (int)st, (int)o.max_iter, afn_last_error());\n'
        "    return (st == AFN_ERR_ARG && h == 0) ? 0 : 1;\n"
        "}\n")
    exe = tmp_path / "caller"
    cc = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                         "-I", HEADER_DIR, str(src), "-L", libdir, "-lafn",
                         "-Wl,-rpath," + libdir, "-o", str(exe)], capture_output=True, text=True)
    assert cc.returncode == 0, cc.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, (run.stdout, run.stderr)
    assert run.stdout.startswith("1 500 ") and "invalid argument" in run.stdout


def test_null_handles_are_refused_or_ignored_without_gpu():
    # the frees are NULL-safe; every other entry point returns AFN_ERR_ARG for a NULL
    # handle or output before it touches the device
    from paper_2304_05460_gb300 import afn
    lib = afn.lib()
    lib.afn_free(None)
    lib.afn_batch_free(None)
    lib.afn_server_destroy(None)
    assert lib.afn_batch_build_ms(None) == 0.0
    bi = afn.afn_build_info()
    si = afn.afn_solve_info()
    buf = (ctypes.c_double * 4)()
    cnt = ctypes.c_int32(0)
    checks = [
        lambda: lib.afn_get_build_info(None, ctypes.byref(bi)),
        lambda: lib.afn_get_perm(None, buf),
        lambda: lib.afn_get_L(None, buf),
        lambda: lib.afn_get_W(None, buf),
        lambda: lib.afn_solve(None, buf, 1, 1e-6, buf, ctypes.byref(si)),
        lambda: lib.afn_apply_precond(None, buf, 1, buf),
        lambda: lib.afn_reset_kernel_stats(None),
        lambda: lib.afn_batch_build_info(None, 0, ctypes.byref(bi)),
        lambda: lib.afn_solve_batched(None, buf, None, 1e-6, buf, None, None, None),
        lambda: lib.afn_server_poll(None, None, 0, ctypes.byref(cnt), 0),
        lambda: lib.afn_server_result(None, 0, buf, None, None, None),
        lambda: lib.afn_server_get_stats(None, None),
    ]
    for i, f in enumerate(checks):
        assert f() == afn.AFN_ERR_ARG, i
        assert afn.last_error(), i


def test_server_config_checked_without_gpu():
    from paper_2304_05460_gb300 import afn
    for kw in (dict(precision=9), dict(precond=afn.PRECOND_NYSTROM), dict(memory_budget=-1),
               dict(max_active=-2), dict(build_threads=-1)):
        with pytest.raises(afn.AfnError) as e:
            afn.Server(**kw)
        assert e.value.status == afn.AFN_ERR_ARG, kw
    cfg = afn.afn_server_config()
    afn.lib().afn_server_default_config(ctypes.byref(cfg))
    assert cfg.opt.precision == afn.PREC_AUTO and cfg.build_threads == 8
    assert cfg.memory_budget == 0 and cfg.max_active == 0
