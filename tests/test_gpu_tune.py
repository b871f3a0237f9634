"""The autotuner on the GPU: after its first few calls a shape has a recorded
choice under its key (the first call runs the default, the next ones each
candidate once, timed), and every candidate gives bit-identical results (row warps of
the tcgen05 matvec, threads per CTA of the FSAI build, CTAs per SM of the
grouped kernels), so what the tuner picks never changes a result."""
import numpy as np
import pytest

from paper_2304_05460_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def afn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_05460_gb300 import afn as a
    return a


def _keys(afn, prefix):
    return [k for k in afn.afn_tune_entries() if k.startswith(prefix)]


def test_matvec_row_warp_split_bit_identical(afn):
    X = inputs.normal_points(3000, 8, 91)
    P = inputs.rhs(3000, 32, 92)
    q0 = afn.afn_kernel_matvec(X, afn.GAUSSIAN, 2.0, 1e-2, P, precision=afn.PREC_MIXED)
    for _ in range(3):
        q = afn.afn_kernel_matvec(X, afn.GAUSSIAN, 2.0, 1e-2, P, precision=afn.PREC_MIXED)
        assert np.array_equal(q, q0)            # whichever candidate ran
    keys = _keys(afn, "mv32u/ds8/nb4/ker0/")
    assert keys, afn.afn_tune_entries()
    out = []
    for c in (0, 1):
        for k in keys:
            afn.afn_tune_put(k, c)
        out.append(afn.afn_kernel_matvec(X, afn.GAUSSIAN, 2.0, 1e-2, P, precision=afn.PREC_MIXED))
    assert np.array_equal(out[0], out[1])
    assert np.array_equal(out[0], q0)


def test_fsai_block_size_bit_identical(afn):
    X = inputs.uniform_points(2500, 3, 93)
    for _ in range(3):
        h = afn.afn_build(X, afn.GAUSSIAN, 0.1, 1e-3, 250, 32, precision=afn.PREC_MIXED)
        afn.afn_free(h)
    keys = _keys(afn, "fsai/wm32/f32/")
    assert keys
    gs = []
    for c in (0, 1):
        for k in keys:
            afn.afn_tune_put(k, c)
        h = afn.afn_build(X, afn.GAUSSIAN, 0.1, 1e-3, 250, 32, precision=afn.PREC_MIXED)
        gs.append(afn.afn_get_G(h)[1])
        afn.afn_free(h)
    assert np.array_equal(gs[0], gs[1])


def test_grouped_grid_sizes_bit_identical(afn):
    systems, rhs = [], []
    for i, (n, d) in enumerate([(900, 3), (1400, 5), (600, 8)]):
        X = inputs.normal_points(n, d, 95 + i)
        systems.append(dict(points=X, kernel=afn.GAUSSIAN, l=1.0 * np.sqrt(d), mu=1e-2,
                            k_max=n // 4, fsai_nnz=16))
        rhs.append(inputs.rhs(n, 8, 98 + i))
    b = afn.afn_build_batched(systems, precision=afn.PREC_MIXED)
    xs0, _ = afn.afn_solve_batched(b, rhs, 1e-6)
    afn.afn_batch_free(b)
    keys = _keys(afn, "gmv32/") + _keys(afn, "gapply/")
    assert keys
    for c in (0, 2):
        for k in keys:
            afn.afn_tune_put(k, c)
        b = afn.afn_build_batched(systems, precision=afn.PREC_MIXED)
        xs, _ = afn.afn_solve_batched(b, rhs, 1e-6)
        afn.afn_batch_free(b)
        for a, c_ in zip(xs0, xs):
            assert np.array_equal(a, c_)


def test_out_of_range_recorded_choice_is_ignored(afn):
    # a cache entry naming no candidate (a hand-edited file, say) is not used: the key is
    # tuned again, the entry replaced by a valid choice, and the results stay the same
    afn.afn_tune_clear()                        # only this test's keys from here on
    systems, rhs = [], []
    for i, (n, d) in enumerate([(800, 3), (1100, 6)]):
        X = inputs.normal_points(n, d, 111 + i)
        systems.append(dict(points=X, kernel=afn.GAUSSIAN, l=1.0 * np.sqrt(d), mu=1e-2,
                            k_max=n // 4, fsai_nnz=16))
        rhs.append(inputs.rhs(n, 8, 113 + i))
    b = afn.afn_build_batched(systems, precision=afn.PREC_MIXED)
    xs0, _ = afn.afn_solve_batched(b, rhs, 1e-6)
    afn.afn_batch_free(b)
    keys = _keys(afn, "gmv32/") + _keys(afn, "gapply/")
    assert keys
    for k in keys:
        afn.afn_tune_put(k, 7)                  # three candidates: 0, 1, 2
    b = afn.afn_build_batched(systems, precision=afn.PREC_MIXED)
    xs, _ = afn.afn_solve_batched(b, rhs, 1e-6)
    afn.afn_batch_free(b)
    for a, c in zip(xs0, xs):
        assert np.array_equal(a, c)
    for k in keys:
        assert 0 <= afn.afn_tune_get(k) < 3
    X = inputs.normal_points(3000, 8, 115)
    P = inputs.rhs(3000, 32, 116)
    q0 = afn.afn_kernel_matvec(X, afn.GAUSSIAN, 2.0, 1e-2, P, precision=afn.PREC_MIXED)
    for _ in range(3):                          # the key of this shape decided
        afn.afn_kernel_matvec(X, afn.GAUSSIAN, 2.0, 1e-2, P, precision=afn.PREC_MIXED)
    mk = _keys(afn, "mv32u/ds8/nb4/ker0/n2^11/")  # n = 3000
    assert mk, afn.afn_tune_entries()
    for k in mk:
        afn.afn_tune_put(k, 9)                  # two candidates: 0, 1
    for _ in range(4):
        q = afn.afn_kernel_matvec(X, afn.GAUSSIAN, 2.0, 1e-2, P, precision=afn.PREC_MIXED)
        assert np.array_equal(q, q0)
    for k in mk:
        assert 0 <= afn.afn_tune_get(k) < 2


def test_online_tuning_from_concurrent_threads(afn):
    # several host threads, each on its own stream, make the first calls of one
    # tuning key at the same time: one of them records the choice while the
    # others are still timing candidates; every result stays bit-identical
    import threading
    import torch
    afn.afn_tune_clear()
    X = inputs.normal_points(2000, 8, 103)
    P = inputs.rhs(2000, 32, 104)
    ref = afn.afn_kernel_matvec(X, afn.GAUSSIAN, 2.0, 1e-2, P, precision=afn.PREC_MIXED)
    afn.afn_tune_clear()
    out, errs = [], []

    def work():
        try:
            st = torch.cuda.Stream()
            for _ in range(5):
                out.append(afn.afn_kernel_matvec(X, afn.GAUSSIAN, 2.0, 1e-2, P,
                                                 precision=afn.PREC_MIXED, stream=st))
        except BaseException as e:      # reported below
            errs.append(e)
    ts = [threading.Thread(target=work) for _ in range(8)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errs, errs
    assert len(out) == 40
    for q in out:
        assert np.array_equal(q, ref)
    assert _keys(afn, "mv32u/ds8/nb4/ker0/")
