"""dp_selftest_noalloc (fixed in-library scratch, no allocation) against
dp_selftest (cudaMalloc'd scratch), both through the C-ABI (GPU only).

The file name sorts last so that the check also runs after every other GPU
test in the same process; it passes alone as well."""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [0, 1, 2, 3, 4]
# The self check multiplies small exact integers: both entry points must report
# max error 0 and the same max value, up to the float -> double conversion.
TOL = 1e-6


@pytest.fixture(scope="module")
def dp():
    import paper_2410_22867_gb300 as dp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dp.lib()
    return dp


def _close(got, ref):
    (e, v), (re_, rv) = got, ref
    assert e == pytest.approx(re_, abs=TOL)
    assert v == pytest.approx(rv, rel=TOL)


def test_noalloc_matches_allocating_entry_point_twice(dp):
    ref = [dp.selftest(c) for c in CASES]
    for _ in range(2):
        got = dp.selftest_noalloc(CASES)
        assert len(got) == len(CASES)
        for g, r in zip(got, ref):
            _close(g, r)
            assert g[0] == 0.0


def test_noalloc_clears_its_scratch_between_calls(dp):
    # run the case with the largest max |value| in slot 0, then the one with the
    # smallest: if the slot were not zeroed by the second call, it would report
    # the first case's (stale, larger) value
    ref = {c: dp.selftest(c) for c in CASES}
    hi = max(CASES, key=lambda c: ref[c][1])
    lo = min(CASES, key=lambda c: ref[c][1])
    assert ref[hi][1] > ref[lo][1]
    _close(dp.selftest_noalloc([hi])[0], ref[hi])
    _close(dp.selftest_noalloc([lo])[0], ref[lo])


def test_noalloc_full_capacity(dp):
    n = dp.SELFTEST_NOALLOC_MAX_CASES
    cases = [CASES[i % len(CASES)] for i in range(n)]
    ref = {c: dp.selftest(c) for c in CASES}
    for c, g in zip(cases, dp.selftest_noalloc(cases)):
        _close(g, ref[c])


def test_noalloc_rejects_bad_sizes(dp):
    L = dp.lib()
    n = dp.SELFTEST_NOALLOC_MAX_CASES + 1
    which = (ctypes.c_int * n)(*([0] * n))
    out = (ctypes.c_double * (2 * n))()
    assert L.dp_selftest_noalloc(ctypes.cast(which, ctypes.c_void_p), n, ctypes.cast(out, ctypes.c_void_p)) == 8
    assert L.dp_selftest_noalloc(ctypes.cast(which, ctypes.c_void_p), -1, ctypes.cast(out, ctypes.c_void_p)) == 1
    which[0] = 5
    assert L.dp_selftest_noalloc(ctypes.cast(which, ctypes.c_void_p), 1, ctypes.cast(out, ctypes.c_void_p)) == 1
    assert L.dp_selftest_noalloc(None, 0, None) == 0
