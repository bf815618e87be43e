"""The C ABI library loads without a GPU, exports every function that
include/*.h declares, and validates its arguments on the host."""
import ctypes
import glob
import math
import os
import re

import pytest

from paper_0809_3098_gb300 import lc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(lc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_0809_3098_gb300 import build

    build.build()
    return lc.lib()


def test_header_declares_the_abi():
    names = declared_functions()
    for required in ("lc_create", "lc_step", "lc_get_psi", "lc_get_omega", "lc_residual", "lc_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    raw = ctypes.CDLL(lc.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(raw, n)]
    assert not missing, missing


def test_create_validates_arguments(L):
    assert not L.lc_create(44, 100.0, 0.0, 1e-10)      # 44 = 4 * 11
    assert "N must be" in lc.last_error()
    assert not L.lc_create(16, -5.0, 0.0, 1e-10)
    assert not L.lc_create(16, 100.0, 0.0, 0.0)
    assert not L.lc_create(4, 100.0, 0.0, 1e-10)


def test_dt_rule_and_params(L):
    h = lc.lc_create(1024, 10000.0, 0.0, 1e-10)
    p = lc.lc_get_params(h)
    assert p[2] == 0.25 * min(1 / 1024, 10000.0 / 1024**2 / 4)
    assert p[5] == 7  # the V-cycle visits 1024 .. 16 (16 solved exactly)
    lc.lc_destroy(h)
    h = lc.lc_create(384, 1000.0, 1e-3, 1e-10)
    p = lc.lc_get_params(h)
    assert p[2] == 1e-3 and p[5] == 6  # 384 .. 12 (12 solved exactly)
    assert lc.lc_set_option(h, "coarse_direct", 0) == lc.LC_OK
    assert lc.lc_get_params(h)[5] == 8  # 384 .. 3, the coarsest grid smoothed
    assert lc.lc_set_option(h, "coarse_direct", 2) == lc.LC_ERR_ARG
    lc.lc_destroy(h)


def test_options_validate_without_gpu(L):
    h = lc.lc_create(64, 1000.0, 0.0, 1e-10)
    assert lc.lc_set_option(h, "nu1", 3) == lc.LC_OK
    assert lc.lc_set_option(h, "nu1", 0) == lc.LC_ERR_ARG
    assert lc.lc_set_option(h, "beta", 2.0) == lc.LC_ERR_ARG
    assert lc.lc_set_option(h, "op", 0) == lc.LC_OK
    assert lc.lc_set_option(h, "op", 2) == lc.LC_ERR_ARG
    assert lc.lc_set_option(h, "nonsense", 1) == lc.LC_ERR_ARG
    assert "unknown option" in lc.last_error()
    # execution options: ranges are checked before any device work
    for key, ok, bad in (("coarse_cluster", (-1, 0, 2, 16), (1, 17, 0.5)), ("cluster_max", (8, 128, 512), (7, 513)),
                         ("cluster_split", (4, 16, 256), (3, 257)), ("pdl", (0, 1), (2, -1)),
                         ("fused", (0, 1, 2, 3), (4, -1)), ("fine_phases", (0, 1, 16), (-1, 17))):
        for v in ok:
            assert lc.lc_set_option(h, key, v) == lc.LC_OK, (key, v)
        for v in bad:
            assert lc.lc_set_option(h, key, v) == lc.LC_ERR_ARG, (key, v)
    lc.lc_destroy(h)
    assert lc.lc_set_option(h, "nu1", 2) == lc.LC_ERR_ARG  # destroyed
    assert lc.lc_step(0, 1) == lc.LC_ERR_ARG
    assert math.isnan(lc.lc_residual(0))


def test_workspace_bytes(L):
    assert lc.lc_workspace_bytes(44, 0) == 0          # 44 = 4 * 11 is not a valid size
    assert lc.lc_workspace_bytes(20, 0) > 0           # 20 = 4 * 5 is
    a, b = lc.lc_workspace_bytes(512, 0), lc.lc_workspace_bytes(1024, 0)
    assert 3.5 < b / a < 4.5
    assert b % 256 == 0


def test_batch_options_validate_without_gpu(L):
    """Batch creation and option checks are host-side: no device is touched."""
    import ctypes

    N = (ctypes.c_int * 2)(128, 256)
    Re = (ctypes.c_double * 2)(1000.0, 5000.0)
    b = L.lc_batch_create(2, N, Re, None, 1e-10, lc.LC_PREC_MIXED)
    assert b
    try:
        for key, ok, bad in (("pdl", (0, 1), (2, -1)), ("graph", (0, 1), (2,)), ("nu1", (1, 4), (0, 5)),
                             ("rhs64", (0, 1), (3,))):
            for v in ok:
                assert L.lc_batch_set_option(b, key.encode(), float(v)) == lc.LC_OK, (key, v)
            for v in bad:
                assert L.lc_batch_set_option(b, key.encode(), float(v)) == lc.LC_ERR_ARG, (key, v)
        assert L.lc_batch_set_option(b, b"nonsense", 1.0) == lc.LC_ERR_ARG
    finally:
        L.lc_batch_destroy(b)
    bad_N = (ctypes.c_int * 1)(100)
    assert not L.lc_batch_create(1, bad_N, Re, None, 1e-10, lc.LC_PREC_MIXED)
    assert not L.lc_batch_create(2, N, Re, None, 1e-10, lc.LC_PREC_FP64)


def test_noalloc_monitor_rejects_bad_arguments_on_the_host(L):
    """lc_monitor_noalloc checks its sizes and pointers before any CUDA call,
    so these run without a device; the pointers are never dereferenced."""
    p = 4096  # a non-NULL address that no check reads
    assert lc.lc_monitor_noalloc(lc.LC_NOALLOC_MAX_N + 1, p, p, p, p, 10**5, 1.0, p) == lc.LC_ERR_SIZE
    assert "LC_NOALLOC_MAX_N" in lc.last_error()
    assert lc.lc_monitor_noalloc(8, p, p, p, p, 8, 1.0, p) == lc.LC_ERR_ARG  # pitch < N + 1
    assert lc.lc_monitor_noalloc(8, 0, p, p, p, 9, 1.0, p) == lc.LC_ERR_ARG  # NULL array
    assert lc.lc_monitor_noalloc(8, p, p, p, p, 9, 1.0, 0) == lc.LC_ERR_ARG  # NULL output
    assert lc.lc_monitor_noalloc(8, p, p, p, p, 9, 0.0, p) == lc.LC_ERR_ARG  # dt <= 0
    assert lc.lc_monitor_noalloc(0, p, p, p, p, 9, 1.0, p) == lc.LC_ERR_ARG  # N < 1


def _levels(N):
    n, lv = N, 1
    while n % 2 == 0 and n >= 4:
        n //= 2
        lv += 1
    return lv


@pytest.mark.parametrize("N", [8, 10, 12, 14, 16, 24, 32, 40, 56, 96, 128, 160, 224, 320, 384, 768, 1024, 2048, 8192])
def test_exact_coarse_level_choice(L, N):
    """The V-cycle ends at the first level below the fine one with at most 16
    intervals (the exact solve), or, with coarse_direct = 0, at the 2-, 3-, 5-
    or 7-interval grid: the same rule the oracle's mg_set_direct applies."""
    h = lc.lc_create(N, 1000.0, 0.0, 1e-10)
    first = next(l for l in range(1, _levels(N)) if N >> l <= 16)
    assert lc.lc_get_params(h)[5] == first + 1
    assert lc.lc_set_option(h, "coarse_direct", 0) == lc.LC_OK
    assert lc.lc_get_params(h)[5] == _levels(N)
    lc.lc_destroy(h)
