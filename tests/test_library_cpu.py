"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, exports
every entry point of include/lbm.h, rejects invalid arguments before any GPU
work, and its own FP64 lattice table satisfies the quadrature conditions."""
import itertools
import os
import re

import numpy as np
import pytest

from paper_1608_06345_gb300 import build as lbm_build
from paper_1608_06345_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    lbm_build.build()
    return lbm.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    declared = header_functions()
    assert "lbm_create" in declared and "lbm_step" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(declared) == sorted(lbm.EXPORTS)


def test_library_is_built_for_sm_103a():
    # the build passes exactly one -gencode for sm_103a
    assert lbm_build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(lbm_build.LIB)


def gauss_moment(n):
    if n % 2:
        return 0.0
    return float(np.prod(np.arange(n - 1, 0, -2))) if n > 0 else 1.0


@pytest.mark.parametrize("lat,D,Q", [(0, 2, 37), (1, 3, 107)])
def test_library_table_isotropy(lib, lat, D, Q):
    """The library's table (its own solver: linear in w for fixed r, secant
    on r) reproduces the unit-Gaussian moments to degree 9."""
    c, w, r = lbm.lbm_lattice_table(lat)
    assert c.shape == (Q, D)
    assert np.all(c[0] == 0)
    # pairs (c, -c) at (2k+1, 2k+2) with equal weights
    for k in range((Q - 1) // 2):
        assert np.all(c[2 * k + 1] == -c[2 * k + 2]) and w[2 * k + 1] == w[2 * k + 2]
    xi = r * c.astype(np.float64)
    worst = 0.0
    for alpha in itertools.product(range(10), repeat=D):
        if sum(alpha) > 9:
            continue
        lhs = np.sum(w * np.prod(xi ** np.array(alpha), axis=1))
        rhs = np.prod([gauss_moment(a) for a in alpha])
        worst = max(worst, abs(lhs - rhs) / max(1.0, abs(rhs)))
    assert worst < 1e-13
    assert abs(r / 1.19697977 - 1) < 1e-8


@pytest.mark.parametrize("kwargs,msg", [
    (dict(gamma=1.0), "gamma"),
    (dict(gamma=2.5), "delta"),
    (dict(tau_f=0.5), "tau"),
    (dict(tau_g=0.3), "tau"),
    (dict(shape=(0, 4)), "dimensions"),
    (dict(shape=(8, 4, 2)), "nz"),
    (dict(prec=9), "precision"),
    (dict(bc=(5, 0, 0)), "boundary"),
    (dict(lattice=7), "lattice"),
    (dict(shape=(65536, 32768)), "2^31"),
    (dict(shape=(4, 70000)), "65535"),
    (dict(gamma=float("nan")), "gamma"),
    (dict(tau_f=float("nan")), "tau"),
    (dict(lattice=1, shape=(8, 8, 0)), "dimensions"),
])
def test_create_rejects_invalid_arguments(lib, kwargs, msg):
    p = dict(lattice=0, gamma=1.4, tau_f=0.6, tau_g=0.6, shape=(8, 4), prec=lbm.LBM_F32, bc=(0, 0, 0))
    p.update(kwargs)
    g = lbm.make_grid(p["shape"], bc=p["bc"], prec=p["prec"])
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create(p["lattice"], p["gamma"], p["tau_f"], p["tau_g"], g)
    assert ei.value.code == lbm.LBM_EINVAL
    assert msg in str(ei.value)


def test_create_rejects_small_caller_buffer(lib):
    g = lbm.make_grid((16, 4), prec=lbm.LBM_F32)
    need = lbm.lbm_state_bytes(0, g)
    g.device_mem = 256 * 1024
    g.device_bytes = need - 1
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create(0, 1.4, 0.6, 0.6, g)
    assert ei.value.code == lbm.LBM_ENOMEM


def test_state_bytes(lib):
    # two buffers of 2Q planes (N rounded up to 64) plus the tail
    g = lbm.make_grid((100, 3), prec=lbm.LBM_F32)
    n = lbm.lbm_state_bytes(0, g)
    plane = 320  # 300 cells -> 320
    buf = ((2 * 37 * plane * 4 + 255) // 256) * 256
    assert n == 2 * buf + 256 + 256 + 8 * 1024 * 5
    g = lbm.make_grid((100, 3), prec=lbm.LBM_F64)
    assert lbm.lbm_state_bytes(0, g) > n
    assert lbm.lbm_state_bytes(0, lbm.make_grid((0, 3))) == 0


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.lbm_destroy(None) == lbm.LBM_OK
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_sync(None) == lbm.LBM_EINVAL
    assert "NULL" in lbm.lbm_last_error()


def test_missing_library_fails_loudly(monkeypatch):
    """There is no CPU fallback: without the compiled library the binding
    raises instead of computing anything on the host."""
    from paper_1608_06345_gb300 import lbm
    monkeypatch.setattr(lbm, "_lib", None)
    monkeypatch.setattr(lbm, "library_path", lambda: os.path.join(os.path.dirname(__file__), "no_such_liblbm.so"))
    with pytest.raises(ImportError, match="not built"):
        lbm.load()


@pytest.mark.parametrize("lat", [0, 1])
def test_library_table_is_the_exact_solution_rounded(lat):
    """The library's refined (w, r) (its own solver: linear in w at fixed r,
    a secant on r, then a double-double correction) equal the 50-digit
    solution of the isotropy conditions rounded to double, to the last bit."""
    pytest.importorskip("mpmath")
    import ctypes

    from paper_1608_06345_gb300 import lbm
    from tests.isotropy_exact import exact_table, group_weights
    D = 2 if lat == 0 else 3
    q, r = ctypes.c_int(), ctypes.c_double()
    c = np.zeros(107 * D, dtype=np.int32)
    w = np.zeros(107)
    assert lbm.load().lbm_lattice_table(lat, ctypes.byref(q), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                        w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(r)) == 0
    Q = q.value
    wg = group_weights(c[:Q * D].reshape(Q, D), w[:Q])
    we, re_ = exact_table(lat, wg, r.value)
    assert r.value == re_
    assert np.array_equal(wg, we)
