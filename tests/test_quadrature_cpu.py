"""The library's general Hermite-quadrature generator (lbm_quadrature, the
construction of Sec. IV for any symmetric integer velocity set) against the
textbook Gauss-Hermite lattices with closed-form weights (r = sqrt 3):
D1Q3 (2/3, 1/6), D2Q9 (4/9, 1/9, 1/36), D3Q15 (2/9, 1/9, 1/72), D3Q19 (1/3,
1/18, 1/36), D3Q27 (8/27, 2/27, 1/54, 1/216); it reproduces the paper's
D2Q37 / D3Q107 tables; a higher-order set (D2Q17) is checked by brute-force
isotropy of the velocity set it returns."""
import itertools
import math

import numpy as np
import pytest

from paper_1608_06345_gb300 import build as lbm_build
from paper_1608_06345_gb300 import lbm


@pytest.fixture(scope="module", autouse=True)
def lib():
    lbm_build.build()
    return lbm.load()


R3 = math.sqrt(3.0)
CLOSED = [
    ("D1Q3", [[0], [1]], [[0], [2], [4]], [2 / 3, 1 / 6], 3),
    ("D2Q9", [[0, 0], [1, 0], [1, 1]], [[0, 0], [2, 0], [4, 0], [2, 2]], [4 / 9, 1 / 9, 1 / 36], 9),
    ("D3Q15", [[0, 0, 0], [1, 0, 0], [1, 1, 1]], [[0, 0, 0], [2, 0, 0], [4, 0, 0], [2, 2, 0]],
     [2 / 9, 1 / 9, 1 / 72], 15),
    ("D3Q19", [[0, 0, 0], [1, 0, 0], [1, 1, 0]], [[0, 0, 0], [2, 0, 0], [4, 0, 0], [2, 2, 0]],
     [1 / 3, 1 / 18, 1 / 36], 19),
    ("D3Q27", [[0, 0, 0], [1, 0, 0], [1, 1, 0], [1, 1, 1]],
     [[0, 0, 0], [2, 0, 0], [4, 0, 0], [2, 2, 0], [2, 2, 2]], [8 / 27, 2 / 27, 1 / 54, 1 / 216], 27),
]


@pytest.mark.parametrize("name,reps,exps,w_exact,Q", CLOSED)
def test_textbook_lattices(name, reps, exps, w_exact, Q):
    w, r, q, res = lbm.lbm_quadrature(reps, exps, r0=1.6)
    assert q == Q
    assert abs(r - R3) < 1e-13
    np.testing.assert_allclose(w, w_exact, rtol=1e-13)
    assert res < 1e-13


def test_fixed_r_keeps_r():
    w, r, q, _ = lbm.lbm_quadrature([[0, 0], [1, 0], [1, 1]], [[0, 0], [2, 0], [2, 2]], r0=R3)
    assert r == R3
    np.testing.assert_allclose(w, [4 / 9, 1 / 9, 1 / 36], rtol=1e-13)


@pytest.mark.parametrize("lat,reps,exps", [
    (0, [[0, 0], [1, 0], [1, 1], [2, 0], [2, 1], [3, 0], [3, 1], [3, 3]],
     [[0, 0], [2, 0], [4, 0], [2, 2], [6, 0], [4, 2], [8, 0], [6, 2], [4, 4]]),
    (1, [[0, 0, 0], [1, 0, 0], [1, 1, 0], [1, 1, 1], [2, 0, 0], [2, 1, 1], [2, 2, 0], [2, 2, 2], [3, 0, 0],
         [3, 1, 1]],
     [[0, 0, 0], [2, 0, 0], [4, 0, 0], [2, 2, 0], [6, 0, 0], [4, 2, 0], [2, 2, 2], [8, 0, 0], [6, 2, 0], [4, 4, 0],
      [4, 2, 2]]),
])
def test_reproduces_the_paper_tables(lat, reps, exps):
    w, r, q, res = lbm.lbm_quadrature(reps, exps, r0=1.19)
    c, wt, rt = lbm.lbm_lattice_table(lat)
    assert q == len(wt) and abs(r - rt) < 1e-13
    D = len(reps[0])
    for g, rep in enumerate(reps):
        i = next(i for i, v in enumerate(c) if sorted(np.abs(v), reverse=True) == sorted(rep, reverse=True)[:D])
        assert abs(w[g] / wt[i] - 1) < 1e-12


def velocity_set(reps):
    D = len(reps[0])
    M = max(max(abs(x) for x in rep) for rep in reps)
    out = []
    for g, rep in enumerate(reps):
        key = sorted(np.abs(rep), reverse=True)
        for v in itertools.product(range(-M, M + 1), repeat=D):
            if sorted(np.abs(v), reverse=True) == key:
                out.append((g, v))
    return out


def test_higher_order_set_is_isotropic():
    """D2Q17 groups (0,0),(1,0),(1,1),(2,2),(3,0) with the even classes up to
    degree 6: every moment of degree <= 7 must be Gaussian."""
    reps = [[0, 0], [1, 0], [1, 1], [2, 2], [3, 0]]
    exps = [[0, 0], [2, 0], [4, 0], [2, 2], [6, 0], [4, 2]]
    w, r, q, res = lbm.lbm_quadrature(reps, exps, r0=1.6)
    vs = velocity_set(reps)
    assert q == len(vs) == 17
    for a in itertools.product(range(8), repeat=2):
        if sum(a) > 7:
            continue
        lhs = sum(w[g] * (r * v[0]) ** a[0] * (r * v[1]) ** a[1] for g, v in vs)
        gm = lambda n: 0.0 if n % 2 else float(np.prod(np.arange(n - 1, 0, -2))) if n else 1.0
        assert abs(lhs - gm(a[0]) * gm(a[1])) < 1e-12 * max(1.0, gm(a[0]) * gm(a[1]))


@pytest.mark.parametrize("reps,exps,msg", [
    ([[0, 0], [1, 0]], [[0, 0], [2, 0], [4, 0], [2, 2]], "conditions"),
    ([[0, 0], [1, 0], [1, 1]], [[0, 0], [1, 0], [4, 0], [2, 2]], "even"),
])
def test_rejects_bad_problems(reps, exps, msg):
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_quadrature(reps, exps, r0=1.6)
    assert ei.value.code == lbm.LBM_EINVAL and msg in str(ei.value)
