"""Every compiled launch shape of the step computes the same scheme (parity
with the oracle for FP64/FP32, agreement with the default shape for 16-bit
storage), and lbm_autotune leaves the instance's state untouched."""
import numpy as np
import pytest

import lbm_inputs as li
from oracle import oracle as ora
from tests.parity import TOL, assert_parity, run_oracle

pytestmark = pytest.mark.gpu

# the second pair: periodic axes shorter than 4 cells (repeated wrap of a
# pull) and rows shorter than one block (mostly-idle tail lanes)
CASES = [(0, (300, 5), (1, 0, 0)), (1, (150, 5, 4), (0, 1, 0)), (0, (7, 3), (0, 0, 0)), (1, (5, 3, 2), (0, 0, 0))]


def run_shape(lat, shape, bc, prec, k, fields, steps):
    from paper_1608_06345_gb300 import lbm
    s = lbm.Solver(lat, 1.4, 0.6, 0.7, shape, bc=bc, prec=prec)
    lbm.lbm_set_shape(s.h, k)
    assert lbm.lbm_get_shape(s.h) == k
    s.init(*fields)
    s.step(steps)
    out = s.moments()
    s.close()
    return out


def shapes(lat, prec):
    from paper_1608_06345_gb300 import lbm
    k = 0
    while lbm.lbm_shape_info(lat, prec, k) is not None:
        k += 1
    return list(range(k))


@pytest.mark.parametrize("lat,shape,bc", CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_every_shape_matches_the_oracle(lat, shape, bc, prec):
    D = len(shape)
    fields = li.random_fields(int(np.prod(shape)), D, seed=17)
    steps = 12
    ref, _ = run_oracle(lat, 1.4, 0.6, 0.7, shape, bc[:D], fields, steps)
    ks = shapes(lat, prec)
    assert len(ks) >= 1
    for k in ks:
        got = run_shape(lat, shape, bc[:D], prec, k, fields, steps)
        assert_parity(got, ref, 1.4, TOL["f64" if prec == 0 else "f32"])


@pytest.mark.parametrize("lat,shape,bc", CASES)
def test_16bit_shapes_agree(lat, shape, bc):
    D = len(shape)
    fields = li.random_fields(int(np.prod(shape)), D, seed=18, u_amp=0.02, rho_amp=0.02, T_amp=0.02)
    base = run_shape(lat, shape, bc[:D], 2, 0, fields, 10)
    for k in shapes(lat, 2)[1:]:
        got = run_shape(lat, shape, bc[:D], 2, k, fields, 10)
        for a, b in zip(got, base):
            assert np.max(np.abs(a - b)) <= 1e-5 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("lat,shape,bc", CASES)
def test_autotune_leaves_the_state_unchanged(lat, shape, bc):
    from paper_1608_06345_gb300 import autotune, lbm
    D = len(shape)
    s = lbm.Solver(lat, 1.4, 0.6, 0.7, shape, bc=bc[:D], prec=1)
    s.init(*li.random_fields(int(np.prod(shape)), D, seed=19))
    s.step(3)
    before = s.moments()
    rec = autotune.tune(s, reps=3, cache_path=None)
    after = s.moments()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    assert rec["index"] in shapes(lat, 1) and rec["us_per_step"] > 0
    assert lbm.lbm_get_shape(s.h) == rec["index"]
    s.close()
