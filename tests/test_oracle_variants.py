"""The oracle's rounding variants (ORA_VARIANT in oracle/lbm_oracle.c) are
second checkers: the shock-tube parity tests allow the library twice the
distance at which they land from the oracle.  A variant that computed
something else would inflate that tolerance, so each one is pinned here:

- on a well-conditioned flow (periodic random fields) every FP64 variant
  agrees with the oracle within the FP64 bar 1e-12 (measured: 2e-13 at
  most), and every FP32 variant within 1e-4 (measured: 6e-5 at most, the
  velocity of a flow at rest to 1%, whose momentum a plain FP32 sum over
  the populations resolves to about 5e-7): they compute the same scheme;
  a dropped term or a wrong sign moves the result by far more;
- every variant does round differently from the oracle (its result is not
  bitwise the oracle's, and an FP32 variant is not within FP64 round-off):
  the build option took effect;
- the deviation variant conserves mass, momentum and energy to round-off on
  a periodic box with tau_f = tau_g (the collision invariants of
  Eq. (14)), and its reference state is an exact change of variables;
- only the deviation builds accept a reference state."""
import numpy as np
import pytest

import lbm_inputs as li
from oracle import oracle as ora
from tests.parity import parity_errors

CASE = dict(shape=(30, 20), bc=(ora.PERIODIC, ora.PERIODIC), gamma=1.4, tau_f=0.6, tau_g=0.7, steps=20)


def run(variant, ref_state=None, lattice=ora.D2Q37, case=CASE, fields=None):
    c = case
    N = int(np.prod(c["shape"]))
    D = len(c["shape"])
    if fields is None:
        fields = li.random_fields(N, D, seed=11)
    o = ora.Oracle(lattice, c["gamma"], c["tau_f"], c["tau_g"], c["shape"], bc=c["bc"], variant=variant)
    if ref_state is not None:
        o.set_reference(*ref_state)
    o.init(*fields)
    o.step(c["steps"])
    out = o.moments(), o.conserved()
    o.close()
    return out


@pytest.fixture(scope="module")
def oracle_result():
    return run(0)


@pytest.mark.parametrize("variant", ora.VARIANTS_F64)
def test_fp64_variant_computes_the_same_scheme(variant, oracle_result):
    (m, c), (m0, c0) = run(variant), oracle_result
    e = max(parity_errors(m, m0, CASE["gamma"]).values())
    assert e <= 1e-12, e
    assert np.all(np.abs(c - c0) <= 1e-13 * abs(c0[0]))
    # and rounds differently somewhere
    assert any(not np.array_equal(a, b) for a, b in zip(m, m0))


@pytest.mark.parametrize("variant", ora.VARIANTS_F32)
def test_fp32_variant_computes_the_same_scheme_in_fp32(variant, oracle_result):
    (m, _), (m0, _) = run(variant), oracle_result
    e = max(parity_errors(m, m0, CASE["gamma"]).values())
    assert 1e-9 < e <= 1e-4, e


@pytest.mark.parametrize("variant", [8, 15])
def test_deviation_variant_conserves_the_totals(variant):
    case = dict(CASE, tau_g=0.6, steps=40)
    fields = li.random_fields(600, 2, seed=3)
    c_init = run(variant, case=dict(case, steps=0), fields=fields)[1]
    c_end = run(variant, case=case, fields=fields)[1]
    scale = np.array([c_init[0]] * 3 + [c_init[-1]])
    assert np.all(np.abs(c_end - c_init) / scale <= 1e-13)


def test_deviation_reference_state_is_a_change_of_variables():
    fields = li.random_fields(600, 2, seed=4)
    (m1, c1), (m2, c2) = run(8, (1.0, 1.0), fields=fields), run(8, (0.6, 1.3), fields=fields)
    assert max(parity_errors(m1, m2, CASE["gamma"]).values()) <= 1e-12
    assert np.all(np.abs(c1 - c2) <= 1e-13 * abs(c1[0]))


def test_deviation_variant_in_3d():
    case = dict(shape=(7, 6, 5), bc=(ora.PERIODIC,) * 3, gamma=1.3, tau_f=0.6, tau_g=0.6, steps=6)
    fields = li.random_fields(210, 3, seed=5)
    (m0, c0) = run(0, lattice=ora.D3Q107, case=case, fields=fields)
    (m, c) = run(15, (0.9, 1.1), lattice=ora.D3Q107, case=case, fields=fields)
    assert max(parity_errors(m, m0, 1.3).values()) <= 1e-12
    assert np.all(np.abs(c - c0) <= 1e-13 * abs(c0[0]))


@pytest.mark.parametrize("variant", [0, 1, 2, 4, 16])
def test_whole_storage_builds_refuse_a_reference_state(variant):
    o = ora.Oracle(ora.D2Q37, 1.4, 0.6, 0.6, (4, 4), variant=variant)
    with pytest.raises(ValueError):
        o.set_reference(1.0, 1.0)
    o.close()
