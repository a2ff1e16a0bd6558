"""16-bit storage (FP32 arithmetic, populations stored in FP16 / BF16 as
deviations from the instance's reference equilibrium) against the FP64
oracle, with the stated error bounds.

Stated bounds (parity norm of tests/parity.py for L-inf; L1 = mean |error|
over mean |oracle| per field):
  smooth periodic box (512^2, 8 Fourier modes, 200 steps), and the 3D
  recipe on a 48 x 12 x 10 box with zero-gradient y and z ends (L-inf only):
      FP16  L-inf <= 1e-3, L1 <= 5e-4      BF16  L-inf <= 1e-2, L1 <= 5e-3
  the paper's shock tube (1000 x 16, rho 4|1, 180 steps):
      FP16  L-inf <= 5e-2, L1 <= 2e-3      BF16  L-inf <= 0.5,  L1 <= 2e-2
The tube bounds are larger: a density jump of 4 sits far from any single
reference equilibrium, and the shock position is sensitive to round-off."""
import numpy as np
import pytest

import lbm_inputs as li
from oracle import oracle as ora
from tests.parity import parity_errors, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

S16F, S16BF = 2, 3
BOUNDS = {
    ("smooth", S16F): (1e-3, 5e-4), ("smooth", S16BF): (1e-2, 5e-3),
    ("tube", S16F): (5e-2, 2e-3), ("tube", S16BF): (0.5, 2e-2),
}


def l1_rel(gpu, ref):
    out = {}
    for k, a, b in [("rho", gpu[0], ref[0]), ("T", gpu[2], ref[2])] + \
            [(f"u{i}", gpu[1][i], ref[1][i]) for i in range(ref[1].shape[0])]:
        den = np.mean(np.abs(b))
        if den > 1e-3:
            out[k] = float(np.mean(np.abs(a - b)) / den)
    return out


@pytest.fixture(scope="module")
def smooth_ref():
    shape = (512, 512)
    fields = li.fourier_fields(shape, seed_u=1, seed_rho=2)
    ref, _ = run_oracle(ora.D2Q37, 1.4, 0.55, 0.7, shape, (0, 0), fields, 200)
    return shape, fields, ref


@pytest.mark.parametrize("prec", [S16F, S16BF])
def test_periodic_fourier_box(smooth_ref, prec):
    shape, fields, ref = smooth_ref
    gpu, _ = run_gpu(0, 1.4, 0.55, 0.7, shape, (0, 0), fields, 200, prec)
    linf, l1 = BOUNDS[("smooth", prec)]
    e = parity_errors(gpu, ref, 1.4)
    assert max(e.values()) <= linf, e
    e1 = l1_rel(gpu, ref)
    assert max(e1.values()) <= l1, e1


@pytest.fixture(scope="module")
def tube_ref():
    shape, bc = (1000, 16), (ora.ZERO_GRADIENT, ora.PERIODIC)
    fields = li.sod_fields(1000, 16, left=(4.0, 0.0, 1.0), right=(1.0, 0.0, 1.0))
    ref, _ = run_oracle(ora.D2Q37, 1.4, 2 / 3, 2 / 3, shape, bc, fields, 180)
    return shape, bc, fields, ref


@pytest.mark.parametrize("prec", [S16F, S16BF])
def test_paper_shock_tube(tube_ref, prec):
    shape, bc, fields, ref = tube_ref
    # reference state of the codec: the volume-averaged density and pressure
    rho0 = 0.5 * (4.0 + 1.0)
    T0 = 0.5 * (4.0 * 1.0 + 1.0 * 1.0) / rho0
    gpu, _ = run_gpu(0, 1.4, 2 / 3, 2 / 3, shape, bc, fields, 180, prec, rho0=rho0, T0=T0)
    linf, l1 = BOUNDS[("tube", prec)]
    e = parity_errors(gpu, ref, 1.4)
    assert max(e.values()) <= linf, e
    e1 = l1_rel(gpu, ref)
    assert max(e1.values()) <= l1, e1


def test_reference_state_changes_only_the_representation():
    """A non-unit reference state (rho0 = 0.6, T0 = 1.3) is an exact change
    of variables: FP64 results stay within 1e-12 of the oracle."""
    shape, bc = (300, 5), (ora.ZERO_GRADIENT, ora.PERIODIC)
    fields = li.random_fields(1500, 2, seed=31)
    ref, _ = run_oracle(ora.D2Q37, 1.4, 0.6, 0.6, shape, bc, fields, 60)
    gpu, _ = run_gpu(0, 1.4, 0.6, 0.6, shape, bc, fields, 60, 0, rho0=0.6, T0=1.3)
    e = parity_errors(gpu, ref, 1.4)
    assert max(e.values()) <= 1e-12, e


@pytest.mark.parametrize("prec", [S16F, S16BF])
def test_d3q107_16bit_interior_and_border_launches(prec):
    """D3Q107 with 16-bit storage on a grid whose step runs as an interior and
    a border launch (Ny, Nz >= 7), with zero-gradient y and z ends, so the
    border rows clamp their pulls: the smooth 3D recipe, 20 steps, against
    the FP64 oracle within the smooth-field bounds."""
    shape, bc = (48, 12, 10), (ora.PERIODIC, ora.ZERO_GRADIENT, ora.ZERO_GRADIENT)
    fields = li.fourier_fields(shape, seed_u=3, seed_rho=4, seed_T=5)
    ref, _ = run_oracle(ora.D3Q107, 1.4, 0.6, 0.6, shape, bc, fields, 20)
    gpu, _ = run_gpu(1, 1.4, 0.6, 0.6, shape, bc, fields, 20, prec)
    e = parity_errors(gpu, ref, 1.4)
    assert max(e.values()) <= BOUNDS[("smooth", prec)][0], e
