"""The GPU finite-difference variant (lbm_step_fd: Sec. III forward Euler with
third-order upwind convection) against the oracle's, element by element:
FP64 <= 1e-12, FP32 <= 1e-5 on small-amplitude random fields (lambda = 0.05,
tau 0.8: inside the scheme's stability range), both boundary kinds, D2Q37 and
D3Q107; 16-bit storage on the smooth recipe within its stated bounds; totals
conserved on a periodic box."""
import numpy as np
import pytest

import lbm_inputs as li
from oracle import oracle as ora
from tests.parity import TOL, assert_parity, parity_errors

pytestmark = pytest.mark.gpu

P, ZG = ora.PERIODIC, ora.ZERO_GRADIENT
LAM = 0.05


def run_pair(lat, shape, bc, prec, steps, fields, tau_f=0.8, tau_g=0.8, lam=LAM, gamma=1.4, **kw):
    from paper_1608_06345_gb300 import lbm
    o = ora.Oracle(lat, gamma, tau_f, tau_g, shape, bc=bc)
    o.init(*fields)
    o.step_fd(steps, lam)
    ref = o.moments()
    cref = o.conserved()
    s = lbm.Solver(lat, gamma, tau_f, tau_g, shape, bc=bc, prec=prec, **kw)
    s.init(*fields)
    s.step_fd(steps, lam)
    got = s.moments()
    cg = s.conserved()
    s.close()
    return got, ref, cg, cref


CASES = [
    (0, (300, 7), (P, P), 40),
    (0, (131, 5), (ZG, P), 40),
    (0, (64, 1), (P, P), 30),
    (1, (40, 5, 6), (ZG, P, P), 8),
    (1, (9, 7, 5), (P, ZG, ZG), 8),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("lat,shape,bc,steps", CASES)
def test_fd_parity(lat, shape, bc, steps, prec):
    D = len(shape)
    fields = li.random_fields(int(np.prod(shape)), D, seed=sum(shape), u_amp=0.02, rho_amp=0.02, T_amp=0.02)
    got, ref, _, _ = run_pair(lat, shape, bc, prec, steps, fields)
    assert_parity(got, ref, 1.4, TOL["f64" if prec == 0 else "f32"])


def test_fd_conserves_on_the_gpu():
    shape = (48, 40)
    fields = li.random_fields(48 * 40, 2, seed=5, u_amp=0.02, rho_amp=0.02, T_amp=0.02)
    from paper_1608_06345_gb300 import lbm
    s = lbm.Solver(0, 1.4, 0.8, 0.8, shape, prec=0)
    s.init(*fields)
    c0 = s.conserved()
    s.step_fd(100, LAM)
    c1 = s.conserved()
    s.close()
    scale = np.array([c0[0]] * 3 + [c0[-1]])
    assert np.all(np.abs(c1 - c0) / scale < 1e-13)


# Stated bounds, larger than for exact streaming: each finite-difference step
# changes a population by only lambda times its gradient, close to the
# resolution of a 16-bit deviation, so storage rounding accumulates over
# many more steps per unit time (measured 2.2e-3 FP16, 4.0e-2 BF16).
@pytest.mark.parametrize("prec,bound", [(2, 5e-3), (3, 6e-2)])
def test_fd_16bit_storage_on_the_smooth_recipe(prec, bound):
    shape = (256, 256)
    fields = li.fourier_fields(shape, seed_u=1, seed_rho=2)
    got, ref, _, _ = run_pair(0, shape, (P, P), prec, 100, fields, tau_f=0.55, tau_g=0.7, lam=0.03)
    e = parity_errors(got, ref, 1.4)
    assert max(e.values()) <= bound, e


def test_fd_rejects_bad_lambda():
    from paper_1608_06345_gb300 import lbm
    s = lbm.Solver(0, 1.4, 0.8, 0.8, (16, 4), prec=1)
    with pytest.raises(lbm.LbmError) as ei:
        s.step_fd(1, 0.0)
    assert ei.value.code == lbm.LBM_EINVAL
    s.close()


# D3Q107, 30 steps: measured 6.9e-4 (FP16) and 5.4e-3 (BF16), on u.
@pytest.mark.parametrize("prec,bound", [(2, 2e-3), (3, 2e-2)])
def test_fd_16bit_storage_3d(prec, bound):
    """D3Q107 finite-difference step with 16-bit storage on a 32^3 box of the
    3D recipe (lambda 0.03, 30 steps) against the FP64 oracle."""
    shape = (32, 32, 32)
    fields = li.fourier_fields(shape, seed_u=3, seed_rho=4, seed_T=5)
    got, ref, _, _ = run_pair(1, shape, (P, P, P), prec, 30, fields, tau_f=0.6, tau_g=0.6, lam=0.03)
    e = parity_errors(got, ref, 1.4)
    assert max(e.values()) <= bound, e
