"""The GPU finite-difference variant (lbm_step_fd: Sec. III forward Euler with
third-order upwind convection) against the oracle's, element by element:
FP64 <= 1e-12, FP32 <= 1e-5 on small-amplitude random fields (lambda = 0.05,
tau 0.8: inside the scheme's stability range), both boundary kinds, D2Q37 and
D3Q107; 16-bit storage on the smooth recipe within its stated bounds; totals
conserved on a periodic box.  The marched kernel (LBM_FD_MARCH, D2Q37) is
compared with the per-cell kernel in every storage precision."""
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
    (0, (132, 5), (ZG, ZG), 40),
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


def run_kernel(shape, bc, prec, steps, fields, kernel, lam=LAM):
    from paper_1608_06345_gb300 import lbm
    s = lbm.Solver(0, 1.4, 0.8, 0.7, shape, bc=bc, prec=prec)
    s.set_fd_kernel(kernel)
    s.init(*fields)
    s.step_fd(steps, lam)
    got = s.moments()
    s.close()
    return got


# The marched kernel (blocks of 32 columns walk bands of rows; the (c, -c)
# pairs split over the warps, each streaming its planes through its own
# shared-memory ring) does each value's arithmetic as the per-cell kernel
# and sums the moments in another order, so the two agree to rounding: FP64
# and FP32 within their parity bounds, 16-bit storage within a few units of
# the stored format's last place.  The shapes cover ragged last strips
# (300 = 9 x 32 + 12 columns) and one-row bands, open x (clamped stencil
# columns) with open or periodic y, grids narrower than the stencil's reach,
# and many strips with multi-row bands.
MARCH_CASES = [
    ((300, 7), (P, P), 10),
    ((131, 9), (ZG, P), 10),
    ((260, 13), (ZG, ZG), 10),
    ((8, 9), (P, ZG), 10),
    ((3, 6), (P, P), 10),
    ((520, 400), (P, P), 4),
]
MARCH_TOL = {0: TOL["f64"], 1: TOL["f32"], 2: 2e-3, 3: 2e-2}


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("shape,bc,steps", MARCH_CASES)
def test_fd_march_matches_cell_kernel(shape, bc, steps, prec):
    from paper_1608_06345_gb300 import lbm
    fields = li.random_fields(int(np.prod(shape)), 2, seed=sum(shape) + prec, u_amp=0.02, rho_amp=0.02,
                              T_amp=0.02)
    cell = run_kernel(shape, bc, prec, steps, fields, lbm.LBM_FD_CELL)
    march = run_kernel(shape, bc, prec, steps, fields, lbm.LBM_FD_MARCH)
    e = parity_errors(march, cell, 1.4)
    assert max(e.values()) <= MARCH_TOL[prec], e


def test_fd_march_at_bench_shape_matches_cell_kernel():
    """The bench's finite-difference workload: D2Q37 FP32 4096^2, lambda
    0.03, tau_f 0.55, tau_g 0.7 on the Fourier recipe, 3 steps with each
    kernel."""
    from paper_1608_06345_gb300 import lbm
    shape = (4096, 4096)
    fields = li.fourier_fields(shape, seed_u=1, seed_rho=2)
    res = []
    for kernel in (lbm.LBM_FD_CELL, lbm.LBM_FD_MARCH):
        s = lbm.Solver(0, 1.4, 0.55, 0.7, shape, prec=lbm.LBM_F32)
        s.set_fd_kernel(kernel)
        s.init(*fields)
        s.step_fd(3, 0.03)
        res.append(s.moments())
        s.close()
    e = parity_errors(res[1], res[0], 1.4)
    assert max(e.values()) <= TOL["f32"], e


def test_fd_kernel_choice_is_checked():
    from paper_1608_06345_gb300 import lbm
    s = lbm.Solver(0, 1.4, 0.8, 0.8, (18, 4), prec=1)
    with pytest.raises(lbm.LbmError) as ei:
        s.set_fd_kernel(7)
    assert ei.value.code == lbm.LBM_EINVAL
    s.set_fd_kernel(lbm.LBM_FD_CELL)
    s.set_fd_kernel(lbm.LBM_FD_MARCH)
    s.close()
    s = lbm.Solver(1, 1.4, 0.8, 0.8, (8, 8, 8), prec=1)
    with pytest.raises(lbm.LbmError):
        s.set_fd_kernel(lbm.LBM_FD_MARCH)
    s.set_fd_kernel(lbm.LBM_FD_AUTO)
    s.close()
