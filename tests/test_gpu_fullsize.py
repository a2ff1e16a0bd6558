"""Parity at full size, in the launch configuration bench.py times (autotuned
shape): 4096^2 D2Q37 (FP32, FP16 and BF16 storage) and 256^3 D3Q107 (FP32 at
gamma 1.4 and 1.3, FP16 storage), seeded Fourier fields; and 272^3 D3Q107
FP32, whose element indices exceed 2^32 (the 64-bit addressing path).

The oracle cannot step these grids in a test, so it checks sampled cells one
by one: after k steps a cell depends only on the cells within 3k of it, so
the oracle runs the (6k+1)-wide patch of initial fields around each sampled
cell for k steps (any boundary: its influence cannot reach the centre in k
steps) and the centre cell must match the GPU's.  Over the full run of the
bench (200 / 100 steps) properties that hold at any size are checked:
finite state, mass and momentum conserved (periodic box; tau_f != tau_g
changes only the energy)."""
import numpy as np
import pytest

import lbm_inputs as li
from oracle import oracle as ora
from tests.parity import TOL

pytestmark = pytest.mark.gpu

K = 3  # steps of the sampled comparison
SAMPLES = 24


def patch(field, shape, center, radius):
    """Periodic patch of a flat field (or (D, N) field) around center."""
    D = len(shape)
    idx = [(np.arange(c - radius, c + radius + 1) % n) for c, n in zip(center, shape)]
    def one(f):
        g = f.reshape(tuple(reversed(shape)))  # (nz, ny, nx) or (ny, nx)
        if D == 2:
            return g[np.ix_(idx[1], idx[0])].reshape(-1)
        return g[np.ix_(idx[2], idx[1], idx[0])].reshape(-1)
    if field.ndim == 2:
        return np.stack([one(f) for f in field])
    return one(field)


def sampled_parity(lat, shape, fields, prec, gamma, tau_f, tau_g, tol, seed=0, tune=True):
    from paper_1608_06345_gb300 import autotune, lbm
    D = len(shape)
    s = lbm.Solver(lat, gamma, tau_f, tau_g, shape, prec=prec)
    s.init(*fields)
    if tune:
        autotune.tune(s, reps=2, cache_path=None)
    s.step(K)
    rho, u, T = s.moments()
    c_before = None
    rng = np.random.default_rng(seed)
    r = 3 * K
    w = 2 * r + 1
    worst = 0.0
    for _ in range(SAMPLES):
        center = [int(rng.integers(0, n)) for n in shape]
        pf = tuple(patch(f, shape, center, r) for f in fields)
        o = ora.Oracle(lat, gamma, tau_f, tau_g, (w,) * D, bc=(ora.ZERO_GRADIENT,) * 3)
        o.init(*pf)
        o.step(K)
        ro, uo, To = o.moments()
        mid = (w ** D) // 2
        cell = center[0] + shape[0] * (center[1] + (shape[1] * center[2] if D == 3 else 0))
        worst = max(worst, abs(rho[cell] - ro[mid]) / abs(ro[mid]), abs(T[cell] - To[mid]) / abs(To[mid]),
                    max(abs(u[a, cell] - uo[a, mid]) for a in range(D)) / 0.02)
        o.close()
    assert worst <= tol, worst
    return s


def test_d2q37_fp32_4096():
    shape = (4096, 4096)
    fields = li.fourier_fields(shape, seed_u=1, seed_rho=2)
    s = sampled_parity(0, shape, fields, 1, 1.4, 0.55, 0.7, TOL["f32"])
    c0 = s.conserved()
    s.step(200 - K)
    c1 = s.conserved()
    s.sync()
    # mass and momentum: FP32 storage rounding only (4 units per step)
    assert abs(c1[0] - c0[0]) / c0[0] <= 4 * 200 * 2.0 ** -24
    assert np.all(np.abs(c1[1:3] - c0[1:3]) / c0[0] <= 4 * 200 * 2.0 ** -24)
    s.close()


def test_d2q37_fp16_storage_4096():
    shape = (4096, 4096)
    fields = li.fourier_fields(shape, seed_u=1, seed_rho=2)
    s = sampled_parity(0, shape, fields, 2, 1.4, 0.55, 0.7, 1e-3)
    s.step(200 - K)
    s.sync()
    s.close()


def test_d3q107_fp32_256():
    shape = (256, 256, 256)
    fields = li.fourier_fields(shape, seed_u=3, seed_rho=4, seed_T=5)
    s = sampled_parity(1, shape, fields, 1, 1.4, 0.6, 0.6, TOL["f32"])
    c0 = s.conserved()
    s.step(100 - K)
    c1 = s.conserved()
    s.sync()
    assert abs(c1[0] - c0[0]) / c0[0] <= 4 * 100 * 2.0 ** -24
    assert abs(c1[-1] - c0[-1]) / c0[-1] <= 4 * 100 * 2.0 ** -24  # tau_f = tau_g: energy too
    s.close()


def test_d3q107_fp32_272_indexes_in_64_bits():
    """272^3 cells: 2Q ps = 214 x 20,123,648 = 4.31e9 element indices, above
    2^32, so the step takes its 64-bit addressing path (below 2^32 it indexes
    in 32 bits).  Default shape, sampled parity and conserved totals."""
    shape = (272, 272, 272)
    assert 2 * 107 * 272 ** 3 > 2 ** 32
    fields = li.fourier_fields(shape, seed_u=3, seed_rho=4, seed_T=5)
    s = sampled_parity(1, shape, fields, 1, 1.4, 0.6, 0.6, TOL["f32"], seed=1, tune=False)
    c0 = s.conserved()
    s.step(7)
    c1 = s.conserved()
    s.sync()
    assert abs(c1[0] - c0[0]) / c0[0] <= 4 * 10 * 2.0 ** -24
    assert abs(c1[-1] - c0[-1]) / c0[-1] <= 4 * 10 * 2.0 ** -24
    s.close()


def test_d3q107_fp32_256_gamma_1_3():
    """The second gamma of the 256^3 workload (delta = 11/3, non-integer)."""
    shape = (256, 256, 256)
    fields = li.fourier_fields(shape, seed_u=3, seed_rho=4, seed_T=5)
    s = sampled_parity(1, shape, fields, 1, 1.3, 0.6, 0.6, TOL["f32"], seed=2)
    c0 = s.conserved()
    s.step(20)
    c1 = s.conserved()
    s.sync()
    assert abs(c1[0] - c0[0]) / c0[0] <= 4 * 23 * 2.0 ** -24
    assert abs(c1[-1] - c0[-1]) / c0[-1] <= 4 * 23 * 2.0 ** -24
    s.close()


def test_d2q37_bf16_storage_4096():
    shape = (4096, 4096)
    fields = li.fourier_fields(shape, seed_u=1, seed_rho=2)
    s = sampled_parity(0, shape, fields, 3, 1.4, 0.55, 0.7, 1e-2, seed=3)
    s.step(200 - K)
    s.sync()
    s.close()


def test_d3q107_fp16_storage_256():
    shape = (256, 256, 256)
    fields = li.fourier_fields(shape, seed_u=3, seed_rho=4, seed_T=5)
    s = sampled_parity(1, shape, fields, 2, 1.4, 0.6, 0.6, 1e-3, seed=4)
    s.step(100 - K)
    s.sync()
    s.close()
