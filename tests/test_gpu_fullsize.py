"""Parity at full size, in the launch configuration bench.py times (autotuned
shape): 4096^2 D2Q37 (FP32, FP16 and BF16 storage) and 256^3 D3Q107 (FP32 at
gamma 1.4 and 1.3, FP16 storage), seeded Fourier fields; and 272^3 D3Q107
FP32, whose element indices exceed 2^32 (the 64-bit addressing path).

The oracle cannot step these grids in a test, so it steps a patch of them:
after K steps a cell depends only on the cells within 3K of it (|c_i| <= 3
per axis), so the oracle runs the initial fields of a periodic patch of
6K + M cells per axis (any boundary will do: its influence reaches only 3K
cells into the patch in K steps) and the central M^D cells of the patch
must match the GPU's, cell by cell.  The 2D patch runs the bench's full 200
steps (1263^2 cells, M = 63); the 3D patches run 20 steps (135^3, M = 15).
Each patch is placed across the periodic corner of the grid, so its cells
pull across both ends of every axis.  One oracle patch serves every storage
precision of the same fields.  Over the full run of the bench (200 / 100
steps) properties that hold at any size are checked as well: finite state,
mass and momentum conserved (periodic box; tau_f != tau_g changes only the
energy)."""
import numpy as np
import pytest

import lbm_inputs as li
from oracle import oracle as ora
from tests.parity import TOL

pytestmark = pytest.mark.gpu

K2, M2 = 200, 63   # 2D: the bench's 200 steps
K3, M3 = 20, 15    # 3D


def patch(field, shape, start, width):
    """Periodic patch of a flat field (or a (D, N) field) whose first cell is
    `start` (per axis) and which is `width` cells wide per axis."""
    D = len(shape)
    idx = [np.arange(s, s + width) % n for s, n in zip(start, shape)]

    def one(f):
        g = f.reshape(tuple(reversed(shape)))  # (nz, ny, nx) or (ny, nx)
        if D == 2:
            return g[np.ix_(idx[1], idx[0])].reshape(-1)
        return g[np.ix_(idx[2], idx[1], idx[0])].reshape(-1)
    if field.ndim == 2:
        return np.stack([one(f) for f in field])
    return one(field)


def valid_block(shape, K, M):
    """Patch origin, width and the first grid cell of its M^D valid cells: a
    block that starts M // 2 cells before the end of each axis and wraps
    past it."""
    vstart = [n - M // 2 for n in shape]
    start = [v - 3 * K for v in vstart]
    width = 6 * K + M
    return start, width, vstart


def oracle_patch(lat, shape, fields, gamma, tau_f, tau_g, K, M):
    """rho, u, T of the oracle on the valid M^D cells after K steps, in the
    order x fastest."""
    D = len(shape)
    start, width, _ = valid_block(shape, K, M)
    pf = tuple(patch(f, shape, start, width) for f in fields)
    o = ora.Oracle(lat, gamma, tau_f, tau_g, (width,) * D, bc=(ora.ZERO_GRADIENT,) * 3)
    o.init(*pf)
    o.step(K)
    rho, u, T = o.moments()
    o.close()
    sel = np.arange(3 * K, 3 * K + M)
    if D == 2:
        take = lambda q: q.reshape(width, width)[np.ix_(sel, sel)].reshape(-1)
    else:
        take = lambda q: q.reshape(width, width, width)[np.ix_(sel, sel, sel)].reshape(-1)
    return take(rho), np.stack([take(c) for c in u]), take(T)


def gpu_block(shape, moments, K, M):
    """The same M^D cells of the GPU's full-grid moments."""
    _, _, vstart = valid_block(shape, K, M)
    rho, u, T = moments
    return patch(rho, shape, vstart, M), patch(u, shape, vstart, M), patch(T, shape, vstart, M)


def errors(g, o, gamma, u_scale):
    """Parity norm over the block: rho and T relative to max |oracle|; u per
    component relative to the field's velocity scale u_scale[a] (max |u_a|
    of the initial field, as the whole-field parity norm would take it; a
    block of the field need not contain the field's largest velocity)."""
    e = {"rho": np.max(np.abs(g[0] - o[0])) / np.max(np.abs(o[0])),
         "T": np.max(np.abs(g[2] - o[2])) / np.max(np.abs(o[2]))}
    for a in range(o[1].shape[0]):
        e[f"u{a}"] = np.max(np.abs(g[1][a] - o[1][a])) / max(u_scale[a], 1e-3 * np.sqrt(gamma))
    return e


def run_gpu(lat, shape, fields, prec, gamma, tau_f, tau_g, K, tune=True):
    from paper_1608_06345_gb300 import autotune, lbm
    s = lbm.Solver(lat, gamma, tau_f, tau_g, shape, prec=prec)
    s.init(*fields)
    if tune:
        autotune.tune(s, reps=2, cache_path=None)
    c0 = s.conserved()
    s.step(K)
    return s, s.moments(), c0


def check_block(name, s_moments, ref, shape, gamma, K, M, tol, fields):
    e = errors(gpu_block(shape, s_moments, K, M), ref, gamma, np.max(np.abs(fields[1]), axis=1))
    print(f"FULLSIZE {name}: {M ** len(shape)} cells after {K} steps, max parity error {max(e.values()):.3e}")
    assert max(e.values()) <= tol, e


@pytest.fixture(scope="module")
def fields_2d():
    return li.fourier_fields((4096, 4096), seed_u=1, seed_rho=2)


@pytest.fixture(scope="module")
def oracle_2d(fields_2d):
    return oracle_patch(0, (4096, 4096), fields_2d, 1.4, 0.55, 0.7, K2, M2)


@pytest.fixture(scope="module")
def fields_3d():
    return li.fourier_fields((256, 256, 256), seed_u=3, seed_rho=4, seed_T=5)


@pytest.fixture(scope="module")
def oracle_3d(fields_3d):
    return oracle_patch(1, (256, 256, 256), fields_3d, 1.4, 0.6, 0.6, K3, M3)


@pytest.mark.parametrize("prec,tol", [(1, TOL["f32"]), (2, 1e-3), (3, 1e-2)])
def test_d2q37_4096_full_run(prec, tol, fields_2d, oracle_2d):
    """The bench workload: D2Q37 4096^2, gamma 1.4, tau_f 0.55, tau_g 0.7,
    the full 200 steps, compared on 63^2 cells across the periodic corner;
    FP32 to 1e-5, FP16 / BF16 storage to their stated 1e-3 / 1e-2."""
    shape = (4096, 4096)
    s, m, c0 = run_gpu(0, shape, fields_2d, prec, 1.4, 0.55, 0.7, K2)
    check_block(f"D2Q37 4096^2 prec {prec}", m, oracle_2d, shape, 1.4, K2, M2, tol, fields_2d)
    c1 = s.conserved()
    s.close()
    if prec == 1:  # mass and momentum: FP32 storage rounding only (4 units per step)
        assert abs(c1[0] - c0[0]) / c0[0] <= 4 * K2 * 2.0 ** -24
        assert np.all(np.abs(c1[1:3] - c0[1:3]) / c0[0] <= 4 * K2 * 2.0 ** -24)


@pytest.mark.parametrize("prec,tol", [(1, TOL["f32"]), (2, 1e-3)])
def test_d3q107_256(prec, tol, fields_3d, oracle_3d):
    """The 3D workload: D3Q107 256^3, gamma 1.4, tau 0.6; 20 steps compared
    on 15^3 cells across the periodic corner, then the rest of the bench's
    100 steps with mass and energy conserved (tau_f = tau_g)."""
    shape = (256, 256, 256)
    s, m, c0 = run_gpu(1, shape, fields_3d, prec, 1.4, 0.6, 0.6, K3)
    check_block(f"D3Q107 256^3 prec {prec}", m, oracle_3d, shape, 1.4, K3, M3, tol, fields_3d)
    s.step(100 - K3)
    c1 = s.conserved()
    s.sync()
    s.close()
    if prec == 1:
        assert abs(c1[0] - c0[0]) / c0[0] <= 4 * 100 * 2.0 ** -24
        assert abs(c1[-1] - c0[-1]) / c0[-1] <= 4 * 100 * 2.0 ** -24


def test_d3q107_fp32_256_gamma_1_3(fields_3d):
    """The second gamma of the 256^3 workload (delta = 11/3, non-integer)."""
    shape = (256, 256, 256)
    ref = oracle_patch(1, shape, fields_3d, 1.3, 0.6, 0.6, K3, M3)
    s, m, c0 = run_gpu(1, shape, fields_3d, 1, 1.3, 0.6, 0.6, K3)
    check_block("D3Q107 256^3 gamma 1.3", m, ref, shape, 1.3, K3, M3, TOL["f32"], fields_3d)
    c1 = s.conserved()
    s.close()
    assert abs(c1[0] - c0[0]) / c0[0] <= 4 * K3 * 2.0 ** -24
    assert abs(c1[-1] - c0[-1]) / c0[-1] <= 4 * K3 * 2.0 ** -24


def test_d3q107_fp32_272_indexes_in_64_bits():
    """272^3 cells: 2Q ps = 214 x 20,123,648 = 4.31e9 element indices, above
    2^32, so the step takes its 64-bit addressing path (below 2^32 it indexes
    in 32 bits).  Default shape; 5 steps on 7^3 cells across the corner."""
    shape = (272, 272, 272)
    assert 2 * 107 * 272 ** 3 > 2 ** 32
    K, M = 5, 7
    fields = li.fourier_fields(shape, seed_u=3, seed_rho=4, seed_T=5)
    ref = oracle_patch(1, shape, fields, 1.4, 0.6, 0.6, K, M)
    s, m, c0 = run_gpu(1, shape, fields, 1, 1.4, 0.6, 0.6, K, tune=False)
    check_block("D3Q107 272^3 (64-bit indexing)", m, ref, shape, 1.4, K, M, TOL["f32"], fields)
    c1 = s.conserved()
    s.close()
    assert abs(c1[0] - c0[0]) / c0[0] <= 4 * K * 2.0 ** -24
    assert abs(c1[-1] - c0[-1]) / c0[-1] <= 4 * K * 2.0 ** -24
