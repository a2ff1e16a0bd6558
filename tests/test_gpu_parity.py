"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs, element by element on rho, u, T.

Tolerances: FP64 <= 1e-12, FP32 <= 1e-5 (relative, parity norm of
tests/parity.py) on well-conditioned flows (random and Fourier-mode fields).
Shock tubes amplify round-off: two correct FP64 evaluations of the classic
Sod tube differ by up to 5e-11 after 500 steps.  There the tolerance is
twice the largest distance at which the oracle's rounding variants land
from the oracle on the same case (tests/parity.py, run_variants and
spread_tolerance), and never below the bar.  Sizes span several thread
blocks with a ragged tail (D2Q37 blocks are 128 cells along x, D3Q107 blocks
64), Ny and Nz below the stencil width 7, and both boundary kinds."""
import numpy as np
import pytest

import lbm_inputs as li
from oracle import oracle as ora
from tests.parity import (TOL, assert_parity, library_reference, report, run_gpu, run_oracle, run_variants,
                          spread_tolerance)

pytestmark = pytest.mark.gpu

P, ZG = ora.PERIODIC, ora.ZERO_GRADIENT
F64, F32 = 0, 1


def fields_for(shape, seed):
    D = len(shape)
    N = int(np.prod(shape))
    return li.random_fields(N, D, seed=seed)


CASES_2D = [
    # shape, bc, gamma, tau_f, tau_g, steps
    ((300, 7), (P, P), 1.4, 0.6, 0.6, 40),
    ((37, 4), (P, P), 1.4, 0.55, 0.7, 60),
    ((131, 5), (ZG, P), 1.3, 0.8, 0.65, 50),
    ((64, 1), (P, P), 1.1, 0.6, 0.6, 30),
    ((5, 9), (ZG, ZG), 5.0 / 3.0, 0.9, 0.9, 20),
    ((1, 1), (P, P), 1.4, 0.6, 0.6, 5),
]


@pytest.mark.parametrize("prec", [F64, F32])
@pytest.mark.parametrize("case", CASES_2D)
def test_d2q37_random_fields(case, prec):
    shape, bc, gamma, tf, tg, steps = case
    fields = fields_for(shape, seed=sum(shape) + steps)
    ref, _ = run_oracle(ora.D2Q37, gamma, tf, tg, shape, bc, fields, steps)
    gpu, _ = run_gpu(0, gamma, tf, tg, shape, bc, fields, steps, prec)
    assert_parity(gpu, ref, gamma, TOL["f64" if prec == F64 else "f32"])


CASES_3D = [
    ((150, 5, 6), (P, P, P), 1.4, 0.6, 0.6, 12),
    ((20, 3, 4), (ZG, P, P), 1.3, 0.7, 0.8, 15),
    ((9, 7, 5), (P, ZG, ZG), 5.0 / 3.0, 0.6, 0.6, 10),
    # Ny, Nz >= 7: the step runs as an interior and a border launch (the border
    # rows pull across y and z faces, wrapped or clamped)
    ((40, 9, 8), (P, ZG, ZG), 1.4, 0.6, 0.7, 8),
    ((24, 11, 7), (ZG, P, ZG), 1.3, 0.65, 0.65, 8),
    ((70, 8, 10), (P, P, P), 1.4, 0.6, 0.6, 8),
]


@pytest.mark.parametrize("prec", [F64, F32])
@pytest.mark.parametrize("case", CASES_3D)
def test_d3q107_random_fields(case, prec):
    shape, bc, gamma, tf, tg, steps = case
    fields = fields_for(shape, seed=sum(shape) + steps)
    ref, _ = run_oracle(ora.D3Q107, gamma, tf, tg, shape, bc, fields, steps)
    gpu, _ = run_gpu(1, gamma, tf, tg, shape, bc, fields, steps, prec)
    assert_parity(gpu, ref, gamma, TOL["f64" if prec == F64 else "f32"])


def rows_equal(q, nrows, nx):
    """The state of a tube that is uniform across it stays bitwise uniform:
    every row equals row 0."""
    r = q.reshape(nrows, nx)
    return bool(np.all(r == r[0]))


def tube_parity(name, lat, shape, fields_full, fields_row, gamma, tau, steps, prec, rho0=0.0):
    """GPU run on the full tube cross-section; the oracle and its rounding
    variants on one row (the tube is uniform across, so every row of the GPU
    state must equal row 0 bitwise, and one row is the same computation per
    cell).  Fields, u and totals are compared against the variants'
    spread; the deviation variants take the instance's reference state."""
    nx = shape[0]
    nrows = int(np.prod(shape[1:]))
    D = len(shape)
    row = (nx,) + (1,) * (D - 1)
    bc = (ZG,) + (P,) * (D - 1)
    E, Ec, ref, cref = run_variants(lat, gamma, tau, tau, row, bc, fields_row, steps, prec,
                                    ref_state=library_reference(prec, rho0))
    gpu, cgpu = run_gpu(lat, gamma, tau, tau, shape, bc, fields_full, steps, prec, rho0=rho0)
    for q in (gpu[0], gpu[2], *gpu[1]):
        assert rows_equal(q, nrows, nx)
    g0 = (gpu[0][:nx], gpu[1][:, :nx], gpu[2][:nx])
    tol = spread_tolerance(prec, E)
    report(f"{name} {'FP64' if prec == F64 else 'FP32'}", assert_parity(g0, ref, gamma, tol), E, tol)
    ctol = spread_tolerance(prec, Ec)
    scale = np.array([abs(cref[0])] * (1 + D) + [abs(cref[-1])])
    assert np.all(np.abs(cgpu / nrows - cref) / scale <= ctol), (cgpu / nrows, cref, ctol)


@pytest.mark.parametrize("prec", [F64, F32])
@pytest.mark.parametrize("steps", [180, 500])
def test_sod_tube_1000x4(steps, prec):
    """Classic Sod on 1000 x 4 (periodic y, zero-gradient x), gamma 1.4,
    tau_f = tau_g = 0.6 (the FP64 shock-tube workload).  The shock leaves
    through the open end near step 340 and the flow then amplifies
    round-off, so the bar is the variants' spread (tube_parity).  The
    density spans a factor 8, so the populations are stored whole
    (rho0 < 0; FP64's default): deviations from one reference state would
    be up to 7 times the populations on the low-density side."""
    tube_parity(f"classic Sod 1000x4, {steps} steps", ora.D2Q37, (1000, 4), li.sod_fields(1000, 4),
                li.sod_fields(1000, 1), 1.4, 0.6, steps, prec, rho0=-1.0)


@pytest.mark.parametrize("prec", [F64, F32])
def test_sod_tube_3d_1024x4x4(prec):
    """Classic Sod on the D3Q107 lattice, 1024 x 4 x 4, 100 steps (whole
    storage, as the 2D tube)."""
    tube_parity("classic Sod 3D 1024x4x4, 100 steps", ora.D3Q107, (1024, 4, 4), li.sod_fields(1024, 4, 4, D=3),
                li.sod_fields(1024, 1, 1, D=3), 1.4, 0.6, 100, prec, rho0=-1.0)


@pytest.mark.parametrize("prec", [F64, F32])
@pytest.mark.parametrize("steps", [180, 500])
def test_paper_shock_tube_2d(steps, prec):
    """The paper's own 2D case (Sec. V): D2Q37, 1000 x 16, delta = 3,
    tau = 2/3, rho 4|1, T 1|1.  In FP64 the variants stay within 5e-13 of
    the oracle, so the bar is the plain 1e-12."""
    L, R = (4.0, 0.0, 1.0), (1.0, 0.0, 1.0)
    tube_parity(f"paper tube 2D 1000x16, {steps} steps", ora.D2Q37, (1000, 16),
                li.sod_fields(1000, 16, left=L, right=R), li.sod_fields(1000, 1, left=L, right=R), 1.4, 2 / 3,
                steps, prec)


@pytest.mark.parametrize("prec", [F64, F32])
def test_periodic_fourier_box_512(prec):
    """The periodic-box recipe (8 random Fourier modes, u amplitude 0.02,
    1% density) at 512^2, gamma 1.4, tau_f 0.55, tau_g 0.7, 200 steps: a
    smooth, well-conditioned flow, held to the plain bars 1e-12 / 1e-5."""
    shape = (512, 512)
    fields = li.fourier_fields(shape, seed_u=1, seed_rho=2)
    ref, _ = run_oracle(ora.D2Q37, 1.4, 0.55, 0.7, shape, (P, P), fields, 200)
    gpu, _ = run_gpu(0, 1.4, 0.55, 0.7, shape, (P, P), fields, 200, prec)
    assert_parity(gpu, ref, 1.4, TOL["f64" if prec == F64 else "f32"])


@pytest.mark.parametrize("prec", [F64, F32])
def test_periodic_fourier_box_3d(prec):
    """The 3D periodic recipe (rho, u, T modes, k in [-4, 4]) at 48^3,
    gamma 1.3 (delta = 11/3, non-integer), tau 0.6, 40 steps."""
    shape = (48, 48, 48)
    fields = li.fourier_fields(shape, seed_u=3, seed_rho=4, seed_T=5)
    ref, _ = run_oracle(ora.D3Q107, 1.3, 0.6, 0.6, shape, (P, P, P), fields, 40)
    gpu, _ = run_gpu(1, 1.3, 0.6, 0.6, shape, (P, P, P), fields, 40, prec)
    assert_parity(gpu, ref, 1.3, TOL["f64" if prec == F64 else "f32"])


@pytest.mark.parametrize("lat,shape", [(0, (48, 40)), (1, (12, 10, 8))])
def test_conserved_totals_match_oracle_and_are_conserved(lat, shape):
    D = len(shape)
    fields = fields_for(shape, seed=77)
    _, c0 = run_oracle(lat, 1.4, 0.6, 0.6, shape, (P,) * D, fields, 0)
    ref, cref = run_oracle(lat, 1.4, 0.6, 0.6, shape, (P,) * D, fields, 25)
    gpu, cgpu = run_gpu(lat, 1.4, 0.6, 0.6, shape, (P,) * D, fields, 25, F64)
    scale = np.array([c0[0]] * (1 + D) + [c0[-1]])
    assert np.all(np.abs(cgpu - cref) / scale < 1e-13)
    assert np.all(np.abs(cgpu - c0) / scale < 1e-13)


@pytest.mark.parametrize("prec", [F64, F32])
def test_uniform_state_stays_uniform(prec):
    from paper_1608_06345_gb300 import lbm
    shape = (77, 6)
    N = 77 * 6
    fields = li.uniform_fields(N, 2, rho=1.2, u=[0.05, -0.02], T=0.95)
    s = lbm.Solver(0, 1.4, 0.7, 0.7, shape, bc=(ZG, P), prec=prec)
    s.init(*fields)
    s.step(30)
    rho, u, T = s.moments()
    for q in (rho, u[0], u[1], T):
        assert np.ptp(q) == 0.0
    tol = 1e-14 if prec == F64 else 2e-6
    assert abs(rho[0] - 1.2) < tol and abs(T[0] - 0.95) < tol


def test_nonfinite_input_is_reported():
    """A NaN in the initial fields propagates; the step's non-finite check
    sets the error word and the next sync point returns LBM_ENONFINITE."""
    from paper_1608_06345_gb300 import lbm
    rho, u, T = li.uniform_fields(64 * 4, 2)
    rho[70] = np.nan
    s = lbm.Solver(0, 1.4, 0.6, 0.6, (64, 4), prec=F32)
    s.init(rho, u, T)
    s.step(2)
    with pytest.raises(lbm.LbmError) as ei:
        s.moments()
    assert ei.value.code == lbm.LBM_ENONFINITE


@pytest.mark.parametrize("lat,shape,prec", [(0, (40, 6), F64), (0, (40, 6), 2), (1, (12, 5, 4), 3)])
def test_checkpoint_roundtrip(lat, shape, prec):
    from paper_1608_06345_gb300 import lbm
    fields = fields_for(shape, seed=5)
    a = lbm.Solver(lat, 1.4, 0.6, 0.7, shape, prec=prec)
    a.init(*fields)
    a.step(7)
    raw = np.zeros(lbm.lbm_raw_state_bytes(a.h), dtype=np.uint8)
    lbm.lbm_get_state(a.h, raw)
    a.step(5)
    ra = a.moments()
    b = lbm.Solver(lat, 1.4, 0.6, 0.7, shape, prec=prec)
    lbm.lbm_set_state(b.h, raw)
    b.step(5)
    rb = b.moments()
    for qa, qb in zip(ra, rb):
        assert np.array_equal(qa, qb)


@pytest.mark.parametrize("prec,dt", [(2, np.float16), (3, None)])
def test_raw_16bit_state_is_paired(prec, dt):
    """16-bit raw state: Q planes of N 4-byte pairs, g_i in the low half and
    h_i in the high half, each scaled by the reference equilibrium.  The
    density decoded on the host from the g halves equals the library's."""
    from paper_1608_06345_gb300 import lbm
    shape = (33, 5)
    N = shape[0] * shape[1]
    rho0, T0 = 0.9, 1.1
    s = lbm.Solver(0, 1.4, 0.6, 0.6, shape, prec=prec, rho0=rho0, T0=T0)
    s.init(*fields_for(shape, seed=8))
    s.step(3)
    raw = np.zeros(lbm.lbm_raw_state_bytes(s.h), dtype=np.uint8)
    lbm.lbm_get_state(s.h, raw)
    assert raw.size == 37 * N * 4
    halves = raw.view(np.uint16).reshape(37, N, 2)
    lo = halves[:, :, 0]
    if dt is not None:
        g = lo.view(dt).astype(np.float64)
    else:  # bfloat16: the upper 16 bits of an IEEE single
        g = (lo.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    gref = ora.feq(ora.D2Q37, rho0, [0.0, 0.0], T0)
    rho_host = (gref[:, None] * (1.0 + g)).sum(axis=0)
    rho, _, _ = s.moments()
    np.testing.assert_allclose(rho_host, rho, rtol=1e-6, atol=0)


@pytest.mark.parametrize("lat,shape,prec", [(0, (150, 6), F64), (1, (40, 5, 4), F32)])
def test_graph_replay_equals_plain_launches(lat, shape, prec):
    """lbm_step replays captured graphs for long runs; the result is bitwise
    that of one launch per step, also when a run starts on the odd buffer."""
    from paper_1608_06345_gb300 import lbm
    D = len(shape)
    fields = fields_for(shape, seed=23)
    out = []
    for gsteps in (0, 8):
        s = lbm.Solver(lat, 1.4, 0.6, 0.7, shape, prec=prec)
        lbm.lbm_set_graph_steps(s.h, gsteps)
        s.init(*fields)
        s.step(1)      # odd parity before the long run
        s.step(37)     # >= 2 graphs + remainder
        s.step(16)
        assert lbm.lbm_steps_done(s.h) == 54
        out.append(s.moments())
        s.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)
