"""Pins of the oracle's time stepping against properties the scheme must have:
collision invariants of the BGK operator with the moment-matching equilibrium
(Eq. (13)-(18)), translation/mirror symmetry, tau = 1 reset, delta = 0, and
the adiabatic sound speed sqrt(gamma T) of the Euler limit."""
import numpy as np
import pytest

import lbm_inputs as li
from oracle import oracle as ora


def run(lat, gamma, tau_f, tau_g, shape, fields, steps, bc=(ora.PERIODIC,) * 3):
    s = ora.Oracle(lat, gamma, tau_f, tau_g, shape, bc=bc)
    s.init(*fields)
    s.step(steps)
    return s


@pytest.mark.parametrize("lat,shape,steps", [(ora.D2Q37, (24, 20), 300), (ora.D3Q107, (10, 8, 6), 40)])
def test_conservation_periodic(lat, shape, steps):
    """Mass, momentum and total energy are collision invariants when
    tau_f = tau_g; with periodic streaming the grid totals stay put to
    round-off."""
    D = len(shape)
    N = int(np.prod(shape))
    fields = li.random_fields(N, D, seed=21)
    s = ora.Oracle(lat, 1.4, 0.6, 0.6, shape)
    s.init(*fields)
    c0 = s.conserved()
    s.step(steps)
    c1 = s.conserved()
    scale = np.array([c0[0]] + [c0[0]] * D + [c0[-1]])
    assert np.all(np.abs(c1 - c0) / scale < 1e-13), (c1 - c0) / scale


def test_unequal_taus_conserve_mass_and_momentum_only():
    """With tau_f != tau_g the energy is not a collision invariant (the paper
    has one tau); mass and momentum still are."""
    shape = (24, 20)
    fields = li.random_fields(480, 2, seed=22, u_amp=0.2, T_amp=0.2)
    s = ora.Oracle(ora.D2Q37, 1.4, 0.55, 0.7, shape)
    s.init(*fields)
    c0 = s.conserved()
    s.step(50)
    c1 = s.conserved()
    assert abs(c1[0] - c0[0]) / c0[0] < 1e-13
    assert np.all(np.abs(c1[1:3] - c0[1:3]) / c0[0] < 1e-13)
    assert abs(c1[3] - c0[3]) / c0[3] > 1e-9


@pytest.mark.parametrize("bcx", [ora.PERIODIC, ora.ZERO_GRADIENT])
@pytest.mark.parametrize("lat,shape", [(ora.D2Q37, (9, 5)), (ora.D3Q107, (5, 4, 3))])
def test_uniform_state_stays_uniform(lat, shape, bcx):
    D = len(shape)
    N = int(np.prod(shape))
    u = [0.1, -0.05, 0.02][:D]
    fields = li.uniform_fields(N, D, rho=1.3, u=u, T=0.9)
    steps = 25
    s = run(lat, 1.3, 0.7, 0.7, shape, fields, steps, bc=(bcx, ora.PERIODIC, ora.PERIODIC))
    rho, uu, T = s.moments()
    for q in (rho, uu[0], uu[-1], T):
        assert np.ptp(q) == 0.0  # bitwise uniform
    # a uniform state repeats the same arithmetic every step, so its values
    # drift linearly by at most the round-off of the Q-term moment sums per
    # step: steps * Q * 2^-53 relative (3e-13 for D3Q107 over 25 steps); a
    # dropped or wrong term moves them by O(1)
    Q = 37 if lat == ora.D2Q37 else 107
    bound = steps * Q * 2.0 ** -53
    assert abs(rho[0] - 1.3) / 1.3 < bound and abs(T[0] - 0.9) / 0.9 < bound
    assert np.all(np.abs(uu[:, 0] - np.array(u)) < bound)


@pytest.mark.parametrize("lat,shape", [(ora.D2Q37, (12, 7)), (ora.D3Q107, (6, 5, 4))])
def test_tau_one_resets_to_equilibrium(lat, shape):
    """With tau = 1 the post-collision state is the equilibrium of the
    pulled state's moments, and those moments are the stored moments."""
    D = len(shape)
    N = int(np.prod(shape))
    s = ora.Oracle(lat, 1.4, 1.0, 1.0, shape)
    s.init(*li.random_fields(N, D, seed=3))
    # push the state off equilibrium, then take one tau = 1 step
    g, h = s.get_pops()
    rng = np.random.default_rng(4)
    s.set_pops(g * (1 + 0.01 * rng.standard_normal(g.shape)), h * (1 + 0.01 * rng.standard_normal(h.shape)))
    s.step(1)
    g, h = s.get_pops()
    rho, u, T = s.moments()
    for cell in range(0, N, 5):
        F = ora.feq(lat, rho[cell], u[:, cell], T[cell])
        np.testing.assert_allclose(g[:, cell], F, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(h[:, cell], 0.5 * s.delta * T[cell] * F, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("lat,D,gamma", [(ora.D2Q37, 2, 2.0), (ora.D3Q107, 3, 5.0 / 3.0)])
def test_delta_zero_has_no_internal_energy(lat, D, gamma):
    """gamma = (D+2)/D gives delta = 0: h is zero for all time (up to the
    rounding of delta itself, 2/(gamma-1) - D ~ 1e-16 for gamma = 5/3)."""
    shape = (10, 6) if D == 2 else (5, 4, 3)
    N = int(np.prod(shape))
    s = run(lat, gamma, 0.6, 0.6, shape, li.random_fields(N, D, seed=8), 10)
    assert abs(s.delta) < 1e-14
    g, h = s.get_pops()
    assert np.max(np.abs(h)) < 1e-14 * np.max(np.abs(g))


def test_mirror_symmetry():
    """A state symmetric under x -> nx-1-x (u_x antisymmetric) stays so."""
    nx, ny = 16, 6
    rng = np.random.default_rng(9)
    half = rng.uniform(-1, 1, (ny, nx // 2))
    sym = np.concatenate([half, half[:, ::-1]], axis=1).reshape(-1)
    asym = np.concatenate([half, -half[:, ::-1]], axis=1).reshape(-1)
    rho = 1 + 0.05 * sym
    T = 1 + 0.03 * sym
    u = np.stack([0.05 * asym, 0.02 * sym])
    s = run(ora.D2Q37, 1.4, 0.6, 0.6, (nx, ny), (rho, u, T), 60, bc=(ora.ZERO_GRADIENT, ora.PERIODIC))
    R, U, TT = s.moments()
    R, TT, U0, U1 = (q.reshape(ny, nx) for q in (R, TT, U[0], U[1]))
    assert np.max(np.abs(R - R[:, ::-1])) < 1e-13
    assert np.max(np.abs(TT - TT[:, ::-1])) < 1e-13
    assert np.max(np.abs(U0 + U0[:, ::-1])) < 1e-13
    assert np.max(np.abs(U1 - U1[:, ::-1])) < 1e-13


def test_translation_invariance():
    """Shifting the initial state by whole cells on a periodic box shifts the
    result by the same amount, exactly."""
    nx, ny = 11, 7
    rho, u, T = li.random_fields(nx * ny, 2, seed=12)
    a = run(ora.D2Q37, 1.4, 0.6, 0.7, (nx, ny), (rho, u, T), 5).moments()
    sh = lambda q: np.roll(q.reshape(-1, ny, nx), (2, 3), axis=(1, 2)).reshape(q.shape)
    b = run(ora.D2Q37, 1.4, 0.6, 0.7, (nx, ny), (sh(rho), sh(u), sh(T)), 5).moments()
    for qa, qb in zip(a, b):
        np.testing.assert_allclose(sh(qa), qb, rtol=0, atol=1e-15)


def velocity_projection_zero_crossings(lat, D, gamma, nx=256, steps=320, tau=0.6):
    """Steps at which the standing wave's velocity mode changes sign."""
    rho, u, T = li.acoustic_wave(nx, D=D, amp=1e-4, gamma=gamma)
    shape = (nx, 1) if D == 2 else (nx, 1, 1)
    s = ora.Oracle(lat, gamma, tau, tau, shape)
    s.init(rho, u, T)
    x = np.arange(nx)
    basis = np.cos(2 * np.pi * x / nx)
    b = []
    for _ in range(steps):
        s.step(1)
        _, uu, _ = s.moments()
        b.append(np.dot(uu[0], basis))
    b = np.array(b)
    z = []
    for k in range(1, len(b)):
        if b[k - 1] * b[k] < 0:
            z.append(k - 1 + b[k - 1] / (b[k - 1] - b[k]))
    return np.array(z) + 1.0  # b[k] is after k+1 steps


@pytest.mark.parametrize("lat,D,gamma", [(ora.D2Q37, 2, 1.4), (ora.D2Q37, 2, 1.3), (ora.D2Q37, 2, 1.1),
                                         (ora.D3Q107, 3, 5.0 / 3.0), (ora.D3Q107, 3, 1.4)])
def test_acoustic_speed(lat, D, gamma):
    """A small standing wave oscillates at omega = k sqrt(gamma T) / r per
    step (lattice units: c_i = xi_i dt/dx with dt = dx/r)."""
    _, _, r = ora.lattice_info(lat)
    nx = 256
    z = velocity_projection_zero_crossings(lat, D, gamma, nx=nx)
    assert len(z) >= 2
    half_period = np.mean(np.diff(z))
    omega = np.pi / half_period
    expected = 2 * np.pi / nx * np.sqrt(gamma * 1.0) / r
    assert abs(omega / expected - 1.0) < 5e-3, (omega, expected)


@pytest.mark.parametrize("lat,D,tau", [(ora.D2Q37, 2, 0.8), (ora.D2Q37, 2, 0.6), (ora.D3Q107, 3, 0.7)])
def test_shear_wave_viscous_decay(lat, D, tau):
    """A small shear wave u_y = A sin(k x) decays as exp(-nu k^2 n) with the
    BGK kinematic viscosity nu = (tau - 1/2) T dt, i.e. (tau - 1/2) T / r^2
    cells^2 per step in lattice units (Chapman-Enskog limit of Eq. (16))."""
    _, _, r = ora.lattice_info(lat)
    nx, steps, A = 64, 200, 1e-4
    x = np.arange(nx)
    rho = np.ones(nx)
    T = np.ones(nx)
    u = np.zeros((D, nx))
    u[1] = A * np.sin(2 * np.pi * x / nx)
    shape = (nx, 1) if D == 2 else (nx, 1, 1)
    s = ora.Oracle(lat, 1.4, tau, tau, shape)
    s.init(rho, u, T)
    s.step(steps)
    _, uu, _ = s.moments()
    amp = 2.0 / nx * np.dot(uu[1], np.sin(2 * np.pi * x / nx))
    nu = (tau - 0.5) * 1.0 / r ** 2
    expected = A * np.exp(-nu * (2 * np.pi / nx) ** 2 * steps)
    assert abs(amp / expected - 1.0) < 5e-3, (amp / A, expected / A)


@pytest.mark.parametrize("lat,shape", [(ora.D2Q37, (300, 7)), (ora.D3Q107, (64, 3, 2))])
def test_totals_are_the_exact_sums(lat, shape):
    """ora_conserved's compensated sums equal the exactly rounded sums
    (math.fsum) of mass, momentum and energy over every population of the
    grid, Eq. (14), to a few ulps."""
    import math
    D = len(shape)
    N = int(np.prod(shape))
    s = run(lat, 1.4, 0.6, 0.7, shape, li.random_fields(N, D, seed=21), 7)
    c = s.conserved()
    g, h = s.get_pops()
    cv, w, r = ora.lattice_info(lat)
    xi = r * cv
    exact = [math.fsum(g.ravel())] + [math.fsum((xi[:, a:a + 1] * g).ravel()) for a in range(D)] + \
            [math.fsum((0.5 * (xi ** 2).sum(1)[:, None] * g + h).ravel())]
    scale = np.array([abs(exact[0])] * (1 + D) + [abs(exact[-1])])
    assert np.all(np.abs(c - np.array(exact)) <= 4 * 2.0 ** -53 * scale), (c, exact)
