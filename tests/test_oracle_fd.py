"""Pins of the oracle's finite-difference variant (Sec. III: forward Euler in
time, third-order upwind convection along each axis, BGK relaxation with the
cell's own moments), with lambda = dt/dx:

- the upwind difference is exact on cubic profiles (its defining order),
  along x, y and z, for both signs of the velocity component;
- the grid totals are conserved on a periodic box (the differences telescope
  and the collision conserves);
- a uniform state stays uniform;
- a small standing wave oscillates at the adiabatic sound speed sqrt(gamma T).
"""
import numpy as np
import pytest

import lbm_inputs as li
from oracle import oracle as ora

LAM = 0.05


def cubic(s):
    return 1e-6 * (s ** 3 - 3.0 * s ** 2 + 2.0 * s) + 1e-3


def dcubic(s):
    return 1e-6 * (3.0 * s ** 2 - 6.0 * s + 2.0)


@pytest.mark.parametrize("lat,shape,axis", [(ora.D2Q37, (40, 3), 0), (ora.D2Q37, (3, 40), 1),
                                            (ora.D3Q107, (3, 3, 30), 2)])
def test_upwind_difference_is_exact_on_cubics(lat, shape, axis):
    """With relaxation switched off (tau = 1e30) one step changes each
    population by -lambda xi_a q'(s) exactly where the stencil stays inside
    the grid (zero-gradient ends along the profile axis)."""
    D = len(shape)
    N = int(np.prod(shape))
    bc = [ora.PERIODIC] * 3
    bc[axis] = ora.ZERO_GRADIENT
    s = ora.Oracle(lat, 1.4, 1e30, 1e30, shape, bc=bc)
    s.init(*li.uniform_fields(N, D))
    idx = np.indices(tuple(reversed(shape))).reshape(len(shape), -1)[::-1]  # x, y, (z) per cell
    pos = idx[axis].astype(float)
    g0 = np.tile(cubic(pos), (s.Q, 1))
    h0 = 0.7 * g0
    s.set_pops(g0, h0)
    s.step_fd(1, LAM)
    g1, h1 = s.get_pops()
    c, w, r = ora.lattice_info(lat)
    n = shape[axis]
    inner = (pos >= 2) & (pos <= n - 3)
    for i in range(s.Q):
        expect = -LAM * r * c[i, axis] * dcubic(pos)
        np.testing.assert_allclose((g1[i] - g0[i])[inner], expect[inner], rtol=0, atol=1e-17)
        np.testing.assert_allclose((h1[i] - h0[i])[inner], 0.7 * expect[inner], rtol=0, atol=1e-17)


@pytest.mark.parametrize("lat,shape,steps", [(ora.D2Q37, (24, 20), 300), (ora.D3Q107, (10, 8, 6), 30)])
def test_fd_conserves_on_a_periodic_box(lat, shape, steps):
    D = len(shape)
    N = int(np.prod(shape))
    s = ora.Oracle(lat, 1.4, 0.8, 0.8, shape)
    s.init(*li.random_fields(N, D, seed=3, u_amp=0.02, rho_amp=0.02, T_amp=0.02))
    c0 = s.conserved()
    s.step_fd(steps, LAM)
    c1 = s.conserved()
    scale = np.array([c0[0]] * (1 + D) + [c0[-1]])
    assert np.all(np.abs(c1 - c0) / scale < 5e-13), (c1 - c0) / scale


def test_fd_uniform_state_stays_uniform():
    fields = li.uniform_fields(9 * 5, 2, rho=1.1, u=[0.05, -0.02], T=0.95)
    s = ora.Oracle(ora.D2Q37, 1.4, 0.7, 0.7, (9, 5), bc=(ora.ZERO_GRADIENT, ora.PERIODIC))
    s.init(*fields)
    s.step_fd(40, LAM)
    rho, u, T = s.moments()
    for q in (rho, u[0], u[1], T):
        assert np.ptp(q) == 0.0
    assert abs(rho[0] - 1.1) < 1e-14 and abs(T[0] - 0.95) < 1e-14


def test_fd_sound_speed():
    """Physical time per step is lambda (dx = 1), so the velocity mode of a
    standing wave of wavelength 64 cells crosses zero every pi/(k c lambda)
    steps with c = sqrt(gamma T)."""
    nx, gamma = 64, 1.4
    rho, u, T = li.acoustic_wave(nx, D=2, amp=1e-4, gamma=gamma)
    s = ora.Oracle(ora.D2Q37, gamma, 0.8, 0.8, (nx, 1))
    s.init(rho, u, T)
    basis = np.cos(2 * np.pi * np.arange(nx) / nx)
    k = 2 * np.pi / nx
    steps = int(1.3 * np.pi / (k * np.sqrt(gamma) * LAM) * 2)
    b = []
    for _ in range(steps):
        s.step_fd(1, LAM)
        b.append(np.dot(s.moments()[1][0], basis))
    b = np.array(b)
    z = [j + b[j - 1] / (b[j - 1] - b[j]) for j in range(1, len(b)) if b[j - 1] * b[j] < 0]
    assert len(z) >= 2
    omega = np.pi / np.mean(np.diff(z)) / LAM
    assert abs(omega / (k * np.sqrt(gamma)) - 1.0) < 5e-3
