"""Seeded synthetic inputs shared by the oracle, the GPU tests and the bench.

This module only synthesises macroscopic initial fields (density, velocity,
temperature) and request streams; it holds none of the lattice Boltzmann
arithmetic, so the CPU oracle and the GPU library stay independent.

Layouts: scalar fields are flat arrays of N = nx*ny*nz cells, cell index
x + nx*(y + ny*z); the velocity is component-major, shape (D, N).
"""
from __future__ import annotations

import numpy as np


def sod_fields(nx, ny=1, nz=None, D=2, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.8)):
    """Shock-tube initial state: (rho, u_x, T) = left for cells x < nx/2 and
    right for x >= nx/2, uniform along y and z, u_y = u_z = 0.

    The defaults are the classic Sod states rho 1|0.125, p 1|0.1 (T = p/rho).
    The paper's own case (Sec. V) is left=(4, 0, 1), right=(1, 0, 1)."""
    if nz is None:
        nz = 1
    N = nx * ny * nz
    xs = np.arange(nx)
    lmask = np.broadcast_to((xs < nx // 2)[None, None, :], (nz, ny, nx)).reshape(N)
    rho = np.where(lmask, left[0], right[0]).astype(np.float64)
    u = np.zeros((D, N))
    u[0] = np.where(lmask, left[1], right[1])
    T = np.where(lmask, left[2], right[2]).astype(np.float64)
    return rho, u, T


def uniform_fields(N, D, rho=1.0, u=None, T=1.0):
    uu = np.zeros((D, N))
    if u is not None:
        for a in range(D):
            uu[a] = u[a]
    return np.full(N, float(rho)), uu, np.full(N, float(T))


def _modes(rng, n_modes, D, kmax):
    ks = []
    while len(ks) < n_modes:
        k = rng.integers(-kmax, kmax + 1, size=D)
        if np.any(k != 0):
            ks.append(k)
    return np.array(ks)


def _phase_field(shape, k, phi):
    """cos(2 pi k.x / n + phi) on the grid; shape = (nx, ny[, nz])."""
    D = len(shape)
    out = None
    # separable evaluation: cos(a + b) = cos a cos b - sin a sin b, built up axis by axis
    arg = [2.0 * np.pi * k[a] * np.arange(shape[a]) / shape[a] for a in range(D)]
    c = np.cos(arg[0] + phi)
    s = np.sin(arg[0] + phi)
    c = c[None, :]
    s = s[None, :]
    # y axis
    cy, sy = np.cos(arg[1])[:, None], np.sin(arg[1])[:, None]
    c2 = c * cy - s * sy
    if D == 2:
        out = c2
        return out.reshape(-1)
    s2 = s * cy + c * sy
    cz, sz = np.cos(arg[2])[:, None, None], np.sin(arg[2])[:, None, None]
    out = c2[None] * cz - s2[None] * sz
    return out.reshape(-1)


def fourier_fields(shape, seed_u, seed_rho, seed_T=None, n_modes=8, amp_u=0.02,
                   amp_rho=0.01, amp_T=0.01, kmax=None):
    """Periodic-box initial state: a sum of seeded random Fourier modes.

    u   = sum_m amp_u * e_m * cos(2 pi k_m.x / n + phi_m)   (e_m random unit vectors)
    rho = 1 + sum_m (amp_rho / n_modes) * cos(2 pi k'_m.x / n + phi'_m)
    T   = 1 (+ the same recipe with amp_T when seed_T is given)
    k components are integers uniform in [-kmax, kmax], not all zero
    (kmax = 8 in 2D, 4 in 3D); phases uniform in [0, 2 pi).
    shape = (nx, ny) or (nx, ny, nz)."""
    D = len(shape)
    if kmax is None:
        kmax = 8 if D == 2 else 4
    N = int(np.prod(shape))
    rng = np.random.default_rng(seed_u)
    ks = _modes(rng, n_modes, D, kmax)
    e = rng.normal(size=(n_modes, D))
    e /= np.linalg.norm(e, axis=1, keepdims=True)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    u = np.zeros((D, N))
    for m in range(n_modes):
        f = _phase_field(shape, ks[m], ph[m])
        for a in range(D):
            u[a] += amp_u * e[m, a] * f
    rng = np.random.default_rng(seed_rho)
    ks = _modes(rng, n_modes, D, kmax)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    rho = np.ones(N)
    for m in range(n_modes):
        rho += (amp_rho / n_modes) * _phase_field(shape, ks[m], ph[m])
    T = np.ones(N)
    if seed_T is not None:
        rng = np.random.default_rng(seed_T)
        ks = _modes(rng, n_modes, D, kmax)
        ph = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
        for m in range(n_modes):
            T += (amp_T / n_modes) * _phase_field(shape, ks[m], ph[m])
    return rho, u, T


def acoustic_wave(nx, D=2, amp=1e-4, gamma=1.4):
    """Isentropic standing wave on an nx x 1 (x 1) periodic box:
    rho = 1 + amp sin(2 pi x/nx), T = 1 + (gamma - 1) amp sin(2 pi x/nx), u = 0."""
    x = np.arange(nx)
    s = np.sin(2.0 * np.pi * x / nx)
    rho = 1.0 + amp * s
    T = 1.0 + (gamma - 1.0) * amp * s
    return rho, np.zeros((D, nx)), T


def random_fields(N, D, seed, u_amp=0.05, rho_amp=0.05, T_amp=0.05):
    """Cell-wise i.i.d. perturbations (rough fields that exercise every
    direction of the stencil): rho, T = 1 + amp U[-1, 1], u_a = u_amp U[-1, 1]."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rho_amp * rng.uniform(-1, 1, N)
    u = u_amp * rng.uniform(-1, 1, (D, N))
    T = 1.0 + T_amp * rng.uniform(-1, 1, N)
    return rho, u, T


def serving_requests(n=512, seed=6, nx_range=(256, 16384), ny=4, gamma_range=(1.1, 1.67),
                     ratio_range=(1.0, 10.0), tau_range=(0.52, 1.0), steps_range=(200, 2000)):
    """Parameters of a stream of shock-tube solves (one dict per request):
    Nx log-uniform, gamma uniform, rho_L/rho_R and p_L/p_R log-uniform
    (normalised geometrically: rho_L = sqrt(R), rho_R = 1/sqrt(R)), tau_f = tau_g
    uniform, steps uniform integer."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nx = int(round(np.exp(rng.uniform(np.log(nx_range[0]), np.log(nx_range[1])))))
        gamma = float(rng.uniform(*gamma_range))
        rr = float(np.exp(rng.uniform(np.log(ratio_range[0]), np.log(ratio_range[1]))))
        rp = float(np.exp(rng.uniform(np.log(ratio_range[0]), np.log(ratio_range[1]))))
        tau = float(rng.uniform(*tau_range))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        rl, rR = np.sqrt(rr), 1.0 / np.sqrt(rr)
        pl, pR = np.sqrt(rp), 1.0 / np.sqrt(rp)
        out.append(dict(id=k, nx=nx, ny=ny, gamma=gamma, tau=tau, steps=steps,
                        left=(rl, 0.0, pl / rl), right=(rR, 0.0, pR / rR)))
    return out


def poisson_arrivals(n, rate, seed=7):
    """Arrival times (seconds) of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
