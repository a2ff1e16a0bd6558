"""Helpers of the parity tests: run the same seeded case through the GPU
library (C ABI via the binding) and through the FP64 oracle, and compare.

Parity norm per field: max over cells of |q_gpu - q_oracle| divided by
max |q_oracle| (rho, T); for each velocity component by
max(max |u_oracle|, 1e-3 sqrt(gamma T_ref)) so that regions at rest do not
turn round-off into a large relative error."""
from __future__ import annotations

import numpy as np

from oracle import oracle as ora

# tolerances per precision (relative, parity norm above)
TOL = {"f64": 1e-12, "f32": 1e-5}
# unit roundoff of the storage / arithmetic of each precision code
UNIT_ROUNDOFF = {0: 2.0 ** -53, 1: 2.0 ** -24, 2: 2.0 ** -11, 3: 2.0 ** -8}
BAR = {0: 1e-12, 1: 1e-5}


def perturbed(fields, unit, seed=1, ulps=4):
    """Initial fields with rho and T multiplied by 1 + ulps*unit*U[-1, 1]."""
    rng = np.random.default_rng(seed)
    rho, u, T = fields
    return (rho * (1 + ulps * unit * rng.uniform(-1, 1, rho.shape)), u,
            T * (1 + ulps * unit * rng.uniform(-1, 1, T.shape)))


def sensitivity(lattice, gamma, tau_f, tau_g, shape, bc, fields, steps, prec, ref=None, seed=1):
    """kappa: how far the oracle's own result moves (parity norm) when every
    stored population is rounded, at every step, by a random relative error
    of the unit roundoff u of precision `prec` (a model of storage rounding:
    amplitude u (|g| + |g - g_ref|), g_ref the equilibrium at rho = 1, u = 0,
    T = 1 that the library's deviation storage is taken from).  It measures
    the conditioning of the case."""
    if ref is None:
        ref, _ = run_oracle(lattice, gamma, tau_f, tau_g, shape, bc, fields, steps)
    unit = UNIT_ROUNDOFF[prec]
    rng = np.random.default_rng(seed)
    D = len(shape)
    gref = ora.feq(lattice, 1.0, np.zeros(D), 1.0)[:, None]
    href = 0.5 * ora.delta_from_gamma(D, gamma) * gref
    s = ora.Oracle(lattice, gamma, tau_f, tau_g, shape, bc=bc)
    s.init(*fields)
    for _ in range(steps):
        s.step(1)
        g, h = s.get_pops()
        g = g + unit * (np.abs(g) + np.abs(g - gref)) * rng.uniform(-1, 1, g.shape)
        h = h + unit * (np.abs(h) + np.abs(h - href)) * rng.uniform(-1, 1, h.shape)
        s.set_pops(g, h)
    out = s.moments()
    s.close()
    return max(parity_errors(out, ref, gamma).values())


def conditioned_tolerance(prec, kappa, steps):
    """Tolerance of an ill-conditioned case (shock tubes).  An independent
    implementation rounds differently at every step and its differences need
    not be random, so its distance from the oracle is allowed 5 sqrt(n) times
    the noise-model sensitivity kappa (measured GPU/kappa ratios on the shock
    tubes stay below 2 sqrt(n)).  Never below the precision's bar."""
    return max(BAR[prec], 5.0 * np.sqrt(steps) * kappa)


def run_oracle(lattice, gamma, tau_f, tau_g, shape, bc, fields, steps):
    s = ora.Oracle(lattice, gamma, tau_f, tau_g, shape, bc=bc)
    s.init(*fields)
    s.step(steps)
    out = s.moments()
    cons = s.conserved()
    s.close()
    return out, cons


def run_gpu(lattice, gamma, tau_f, tau_g, shape, bc, fields, steps, prec, rho0=0.0, T0=0.0):
    from paper_1608_06345_gb300 import lbm
    s = lbm.Solver(lattice, gamma, tau_f, tau_g, shape, bc=bc, prec=prec, rho0=rho0, T0=T0)
    s.init(*fields)
    s.step(steps)
    out = s.moments()
    cons = s.conserved()
    s.close()
    return out, cons


def parity_errors(gpu, ref, gamma, T_ref=1.0):
    rho_g, u_g, T_g = gpu
    rho_o, u_o, T_o = ref
    e = {"rho": np.max(np.abs(rho_g - rho_o)) / np.max(np.abs(rho_o)),
         "T": np.max(np.abs(T_g - T_o)) / np.max(np.abs(T_o))}
    floor = 1e-3 * np.sqrt(gamma * T_ref)
    for a in range(u_o.shape[0]):
        e[f"u{a}"] = np.max(np.abs(u_g[a] - u_o[a])) / max(np.max(np.abs(u_o[a])), floor)
    return e


def assert_parity(gpu, ref, gamma, tol, T_ref=1.0):
    e = parity_errors(gpu, ref, gamma, T_ref)
    bad = {k: v for k, v in e.items() if not (v <= tol)}
    assert not bad, f"parity errors above {tol}: {e}"
    return e
