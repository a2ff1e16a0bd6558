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
BAR = {0: 1e-12, 1: 1e-5}


def perturbed(fields, unit, seed=1, ulps=4):
    """Initial fields with rho and T multiplied by 1 + ulps*unit*U[-1, 1]."""
    rng = np.random.default_rng(seed)
    rho, u, T = fields
    return (rho * (1 + ulps * unit * rng.uniform(-1, 1, rho.shape)), u,
            T * (1 + ulps * unit * rng.uniform(-1, 1, T.shape)))


def run_variants(lattice, gamma, tau_f, tau_g, shape, bc, fields, steps, prec, ref_state=(1.0, 1.0), ref=None):
    """Distances of the oracle's rounding variants from the oracle on one
    case: E = max over the variants of precision `prec` (oracle.VARIANTS_F64
    for FP64, VARIANTS_F32 for the FP32-compute precisions) of the parity
    norm between the variant's rho, u, T and the oracle's, and Ec = the same
    for the grid totals (mass and momentum relative to the mass, energy
    relative to the energy).  The deviation variants (bit 8) store their
    populations as deviations from the equilibrium of ref_state, the
    reference state (rho0, T0) of the library instance under test.  E
    measures how far a correct evaluation of the same arithmetic in that
    precision lands from the oracle on this flow.  Returns (E, Ec, oracle
    result, oracle totals)."""
    if ref is None:
        ref = run_oracle(lattice, gamma, tau_f, tau_g, shape, bc, fields, steps)
    out, cref = ref
    scale = np.array([abs(cref[0])] * (len(cref) - 1) + [abs(cref[-1])])
    E = Ec = 0.0
    for v in (ora.VARIANTS_F64 if prec == 0 else ora.VARIANTS_F32):
        s = ora.Oracle(lattice, gamma, tau_f, tau_g, shape, bc=bc, variant=v)
        if v & 8:
            s.set_reference(*ref_state)
        s.init(*fields)
        s.step(steps)
        E = max(E, max(parity_errors(s.moments(), out, gamma).values()))
        Ec = max(Ec, float(np.max(np.abs(s.conserved() - cref) / scale)))
        s.close()
    return E, Ec, out, cref


def library_reference(prec, rho0=0.0, T0=0.0):
    """The reference state (rho0, T0) a library instance of precision prec
    stores its populations against, for the rho0, T0 it was created with
    (include/lbm.h): rho0 > 0 as given, rho0 < 0 whole storage (rho0 = 0),
    otherwise whole storage for FP64 and rho0 = 1 for FP32; T0 <= 0 means 1.
    The oracle's deviation variants take the same state (rho0 = 0 stores
    whole: they then round as the oracle does)."""
    if rho0 > 0:
        r = rho0
    elif rho0 < 0:
        r = 0.0
    else:
        r = 0.0 if prec == 0 else 1.0
    return r, (T0 if T0 > 0 else 1.0)


def spread_tolerance(prec, E):
    """Tolerance of a case whose variant distance is E (run_variants):
    max(bar, 2 E).  The library is one more evaluation of the same
    arithmetic.  It differs from the oracle in more respects than any one
    variant (all of the variants' changes at once, plus its regrouped
    equilibrium and its temperature formed as a deviation), so it is
    allowed twice the largest distance at which a variant lands.  Never
    below the precision's bar (1e-12 FP64, 1e-5 FP32)."""
    return max(BAR[prec], 2.0 * E)


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


def report(name, errs, E, tol):
    """One line per conditioned case: the library's parity error beside the
    variants' distance E and the tolerance (shown with pytest -s)."""
    print(f"PARITY {name}: library {max(errs.values()):.3e}  variants {E:.3e}  tolerance {tol:.3e}")

