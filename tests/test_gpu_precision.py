"""Storage precision against the FP64 oracle (L1 and L-infinity per field):
FP32, FP16 and BF16 storage on the smooth periodic recipe (1024^2, 200
steps) and on the paper's shock tube at Nx = 8192 (rho 4|1, T 1|1,
tau = 2/3, gamma = 1.4, t = 0.1504), plus the exact-solution L1 of the GPU
FP64 Sod tube of 1000 x 4 at 500 steps.  The classic Sod tube at Nx = 8192
is not measured: the scheme itself goes non-finite there (the oracle does
too), see test_classic_sod_at_8192_is_unstable_in_the_oracle.

Run with -s to print the table."""
import numpy as np
import pytest

import lbm_inputs as li
from oracle import oracle as ora
from oracle import riemann
from tests.parity import parity_errors, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

NAMES = {1: "FP32", 2: "FP16", 3: "BF16"}
# stated bounds: (L-inf, L1) relative
SMOOTH = {1: (1e-5, 1e-5), 2: (1e-3, 5e-4), 3: (1e-2, 5e-3)}
# on the tube, 16-bit storage moves the shock by a fraction of a cell: the
# L-inf error is then the jump itself (order 1) and only L1 is bounded
TUBE = {1: (5e-3, 1e-4), 2: (None, 2e-3), 3: (None, 2e-2)}


def l1_rel(g, o):
    out = {}
    pairs = [("rho", g[0], o[0]), ("T", g[2], o[2])] + [(f"u{a}", g[1][a], o[1][a]) for a in range(o[1].shape[0])]
    for k, a, b in pairs:
        den = np.mean(np.abs(b))
        if den > 1e-3:
            out[k] = float(np.mean(np.abs(a - b)) / den)
    return out


def test_precision_on_the_smooth_recipe_1024():
    shape = (1024, 1024)
    fields = li.fourier_fields(shape, seed_u=1, seed_rho=2)
    ref, _ = run_oracle(ora.D2Q37, 1.4, 0.55, 0.7, shape, (0, 0), fields, 200)
    for prec in (1, 2, 3):
        gpu, _ = run_gpu(0, 1.4, 0.55, 0.7, shape, (0, 0), fields, 200, prec)
        linf = max(parity_errors(gpu, ref, 1.4).values())
        l1 = max(l1_rel(gpu, ref).values())
        print(f"smooth 1024^2 x 200 {NAMES[prec]}: Linf {linf:.3e}  L1 {l1:.3e}")
        assert linf <= SMOOTH[prec][0] and l1 <= SMOOTH[prec][1]


def test_precision_on_the_paper_tube_8192():
    nx = 8192
    _, _, r = ora.lattice_info(ora.D2Q37)
    steps = int(round(0.1504 * nx * r))
    L, R = (4.0, 0.0, 1.0), (1.0, 0.0, 1.0)
    ref, _ = run_oracle(ora.D2Q37, 1.4, 2 / 3, 2 / 3, (nx, 1), (1, 0), li.sod_fields(nx, 1, left=L, right=R), steps)
    rho0 = 2.5
    T0 = 1.0
    res = {}
    for prec in (1, 2, 3):
        gpu, _ = run_gpu(0, 1.4, 2 / 3, 2 / 3, (nx, 4), (1, 0), li.sod_fields(nx, 4, left=L, right=R), steps, prec,
                         rho0=rho0, T0=T0)
        g = (gpu[0][:nx], gpu[1][:, :nx], gpu[2][:nx])
        res[prec] = (max(parity_errors(g, ref, 1.4).values()), max(l1_rel(g, ref).values()))
        print(f"paper tube 8192 x {steps} {NAMES[prec]}: Linf {res[prec][0]:.3e}  L1 {res[prec][1]:.3e}")
    for prec, (linf, l1) in res.items():
        assert (TUBE[prec][0] is None or linf <= TUBE[prec][0]) and l1 <= TUBE[prec][1], (NAMES[prec], linf, l1)


def test_sod_1000x4_fp64_against_the_exact_solution():
    """Config 0 on the GPU: FP64, 500 steps; L1 against the exact Riemann
    solution over cells 0..nx/2 (the shock has left through the open end by
    step ~340, the rarefaction has not)."""
    nx, steps = 1000, 500
    gpu, _ = run_gpu(0, 1.4, 0.6, 0.6, (nx, 4), (1, 0), li.sod_fields(nx, 4), steps, 0)
    _, _, r = ora.lattice_info(ora.D2Q37)
    er, eu, eT = riemann.shock_tube_profile((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, nx,
                                            riemann.lattice_time(steps, nx, r))
    half = slice(0, nx // 2)
    e = [riemann.l1_error(gpu[0][:nx], er, half), riemann.l1_error(gpu[1][0][:nx], eu, half),
         riemann.l1_error(gpu[2][:nx], eT, half)]
    print(f"Sod 1000x4 FP64 500 steps, L1 vs exact on cells 0..499: rho {e[0]:.4f} u {e[1]:.4f} T {e[2]:.4f}")
    assert max(e) < 0.005


def test_classic_sod_at_8192_is_unstable_in_the_oracle():
    nx = 8192
    _, _, r = ora.lattice_info(ora.D2Q37)
    steps = int(round(0.1504 * nx * r))
    out, _ = run_oracle(ora.D2Q37, 1.4, 0.6, 0.6, (nx, 1), (1, 0), li.sod_fields(nx, 1), steps)
    assert not np.all(np.isfinite(out[0]))
