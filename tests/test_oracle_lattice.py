"""Pins of the oracle's velocity sets against Tables I/II (Sec. IV) and the
Gaussian moments that a Hermite quadrature must reproduce."""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as ora

LATTICES = [(ora.D2Q37, 2, 37), (ora.D3Q107, 3, 107)]


def gauss_moment(n):
    """E[x^n] of the unit normal: (n-1)!! for even n, 0 for odd n."""
    if n % 2:
        return 0.0
    return float(np.prod(np.arange(n - 1, 0, -2))) if n > 0 else 1.0


@pytest.mark.parametrize("lat,D,Q", LATTICES)
def test_velocity_set_structure(lat, D, Q, golden):
    c, w, r = ora.lattice_info(lat)
    assert c.shape == (Q, D)
    assert len({tuple(v) for v in c}) == Q
    # closed under sign flips and axis permutations (the "Perm" of the tables)
    cs = {tuple(v) for v in c}
    for v in c:
        for p in itertools.permutations(v):
            for sg in itertools.product([1, -1], repeat=D):
                assert tuple(a * b for a, b in zip(p, sg)) in cs
    # group membership counts; the printed k of Table I is wrong for 2 groups
    name = "D2Q37" if D == 2 else "D3Q107"
    rows = [rw for rw in golden("paper_tables.txt") if rw[0] == name]
    total = 0
    for rw in rows:
        rep = tuple(int(x) for x in rw[1].split(","))
        members = [v for v in c if tuple(sorted(np.abs(v), reverse=True)) == rep]
        total += len(members)
        if D == 2 and rep in [(2, 1), (3, 1)]:
            assert len(members) == 8 and int(rw[2]) == 4  # printed misprint
        else:
            assert len(members) == int(rw[2])
        # all members of a group share the weight
        idx = [i for i, v in enumerate(c) if tuple(sorted(np.abs(v), reverse=True)) == rep]
        assert np.ptp(w[idx]) == 0.0
    assert total == Q


@pytest.mark.parametrize("lat,D,Q", LATTICES)
def test_isotropy_to_degree_9(lat, D, Q):
    """sum_i w_i xi_i^alpha equals the unit-Gaussian moment for every
    monomial of degree <= 9 (a 4th-order Hermite equilibrium needs the
    quadrature exact to degree 8 + 1 odd)."""
    c, w, r = ora.lattice_info(lat)
    xi = r * c.astype(np.float64)
    worst = 0.0
    for alpha in itertools.product(range(10), repeat=D):
        if sum(alpha) > 9:
            continue
        lhs = np.sum(w * np.prod(xi ** np.array(alpha), axis=1))
        rhs = np.prod([gauss_moment(a) for a in alpha])
        worst = max(worst, abs(lhs - rhs) / max(1.0, abs(rhs)))
    assert worst < 1e-13, worst


@pytest.mark.parametrize("lat,D,Q", LATTICES)
def test_degree_10_not_exact(lat, D, Q):
    """The quadrature is of degree 9, not more: the x^10 moment misses 945."""
    c, w, r = ora.lattice_info(lat)
    xi = r * c[:, 0].astype(np.float64)
    assert abs(np.sum(w * xi ** 10) - 945.0) > 1.0


@pytest.mark.parametrize("lat,D,Q", LATTICES)
def test_refined_weights_close_to_printed(lat, D, Q, golden):
    """The refined (r, w) stay close to the printed tables: <= 6e-8 relative
    (the printed r and weights are rounded to 9-10 digits), <= 2e-7 for the
    tiny D2Q37 (3,1) weight."""
    c, w, r = ora.lattice_info(lat)
    name = "D2Q37" if D == 2 else "D3Q107"
    for rw in golden("paper_tables.txt"):
        if rw[0] != name:
            continue
        rep = tuple(int(x) for x in rw[1].split(","))
        i = next(i for i, v in enumerate(c) if tuple(sorted(np.abs(v), reverse=True)) == rep)
        tol = 2e-7 if (D == 2 and rep == (3, 1)) else 6e-8
        assert abs(w[i] / float(rw[3]) - 1.0) < tol, (rep, w[i], rw[3])
    r_tab = float(next(rw for rw in golden("paper_tables.txt") if rw[0] == "r_table")[1])
    assert abs(r / r_tab - 1.0) < 1e-8
    assert abs(np.sum(w) - 1.0) < 1e-15


def test_printed_weights_are_not_normalised(golden):
    """Why the tables are refined: the printed D2Q37 weights sum to 1 + 1e-8."""
    c, w, r = ora.lattice_info(ora.D2Q37)
    printed = {tuple(int(x) for x in rw[1].split(",")): float(rw[3])
               for rw in golden("paper_tables.txt") if rw[0] == "D2Q37"}
    s = sum(printed[tuple(sorted(np.abs(v), reverse=True))] for v in c)
    assert abs(s - 1.0) > 5e-9


def test_same_r_in_2d_and_3d(golden):
    _, _, r2 = ora.lattice_info(ora.D2Q37)
    _, _, r3 = ora.lattice_info(ora.D3Q107)
    assert abs(r2 - r3) < 1e-14
    r5 = float(next(rw for rw in golden("paper_tables.txt") if rw[0] == "r_sec5")[1])
    assert abs(r2 / r5 - 1.0) < 1e-8


def test_time_mapping_sec5(golden):
    """Sec. V: t = step / (X r); 180 steps on X = 1000 give t = 0.1504."""
    from oracle import riemann
    rw = next(rw for rw in golden("paper_tables.txt") if rw[0] == "t_sec5")
    steps, X, t_printed = int(rw[1]), int(rw[2]), float(rw[3])
    _, _, r = ora.lattice_info(ora.D2Q37)
    assert round(riemann.lattice_time(steps, X, r), 4) == t_printed


def test_gamma_delta_relation():
    """Eq. (3): gamma = (delta + D + 2)/(delta + D)."""
    for D in (2, 3):
        for gamma in (1.1, 1.3, 1.4, 5.0 / 3.0):
            d = ora.delta_from_gamma(D, gamma)
            assert math.isclose((d + D + 2) / (d + D), gamma, rel_tol=1e-14)
    assert math.isclose(ora.delta_from_gamma(2, 1.4), 3.0, rel_tol=1e-14)   # Sec. V, 2D
    assert math.isclose(ora.delta_from_gamma(3, 1.4), 2.0, rel_tol=1e-14)   # Sec. V, 3D


@pytest.mark.parametrize("lat", [ora.D2Q37, ora.D3Q107])
def test_refined_table_is_the_exact_solution_rounded(lat):
    """The oracle's refined (w, r) equal the solution of the isotropy
    conditions solved at 50 digits and rounded to double, to the last bit:
    the refinement's double-double residuals leave no algorithm-dependent
    error (reading R3)."""
    pytest.importorskip("mpmath")
    from tests.isotropy_exact import exact_table, group_weights
    c, w, r = ora.lattice_info(lat)
    wg = group_weights(c, w)
    we, re_ = exact_table(lat, wg, r)
    assert r == re_
    assert np.array_equal(wg, we)
