"""Pins of the oracle's equilibrium, Eq. (18), against the Maxwellian of
Eq. (10) it approximates: its velocity moments through order 4 must equal the
Maxwellian's closed-form moments, and the scalar Hermite contractions must
equal an explicit tensor evaluation of a(k).H(k)."""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as ora

LATTICES = [(ora.D2Q37, 2), (ora.D3Q107, 3)]


def normal_raw_moment(n, mu, var):
    """E[x^n] for x ~ N(mu, var): sum_k C(n, 2k) mu^(n-2k) var^k (2k-1)!!."""
    s = 0.0
    for k in range(n // 2 + 1):
        dfact = float(np.prod(np.arange(2 * k - 1, 0, -2))) if k > 0 else 1.0
        s += math.comb(n, 2 * k) * mu ** (n - 2 * k) * var ** k * dfact
    return s


def random_states(n, D, seed):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        yield rng.uniform(0.5, 2.0), rng.uniform(-0.3, 0.3, D), rng.uniform(0.7, 1.3)


@pytest.mark.parametrize("lat,D", LATTICES)
def test_moments_match_maxwellian_to_order_4(lat, D):
    c, w, r = ora.lattice_info(lat)
    xi = r * c.astype(np.float64)
    worst = 0.0
    for rho, u, T in random_states(12, D, seed=11 + D):
        F = ora.feq(lat, rho, u, T)
        for alpha in itertools.product(range(5), repeat=D):
            if sum(alpha) > 4:
                continue
            lhs = np.sum(F * np.prod(xi ** np.array(alpha), axis=1)) / rho
            rhs = np.prod([normal_raw_moment(a, u[k], T) for k, a in enumerate(alpha)])
            worst = max(worst, abs(lhs - rhs))
    assert worst < 1e-13, worst


@pytest.mark.parametrize("lat,D", LATTICES)
def test_order_5_is_not_matched(lat, D):
    """A 4th-order expansion misses the 5th moment away from u = 0."""
    c, w, r = ora.lattice_info(lat)
    xi = r * c[:, 0].astype(np.float64)
    u = np.zeros(D)
    u[0] = 0.3
    F = ora.feq(lat, 1.0, u, 1.2)
    assert abs(np.sum(F * xi ** 5) - normal_raw_moment(5, 0.3, 1.2)) > 1e-4


@pytest.mark.parametrize("lat,D", LATTICES)
def test_rest_state_gives_weights(lat, D):
    c, w, r = ora.lattice_info(lat)
    F = ora.feq(lat, 1.7, np.zeros(D), 1.0)
    np.testing.assert_allclose(F, 1.7 * w, rtol=1e-15, atol=0)


def hermite_tensors(x, D):
    """Tensor Hermite polynomials H0..H4 of the unit Gaussian weight,
    built from their definitions H(k) = (-1)^k w^{-1} grad^k w."""
    I = np.eye(D)
    H1 = x.copy()
    H2 = np.einsum("a,b->ab", x, x) - I
    H3 = (np.einsum("a,b,c->abc", x, x, x)
          - np.einsum("a,bc->abc", x, I) - np.einsum("b,ac->abc", x, I) - np.einsum("c,ab->abc", x, I))
    xx = np.einsum("a,b->ab", x, x)
    H4 = (np.einsum("a,b,c,d->abcd", x, x, x, x)
          - sum(np.einsum(s, xx, I) for s in ["ab,cd->abcd", "ac,bd->abcd", "ad,bc->abcd",
                                               "bc,ad->abcd", "bd,ac->abcd", "cd,ab->abcd"])
          + np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I) + np.einsum("ad,bc->abcd", I, I))
    return 1.0, H1, H2, H3, H4


def maxwellian_coeffs(u, T, D):
    """Hermite coefficients a(k) of the rho-normalised Maxwellian N(u, T I)
    about the unit Gaussian: a(k) = E[H(k)(x)] for x ~ N(u, T I), taken
    here by exact Gauss-Hermite quadrature of that expectation (10 points per
    axis), independent of any closed form."""
    z, wz = np.polynomial.hermite_e.hermegauss(10)
    wz = wz / wz.sum()
    a = [0.0, np.zeros(D), np.zeros((D,) * 2), np.zeros((D,) * 3), np.zeros((D,) * 4)]
    for idx in itertools.product(range(len(z)), repeat=D):
        x = u + np.sqrt(T) * z[list(idx)]
        wt = np.prod(wz[list(idx)])
        H = hermite_tensors(x, D)
        a[0] += wt * H[0]
        for k in range(1, 5):
            a[k] = a[k] + wt * H[k]
    return a


@pytest.mark.parametrize("lat,D", LATTICES)
def test_scalar_contractions_equal_tensor_form(lat, D):
    c, w, r = ora.lattice_info(lat)
    xi = r * c.astype(np.float64)
    fact = [1.0, 1.0, 2.0, 6.0, 24.0]
    for rho, u, T in random_states(3, D, seed=5 + D):
        a = maxwellian_coeffs(u, T, D)
        F = ora.feq(lat, rho, u, T)
        for i in range(0, len(xi), 7 if D == 3 else 3):
            H = hermite_tensors(xi[i], D)
            s = a[0] * H[0]
            for k in range(1, 5):
                s += np.sum(a[k] * H[k]) / fact[k]
            assert abs(F[i] - w[i] * rho * s) <= 1e-13 * max(1.0, abs(w[i] * rho * s)) + 1e-16


@pytest.mark.parametrize("lat,D", LATTICES)
def test_printed_form_of_eq18_fails_mass(lat, D):
    """The reading that the printed a(2..4).H(2..4) are garbled: evaluated as
    printed (with (theta-1)(theta^2-D) in a2 and u^2 <-> xi^2 swapped in a3,
    a4), the sum of F_i is not rho."""
    c, w, r = ora.lattice_info(lat)
    xi = r * c.astype(np.float64)
    rho, u, T = 1.0, np.full(D, 0.1), 1.1
    s = xi @ u
    u2 = u @ u
    x2 = np.sum(xi * xi, axis=1)
    t = T - 1.0
    p2 = s * s + t * (T * T - D) - u2
    p3 = s * (s * s - 3 * u2 + 3 * t * (u2 - D - 2))
    p4 = (s ** 4 - 6 * s * s * u2 + 3 * u2 ** 2 + 6 * t * (s * s * (u2 - D - 4) + (D + 2 - u2) * x2)
          + 3 * t * t * (u2 ** 2 - 2 * (D + 2) * u2 + D * (D + 2)))
    F_printed = w * rho * (1 + s + p2 / 2 + p3 / 6 + p4 / 24)
    assert abs(F_printed.sum() - rho) > 0.1
    assert abs(ora.feq(lat, rho, u, T).sum() - rho) < 1e-14
