"""The exact refined velocity tables: the solution of the even-moment
isotropy conditions of degree 0..8 (Tables I/II, reading R3), solved at 50
significant digits with mpmath and rounded to double.  An independent
statement of what both refinements (the oracle's and the library's) must
return; used by the CPU pins only."""
import numpy as np

# even monomial classes (exponents of x, y, z) of degree <= 8, one per
# condition: G + 1 conditions for the G group weights and r
MONOMIALS = {
    0: [(0, 0, 0), (2, 0, 0), (4, 0, 0), (2, 2, 0), (6, 0, 0), (4, 2, 0), (8, 0, 0), (6, 2, 0), (4, 4, 0)],
    1: [(0, 0, 0), (2, 0, 0), (4, 0, 0), (2, 2, 0), (6, 0, 0), (4, 2, 0), (2, 2, 2), (8, 0, 0), (6, 2, 0),
        (4, 4, 0), (4, 2, 2)],
}
# group representatives (sorted |c|) of Tables I and II
GROUPS = {
    0: [(0, 0, 0), (1, 0, 0), (1, 1, 0), (2, 0, 0), (2, 1, 0), (3, 0, 0), (3, 1, 0), (3, 3, 0)],
    1: [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1), (2, 0, 0), (2, 1, 1), (2, 2, 0), (2, 2, 2), (3, 0, 0),
        (3, 1, 1)],
}


def _gauss(n):
    if n % 2:
        return 0
    m = 1
    for k in range(n - 1, 1, -2):
        m *= k
    return m


def exact_table(lattice, w_start, r_start):
    """(group weights, r) rounded to double from a 50-digit Newton solve
    started at (w_start, r_start)."""
    import mpmath as mp
    mp.mp.dps = 50
    D = 2 if lattice == 0 else 3
    reps = GROUPS[lattice]
    rng = range(-3, 4)
    members = [[] for _ in reps]
    for x in rng:
        for y in rng:
            for z in (rng if D == 3 else [0]):
                key = tuple(sorted((abs(x), abs(y), abs(z)), reverse=True))
                if key in reps:
                    members[reps.index(key)].append((x, y, z))
    monos = MONOMIALS[lattice]
    G = len(reps)
    M = [[sum(c[0] ** m[0] * c[1] ** m[1] * c[2] ** m[2] for c in members[g]) for g in range(G)] for m in monos]
    deg = [sum(m) for m in monos]
    tgt = [_gauss(m[0]) * _gauss(m[1]) * _gauss(m[2]) for m in monos]

    def F(*x):
        return [x[G] ** deg[k] * sum(x[g] * M[k][g] for g in range(G)) - tgt[k] for k in range(G + 1)]
    sol = mp.findroot(F, [mp.mpf(float(v)) for v in w_start] + [mp.mpf(float(r_start))])
    return np.array([float(sol[g]) for g in range(G)]), float(sol[G])


def group_weights(c, w):
    """Per-group weights of a velocity table (c[Q, D], w[Q]) in the order of
    GROUPS."""
    D = c.shape[1]
    reps = GROUPS[0 if D == 2 else 1]
    out = np.zeros(len(reps))
    for v, wi in zip(c, w):
        key = tuple(sorted([abs(int(a)) for a in v] + [0] * (3 - D), reverse=True))
        out[reps.index(key)] = wi
    return out
