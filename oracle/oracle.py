"""ctypes binding of the plain FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline / reference arm use this module to compute what the GPU library
must reproduce.  The product package never imports it.

The oracle follows the paper (arXiv 1608.06345) step by step in FP64:
Eq. (18) equilibrium (with the derived Hermite contractions), Eq. (14)/(15)
moments, exact pull streaming and the BGK relaxation of Eq. (16)/(17), on the
D2Q37 / D3Q107 velocity sets of Tables I and II (weights refined by Newton's
method on the isotropy conditions).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "_build", "liblbm_oracle.so")

# Rounding variants of the oracle (bits of ORA_VARIANT in lbm_oracle.c):
# 1 reversed velocity order of every sum, 2 fused multiply-adds, 4 the
# relaxation as (1 - 1/tau) q + Q_eq/tau, 8 populations held as deviations
# from a reference equilibrium (Oracle.set_reference), 16 FP32 arithmetic and
# storage, 32 the equilibrium as a polynomial in s (Horner).  They change
# rounding only; the tests use them as second checkers
# to measure how far correct evaluations of the scheme in FP64 (or in FP32)
# land from the oracle on a flow.
VARIANTS_F64 = (1, 2, 4, 7, 8, 15, 32, 47)
VARIANTS_F32 = (16, 17, 18, 20, 23, 24, 31, 48, 63)
VARIANTS = VARIANTS_F64 + VARIANTS_F32

D2Q37 = 0
D3Q107 = 1
PERIODIC = 0
ZERO_GRADIENT = 1

_libs = {}


def lib_path(variant: int = 0) -> str:
    return LIB if variant == 0 else os.path.join(HERE, "_build", f"liblbm_oracle_v{variant}.so")


def build(force: bool = False, variants=(0,) + VARIANTS) -> str:
    """Compile the oracle (and its rounding variants) with gcc: FP64, no
    FMA contraction by the compiler, OpenMP.  Returns the oracle's path."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    for v in variants:
        out = lib_path(v)
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(SRC):
            cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                   "-fopenmp", "-shared", "-fPIC", f"-DORA_VARIANT={v}", SRC, "-o", out + ".tmp", "-lm"]
            if v & 16:  # FP32 variants: unsuffixed literals stay FP32
                cmd.insert(1, "-fsingle-precision-constant")
            subprocess.check_call(cmd)
            os.replace(out + ".tmp", out)
    return LIB


def _load(variant: int = 0):
    if variant in _libs:
        return _libs[variant]
    if variant != 0 and variant not in VARIANTS:
        raise ValueError(f"unknown oracle variant {variant}")
    build(variants=(variant,))
    lib = ctypes.CDLL(lib_path(variant))
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.ora_new.restype = ctypes.c_void_p
    lib.ora_new.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.ora_free.argtypes = [ctypes.c_void_p]
    lib.ora_init.argtypes = [ctypes.c_void_p, dp, dp, dp]
    lib.ora_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
    lib.ora_step_fd.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_double]
    lib.ora_moments.argtypes = [ctypes.c_void_p, dp, dp, dp]
    lib.ora_conserved.argtypes = [ctypes.c_void_p, dp]
    lib.ora_get_pops.argtypes = [ctypes.c_void_p, dp, dp]
    lib.ora_set_pops.argtypes = [ctypes.c_void_p, dp, dp]
    lib.ora_delta.restype = ctypes.c_double
    lib.ora_delta.argtypes = [ctypes.c_void_p]
    lib.ora_delta_from_gamma.restype = ctypes.c_double
    lib.ora_delta_from_gamma.argtypes = [ctypes.c_int, ctypes.c_double]
    lib.ora_lattice_info.restype = ctypes.c_int
    lib.ora_lattice_info.argtypes = [ctypes.c_int, ip, ip, dp, dp]
    lib.ora_feq.restype = ctypes.c_int
    lib.ora_feq.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, dp]
    lib.ora_set_threads.argtypes = [ctypes.c_int]
    lib.ora_get_threads.restype = ctypes.c_int
    lib.ora_set_reference.restype = ctypes.c_int
    lib.ora_set_reference.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
    _libs[variant] = lib
    return lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def dim(lattice: int) -> int:
    return 2 if lattice == D2Q37 else 3


def lattice_info(lattice: int):
    """(c[Q, D] int, w[Q], r) of the oracle's refined lattice."""
    lib = _load()
    q = ctypes.c_int()
    D = dim(lattice)
    c = np.zeros(107 * D, dtype=np.int32)
    w = np.zeros(107)
    r = ctypes.c_double()
    rc = lib.ora_lattice_info(lattice, ctypes.byref(q), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                              _p(w), ctypes.byref(r))
    if rc:
        raise RuntimeError(f"oracle lattice build failed: {rc}")
    Q = q.value
    return c[: Q * D].reshape(Q, D).astype(np.int64), w[:Q].copy(), r.value


def feq(lattice: int, rho: float, u, T: float) -> np.ndarray:
    """Equilibrium F_i of Eq. (18) for one state."""
    lib = _load()
    uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    F = np.zeros(107)
    rc = lib.ora_feq(lattice, float(rho), _p(uu), float(T), _p(F))
    if rc:
        raise RuntimeError("oracle feq failed")
    Q = 37 if lattice == D2Q37 else 107
    return F[:Q].copy()


def delta_from_gamma(D: int, gamma: float) -> float:
    return _load().ora_delta_from_gamma(D, gamma)


def set_threads(n: int) -> None:
    _load().ora_set_threads(int(n))


def get_threads() -> int:
    return int(_load().ora_get_threads())


class Oracle:
    """One FP64 solver instance: ``init`` -> ``step(n)`` -> ``moments``.
    ``variant`` selects a rounding variant (VARIANTS) instead of the oracle."""

    def __init__(self, lattice: int, gamma: float, tau_f: float, tau_g: float,
                 shape, bc=(PERIODIC, PERIODIC, PERIODIC), variant: int = 0):
        lib = _load(variant)
        self.lattice = lattice
        self.D = dim(lattice)
        shape = tuple(int(s) for s in shape)
        if len(shape) == 2:
            shape = shape + (1,)
        self.nx, self.ny, self.nz = shape
        self.N = self.nx * self.ny * self.nz
        self.Q = 37 if lattice == D2Q37 else 107
        bc = tuple(bc) + (PERIODIC,) * (3 - len(bc))
        self._h = lib.ora_new(lattice, gamma, tau_f, tau_g, self.nx, self.ny, self.nz, *bc[:3])
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        self._lib = lib
        self.delta = lib.ora_delta(self._h)

    def close(self):
        if self._h:
            self._lib.ora_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_reference(self, rho_r: float, T_r: float):
        """Reference state of a deviation variant (bit 8); call before init."""
        if self._lib.ora_set_reference(self._h, float(rho_r), float(T_r)):
            raise ValueError("this oracle build stores the populations whole")

    def init(self, rho, u, T):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(-1)
        assert rho.size == self.N and T.size == self.N and u.size == self.D * self.N
        self._lib.ora_init(self._h, _p(rho), _p(u), _p(T))

    def step(self, n: int = 1):
        self._lib.ora_step(self._h, int(n))

    def step_fd(self, n=1, lam=0.1):
        """Finite-difference steps of Sec. III with lambda = dt/dx."""
        self._lib.ora_step_fd(self._h, int(n), float(lam))

    def moments(self):
        rho = np.zeros(self.N)
        u = np.zeros(self.D * self.N)
        T = np.zeros(self.N)
        self._lib.ora_moments(self._h, _p(rho), _p(u), _p(T))
        return rho, u.reshape(self.D, self.N), T

    def conserved(self) -> np.ndarray:
        out = np.zeros(2 + self.D)
        self._lib.ora_conserved(self._h, _p(out))
        return out

    def get_pops(self):
        g = np.zeros(self.Q * self.N)
        h = np.zeros(self.Q * self.N)
        self._lib.ora_get_pops(self._h, _p(g), _p(h))
        return g.reshape(self.Q, self.N), h.reshape(self.Q, self.N)

    def set_pops(self, g, h):
        g = np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
        h = np.ascontiguousarray(h, dtype=np.float64).reshape(-1)
        assert g.size == self.Q * self.N and h.size == self.Q * self.N
        self._lib.ora_set_pops(self._h, _p(g), _p(h))
