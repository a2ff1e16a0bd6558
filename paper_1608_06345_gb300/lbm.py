"""Python binding of the C ABI in ``include/lbm.h`` (ctypes).

The functions keep the C names (``lbm_create``, ``lbm_init``, ``lbm_step``,
``lbm_moments``, ``lbm_conserved``, ``lbm_destroy`` ...) and only marshal
arguments; every step of the computation runs in the CUDA library.  PyTorch
supplies device memory (``Solver`` allocates the instance's buffer as a torch
tensor, so it comes from torch's caching allocator) and streams.

There is no CPU fallback: if the shared library is missing the import fails
loudly (build it with ``python -m paper_1608_06345_gb300.build``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_EBUSY = range(7)
LBM_D2Q37, LBM_D3Q107 = 0, 1
LBM_PERIODIC, LBM_ZERO_GRADIENT = 0, 1
LBM_F64, LBM_F32, LBM_F32_S16F, LBM_F32_S16BF = 0, 1, 2, 3
LBM_FD_AUTO, LBM_FD_CELL, LBM_FD_MARCH = 0, 1, 2

PREC_NAMES = {"f64": LBM_F64, "f32": LBM_F32, "f32_s16f": LBM_F32_S16F, "f32_s16bf": LBM_F32_S16BF}
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_ENONFINITE",
                5: "LBM_ETIMEOUT", 6: "LBM_EBUSY"}

# every entry point of include/lbm.h
EXPORTS = ["lbm_state_bytes", "lbm_create", "lbm_destroy", "lbm_init", "lbm_init_device", "lbm_step",
           "lbm_moments", "lbm_moments_device", "lbm_conserved", "lbm_sync", "lbm_steps_done",
           "lbm_raw_state_bytes", "lbm_get_state", "lbm_set_state", "lbm_lattice_table", "lbm_last_error",
           "lbm_conserved_noalloc", "lbm_pool_bytes", "lbm_pool_create", "lbm_pool_destroy",
           "lbm_pool_instance_bytes", "lbm_pool_submit", "lbm_pool_run", "lbm_pool_sync", "lbm_pool_poll",
           "lbm_pool_result", "lbm_pool_stats", "lbm_shape_info", "lbm_set_shape", "lbm_get_shape",
           "lbm_autotune", "lbm_set_graph_steps", "lbm_quadrature", "lbm_step_fd", "lbm_set_fd_kernel",
           "lbm_slab_plan",
           "lbm_slab_pack", "lbm_slab_unpack"]


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class lbm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("bc", ctypes.c_int * 3), ("prec", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("device_mem", ctypes.c_void_p), ("device_bytes", ctypes.c_size_t),
                ("rho0", ctypes.c_double), ("T0", ctypes.c_double)]


class lbm_slab(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("axis", ctypes.c_int), ("n", ctypes.c_int * 3),
                ("periodic", ctypes.c_int), ("nranks", ctypes.c_int), ("rank", ctypes.c_int),
                ("begin", ctypes.c_int), ("end", ctypes.c_int), ("lo", ctypes.c_int), ("hi", ctypes.c_int),
                ("layer_cells", ctypes.c_int), ("local_n", ctypes.c_int * 3), ("msg_values", ctypes.c_longlong)]


class lbm_pool_config(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("prec", ctypes.c_int), ("budget_bytes", ctypes.c_size_t),
                ("max_instances", ctypes.c_int), ("max_tiles", ctypes.c_int), ("bundle_steps", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("device_mem", ctypes.c_void_p), ("device_bytes", ctypes.c_size_t)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load liblbm.so (raising if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise ImportError(f"CUDA library not built: {path} (run python -m paper_1608_06345_gb300.build)")
    lib = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    gp = ctypes.POINTER(lbm_grid)
    sig = {
        "lbm_state_bytes": (ctypes.c_size_t, [ctypes.c_int, gp]),
        "lbm_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, gp]),
        "lbm_destroy": (ctypes.c_int, [vp]),
        "lbm_init": (ctypes.c_int, [vp, vp, vp, vp]),
        "lbm_init_device": (ctypes.c_int, [vp, vp, vp, vp]),
        "lbm_step": (ctypes.c_int, [vp, ctypes.c_long]),
        "lbm_step_fd": (ctypes.c_int, [vp, ctypes.c_long, ctypes.c_double]),
        "lbm_moments": (ctypes.c_int, [vp, vp, vp, vp]),
        "lbm_moments_device": (ctypes.c_int, [vp, vp, vp, vp]),
        "lbm_conserved": (ctypes.c_int, [vp, dp]),
        "lbm_sync": (ctypes.c_int, [vp]),
        "lbm_steps_done": (ctypes.c_long, [vp]),
        "lbm_raw_state_bytes": (ctypes.c_size_t, [vp]),
        "lbm_get_state": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
        "lbm_set_state": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
        "lbm_lattice_table": (ctypes.c_int, [ctypes.c_int, ip, ip, dp, dp]),
        "lbm_last_error": (ctypes.c_char_p, []),
        "lbm_conserved_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_double, vp, ctypes.c_longlong, ctypes.c_longlong, vp, dp]),
        "lbm_shape_info": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip]),
        "lbm_set_shape": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_get_shape": (ctypes.c_int, [vp]),
        "lbm_autotune": (ctypes.c_int, [vp, ctypes.c_int, ip, dp]),
        "lbm_set_graph_steps": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_set_fd_kernel": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_quadrature": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, ip, ctypes.c_double, ip,
                                          dp, dp, dp]),
        "lbm_slab_plan": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.POINTER(lbm_slab)]),
        "lbm_slab_pack": (ctypes.c_int, [ctypes.POINTER(lbm_slab), vp, ctypes.c_longlong, vp, vp]),
        "lbm_slab_unpack": (ctypes.c_int, [ctypes.POINTER(lbm_slab), vp, ctypes.c_longlong, vp, vp]),
        "lbm_pool_bytes": (ctypes.c_size_t, [ctypes.POINTER(lbm_pool_config)]),
        "lbm_pool_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(lbm_pool_config)]),
        "lbm_pool_destroy": (ctypes.c_int, [vp]),
        "lbm_pool_instance_bytes": (ctypes.c_size_t, [vp, gp]),
        "lbm_pool_submit": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, gp, vp, vp, vp,
                                           ctypes.c_long, ctypes.POINTER(ctypes.c_longlong)]),
        "lbm_pool_run": (ctypes.c_int, [vp, ctypes.c_int]),
        "lbm_pool_sync": (ctypes.c_int, [vp]),
        "lbm_pool_poll": (ctypes.c_int, [vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_long)]),
        "lbm_pool_result": (ctypes.c_int, [vp, ctypes.c_longlong, vp, vp, vp]),
        "lbm_pool_stats": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_longlong)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc):
    if rc != LBM_OK:
        raise LbmError(rc, load().lbm_last_error().decode())
    return rc


def _ptr(a):
    """Address of a numpy array or torch tensor (None for None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def dim(lattice):
    return 2 if lattice == LBM_D2Q37 else 3


def make_grid(shape, bc=(LBM_PERIODIC,) * 3, prec=LBM_F32, stream=None, device_mem=None, device_bytes=0,
              rho0=0.0, T0=0.0):
    shape = tuple(int(s) for s in shape) + (1,) * (3 - len(shape))
    bc = tuple(bc) + (LBM_PERIODIC,) * (3 - len(bc))
    g = lbm_grid()
    g.nx, g.ny, g.nz = shape
    g.bc[0], g.bc[1], g.bc[2] = bc[:3]
    g.prec = prec
    g.stream = stream
    g.device_mem = device_mem
    g.device_bytes = device_bytes
    g.rho0 = rho0
    g.T0 = T0
    return g


def lbm_state_bytes(lattice, grid):
    return load().lbm_state_bytes(lattice, ctypes.byref(grid))


def lbm_create(lattice, gamma, tau_f, tau_g, grid):
    h = ctypes.c_void_p()
    _check(load().lbm_create(ctypes.byref(h), lattice, gamma, tau_f, tau_g, ctypes.byref(grid)))
    return h


def lbm_destroy(h):
    return _check(load().lbm_destroy(h))


def lbm_init(h, rho, u, T):
    return _check(load().lbm_init(h, _ptr(rho), _ptr(u), _ptr(T)))


def lbm_init_device(h, rho, u, T):
    return _check(load().lbm_init_device(h, _ptr(rho), _ptr(u), _ptr(T)))


def lbm_step(h, n):
    return _check(load().lbm_step(h, int(n)))


def lbm_step_fd(h, n, lam):
    return _check(load().lbm_step_fd(h, int(n), float(lam)))


def lbm_moments(h, rho, u, T):
    return _check(load().lbm_moments(h, _ptr(rho), _ptr(u), _ptr(T)))


def lbm_moments_device(h, rho, u, T):
    return _check(load().lbm_moments_device(h, _ptr(rho), _ptr(u), _ptr(T)))


def lbm_conserved(h, D):
    out = np.zeros(2 + D)
    _check(load().lbm_conserved(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def lbm_sync(h):
    return _check(load().lbm_sync(h))


def lbm_steps_done(h):
    return load().lbm_steps_done(h)


def lbm_raw_state_bytes(h):
    return load().lbm_raw_state_bytes(h)


def lbm_get_state(h, host):
    return _check(load().lbm_get_state(h, _ptr(host), host.nbytes))


def lbm_set_state(h, host):
    return _check(load().lbm_set_state(h, _ptr(host), host.nbytes))


def lbm_lattice_table(lattice):
    """(c[Q, D], w[Q], r) of the library's refined lattice."""
    q = ctypes.c_int()
    D = dim(lattice)
    c = np.zeros(107 * D, dtype=np.int32)
    w = np.zeros(107)
    r = ctypes.c_double()
    _check(load().lbm_lattice_table(lattice, ctypes.byref(q), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                    w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(r)))
    Q = q.value
    return c[: Q * D].reshape(Q, D).astype(np.int64), w[:Q].copy(), r.value


def lbm_shape_info(lattice, prec, index):
    """(stage, block) of candidate shape `index`, or None past the end."""
    st, bx = ctypes.c_int(), ctypes.c_int()
    rc = load().lbm_shape_info(lattice, prec, index, ctypes.byref(st), ctypes.byref(bx))
    return (st.value, bx.value) if rc == LBM_OK else None


def lbm_set_shape(h, index):
    return _check(load().lbm_set_shape(h, int(index)))


def lbm_get_shape(h):
    return load().lbm_get_shape(h)


def lbm_quadrature(reps, exps, r0=1.0):
    """General Hermite quadrature: reps (G x D group representatives), exps
    (n x D even exponents).  Returns (weights per group, r, Q, max residual)."""
    reps = np.ascontiguousarray(np.asarray(reps, dtype=np.int32))
    exps = np.ascontiguousarray(np.asarray(exps, dtype=np.int32))
    G, D = reps.shape
    n = exps.shape[0]
    w = np.zeros(G)
    q, r, res = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    _check(load().lbm_quadrature(D, G, reps.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), n,
                                 exps.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), float(r0), ctypes.byref(q),
                                 w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(r),
                                 ctypes.byref(res)))
    return w, r.value, q.value, res.value


def lbm_set_graph_steps(h, steps):
    return _check(load().lbm_set_graph_steps(h, int(steps)))


def lbm_set_fd_kernel(h, kernel):
    return _check(load().lbm_set_fd_kernel(h, int(kernel)))


def lbm_autotune(h, reps=5):
    """(best shape index, microseconds per step)."""
    k, us = ctypes.c_int(), ctypes.c_double()
    _check(load().lbm_autotune(h, int(reps), ctypes.byref(k), ctypes.byref(us)))
    return k.value, us.value


def lbm_conserved_noalloc(lattice, prec, gamma, state, ncells, plane_stride, stream=None, rho0=0.0, T0=0.0):
    """Totals of a raw device state without any allocation (see include/lbm.h).
    `state` is a device pointer (int) or a CUDA tensor; returns out[D + 2].
    A tensor must hold the whole extent of the planes: (2Q-1) plane_stride +
    ncells words (Q-1 strides plus ncells 4-byte pairs for 16-bit storage)."""
    if isinstance(state, int):
        ptr = state
    else:
        Q = 37 if lattice == LBM_D2Q37 else 107
        word = 8 if prec == LBM_F64 else 4
        planes = Q if prec in (LBM_F32_S16F, LBM_F32_S16BF) else 2 * Q
        need = ((planes - 1) * int(plane_stride) + int(ncells)) * word if ncells > 0 else 0
        have = state.numel() * state.element_size()
        if have < need:
            raise LbmError(LBM_EINVAL, f"state holds {have} bytes, the planes need {need}")
        ptr = _ptr(state)
    out = np.zeros(2 + dim(lattice))
    _check(load().lbm_conserved_noalloc(lattice, prec, gamma, rho0, T0, ptr, int(ncells), int(plane_stride),
                                        stream, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def lbm_slab_plan(lattice, n, periodic, nranks, rank):
    """Slab plan of one rank (include/lbm.h); returns an lbm_slab."""
    nn = (ctypes.c_int * 3)(*[int(v) for v in tuple(n) + (1,) * (3 - len(n))])
    s = lbm_slab()
    _check(load().lbm_slab_plan(lattice, nn, int(bool(periodic)), nranks, rank, ctypes.byref(s)))
    return s


def lbm_slab_pack(s, state, plane_stride, to_lo, to_hi):
    """state: float64 array of 2Q planes of plane_stride values; to_lo /
    to_hi: float64 arrays of s.msg_values (or None)."""
    for a in (to_lo, to_hi):
        assert a is None or (a.dtype == np.float64 and a.size >= s.msg_values)
    assert state.dtype == np.float64 and state.flags.c_contiguous
    _check(load().lbm_slab_pack(ctypes.byref(s), _ptr(state), int(plane_stride), _ptr(to_lo), _ptr(to_hi)))


def lbm_slab_unpack(s, state, plane_stride, from_lo, from_hi):
    for a in (from_lo, from_hi):
        assert a is None or (a.dtype == np.float64 and a.size >= s.msg_values)
    assert state.dtype == np.float64 and state.flags.c_contiguous
    _check(load().lbm_slab_unpack(ctypes.byref(s), _ptr(state), int(plane_stride), _ptr(from_lo), _ptr(from_hi)))


def lbm_last_error():
    return load().lbm_last_error().decode()


class Solver:
    """One simulation instance on the current CUDA device.

    Device memory is a torch uint8 tensor of ``lbm_state_bytes`` (torch's
    caching allocator); work runs on ``stream`` (default: torch's current
    stream), so torch events and syncs order correctly with it."""

    def __init__(self, lattice, gamma, tau_f, tau_g, shape, bc=(LBM_PERIODIC,) * 3, prec=LBM_F32,
                 stream=None, rho0=0.0, T0=0.0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Solver needs a CUDA device")
        self.lattice = lattice
        self.D = dim(lattice)
        self.Q = 37 if lattice == LBM_D2Q37 else 107
        shape = tuple(int(s) for s in shape) + (1,) * (3 - len(shape))
        self.shape = shape
        self.N = shape[0] * shape[1] * shape[2]
        self.prec = prec
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g = make_grid(shape, bc, prec, stream=self.stream.cuda_stream, rho0=rho0, T0=T0)
        nbytes = lbm_state_bytes(lattice, g)
        if nbytes == 0:
            raise LbmError(LBM_EINVAL, "invalid grid")
        with torch.cuda.stream(self.stream):
            self.mem = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        g.device_mem = self.mem.data_ptr()
        g.device_bytes = nbytes
        self.grid = g
        self.h = lbm_create(lattice, gamma, tau_f, tau_g, g)

    def close(self):
        if getattr(self, "h", None) is not None:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho, u, T):
        """Host (numpy float64) or device (torch float64 cuda) fields."""
        if isinstance(rho, np.ndarray):
            rho = np.ascontiguousarray(rho, dtype=np.float64)
            u = np.ascontiguousarray(u, dtype=np.float64)
            T = np.ascontiguousarray(T, dtype=np.float64)
            assert rho.size == self.N and u.size == self.D * self.N and T.size == self.N
            lbm_init(self.h, rho, u, T)
        else:
            assert rho.is_cuda and rho.is_contiguous() and u.is_contiguous() and T.is_contiguous()
            lbm_init_device(self.h, rho, u, T)

    def step(self, n=1):
        lbm_step(self.h, n)

    def step_fd(self, n=1, lam=0.05):
        """Finite-difference steps (Sec. III) with lambda = dt/dx."""
        lbm_step_fd(self.h, n, lam)

    def set_fd_kernel(self, kernel):
        """LBM_FD_AUTO, LBM_FD_CELL or LBM_FD_MARCH (lbm_set_fd_kernel)."""
        lbm_set_fd_kernel(self.h, kernel)

    def moments(self):
        rho = np.zeros(self.N)
        u = np.zeros(self.D * self.N)
        T = np.zeros(self.N)
        lbm_moments(self.h, rho, u, T)
        return rho, u.reshape(self.D, self.N), T

    def moments_device(self, rho, u, T):
        lbm_moments_device(self.h, rho, u, T)

    def conserved(self):
        return lbm_conserved(self.h, self.D)

    def sync(self):
        lbm_sync(self.h)


# ---------------------------------------------------------------------------
# continuous-batching pool
# ---------------------------------------------------------------------------
def make_pool_config(lattice, prec, budget_bytes, max_instances, bundle_steps, max_tiles=0, stream=None,
                     device_mem=None, device_bytes=0):
    c = lbm_pool_config()
    c.lattice, c.prec = lattice, prec
    c.budget_bytes = int(budget_bytes)
    c.max_instances, c.max_tiles, c.bundle_steps = int(max_instances), int(max_tiles), int(bundle_steps)
    c.stream, c.device_mem, c.device_bytes = stream, device_mem, device_bytes
    return c


def lbm_pool_bytes(cfg):
    return load().lbm_pool_bytes(ctypes.byref(cfg))


def lbm_pool_create(cfg):
    h = ctypes.c_void_p()
    _check(load().lbm_pool_create(ctypes.byref(h), ctypes.byref(cfg)))
    return h


def lbm_pool_destroy(p):
    return _check(load().lbm_pool_destroy(p))


def lbm_pool_instance_bytes(p, grid):
    return load().lbm_pool_instance_bytes(p, ctypes.byref(grid))


def lbm_pool_submit(p, gamma, tau_f, tau_g, grid, rho, u, T, steps):
    """Ticket of the admitted instance, or None when the pool is busy (LBM_EBUSY)."""
    t = ctypes.c_longlong()
    rc = load().lbm_pool_submit(p, gamma, tau_f, tau_g, ctypes.byref(grid), _ptr(rho), _ptr(u), _ptr(T),
                                int(steps), ctypes.byref(t))
    if rc == LBM_EBUSY:
        return None
    _check(rc)
    return t.value


def lbm_pool_run(p, bundles=1):
    return _check(load().lbm_pool_run(p, int(bundles)))


def lbm_pool_sync(p):
    return _check(load().lbm_pool_sync(p))


def lbm_pool_poll(p, ticket):
    done = ctypes.c_int()
    steps = ctypes.c_long()
    _check(load().lbm_pool_poll(p, ticket, ctypes.byref(done), ctypes.byref(steps)))
    return bool(done.value), steps.value


def lbm_pool_result(p, ticket, rho, u, T):
    """Returns the status (LBM_OK or LBM_ENONFINITE); other errors raise."""
    rc = load().lbm_pool_result(p, ticket, _ptr(rho), _ptr(u), _ptr(T))
    if rc not in (LBM_OK, LBM_ENONFINITE):
        _check(rc)
    return rc


def lbm_pool_stats(p):
    out = (ctypes.c_longlong * 6)()
    _check(load().lbm_pool_stats(p, out))
    keys = ("resident", "finished", "bytes_used", "bytes_budget", "tiles", "grid")
    return dict(zip(keys, list(out)))


class Pool:
    """A continuous-batching pool on the current CUDA device; its device
    memory is a torch tensor of lbm_pool_bytes (torch's allocator)."""

    def __init__(self, lattice, prec, budget_bytes, max_instances=512, bundle_steps=50, stream=None):
        import torch
        self.lattice, self.prec, self.D = lattice, prec, dim(lattice)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        cfg = make_pool_config(lattice, prec, budget_bytes, max_instances, bundle_steps,
                               stream=self.stream.cuda_stream)
        nbytes = lbm_pool_bytes(cfg)
        if nbytes == 0:
            raise LbmError(LBM_EINVAL, "invalid pool configuration")
        with torch.cuda.stream(self.stream):
            self.mem = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        cfg.device_mem, cfg.device_bytes = self.mem.data_ptr(), nbytes
        torch.cuda.synchronize()
        self.h = lbm_pool_create(cfg)
        self.bundle_steps = bundle_steps

    def close(self):
        if getattr(self, "h", None) is not None:
            lbm_pool_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, gamma, tau_f, tau_g, shape, bc, fields, steps, rho0=0.0, T0=0.0):
        grid = make_grid(shape, bc=bc, prec=self.prec, rho0=rho0, T0=T0)
        rho, u, T = (np.ascontiguousarray(a, dtype=np.float64) for a in fields)
        return lbm_pool_submit(self.h, gamma, tau_f, tau_g, grid, rho, u, T, steps)

    def instance_bytes(self, shape):
        return lbm_pool_instance_bytes(self.h, make_grid(shape, prec=self.prec))

    def run(self, bundles=1):
        lbm_pool_run(self.h, bundles)

    def sync(self):
        lbm_pool_sync(self.h)

    def poll(self, ticket):
        return lbm_pool_poll(self.h, ticket)

    def result(self, ticket, N):
        rho, u, T = np.zeros(N), np.zeros(self.D * N), np.zeros(N)
        rc = lbm_pool_result(self.h, ticket, rho, u, T)
        return rc, (rho, u.reshape(self.D, N), T)

    def stats(self):
        return lbm_pool_stats(self.h)
