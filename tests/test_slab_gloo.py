"""Slab decomposition along the slowest axis (lbm_slab_plan / pack / unpack)
on gloo CPU ranks.  Each rank steps its slab -- owned layers plus 3 ghost
layers per side -- with the FP64 oracle as the stepper, and before every
step exchanges with its neighbours exactly the messages the plan packs: the
populations of its 3 boundary layers that cross each face.  After the run
the owned layers of all ranks, stitched together, must equal the
single-domain oracle bitwise (every owned cell sees the same pulled values,
so it does the same arithmetic), for periodic and zero-gradient split axes,
2D and 3D, and world sizes 1 (periodic self-exchange), 2 and 3."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

P, ZG = 0, 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fields(shape, seed):
    import lbm_inputs as li
    N = int(np.prod(shape))
    return li.random_fields(N, len(shape), seed=seed)


def _layer_view(q, shape):
    """Flat field -> array indexed [layer along the split axis][rest]."""
    D = len(shape)
    if D == 2:
        return q.reshape(shape[1], shape[0])
    return q.reshape(shape[2], shape[1] * shape[0])


def _orders(lattice):
    """Index maps between the oracle's velocity order and the library's:
    lib_of_ora[i] is the library index of the oracle's velocity i."""
    import ctypes

    from oracle import oracle as ora
    from paper_1608_06345_gb300 import lbm
    c_ora, _, _ = ora.lattice_info(lattice)
    D = c_ora.shape[1]
    q = ctypes.c_int()
    c = np.zeros(107 * D, dtype=np.int32)
    assert lbm.load().lbm_lattice_table(lattice, ctypes.byref(q), c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                        None, None) == 0
    c_lib = c[:q.value * D].reshape(q.value, D)
    idx = {tuple(v): k for k, v in enumerate(c_lib)}
    return np.array([idx[tuple(v)] for v in c_ora])


def _worker(rank, world, port, lattice, shape, bc_axis, steps, seed, out):
    import torch
    import torch.distributed as dist

    from oracle import oracle as ora
    from paper_1608_06345_gb300 import lbm
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ora.set_threads(1)
    D = len(shape)
    n = tuple(shape) + (1,) * (3 - D)
    s = lbm.lbm_slab_plan(lattice, n, bc_axis == P, world, rank)
    local = tuple(s.local_n[a] for a in range(D))
    lc = s.layer_cells
    # initial fields of the local grid: global layers begin-3 .. end+2
    # (wrapped on a periodic axis, clamped at zero-gradient ends); the ghost
    # values are replaced by the first exchange anyway
    rho, u, T = _fields(shape, seed)
    L = shape[-1]
    layers = np.arange(s.begin - 3, s.end + 3)
    layers = layers % L if bc_axis == P else np.clip(layers, 0, L - 1)
    take = lambda q: _layer_view(q, shape)[layers].reshape(-1)
    f_loc = (take(rho), np.stack([take(c) for c in u]), take(T))
    # the other axes as in the single domain (periodic); the split axis of
    # the local grid zero-gradient: its ghost layers are refreshed each step
    bc = (P,) * (D - 1) + (ZG,)
    o = ora.Oracle(lattice, 1.4, 0.6, 0.7, local, bc=bc)
    o.init(*f_loc)
    lib_of_ora = _orders(lattice)
    Q = len(lib_of_ora)
    Nloc = int(np.prod(local))
    msg = s.msg_values
    for _ in range(steps):
        g, h = o.get_pops()
        state = np.zeros((2 * Q, Nloc))
        state[lib_of_ora] = g
        state[Q + lib_of_ora] = h
        to_lo, to_hi = np.zeros(msg), np.zeros(msg)
        lbm.lbm_slab_pack(s, state, Nloc, to_lo, to_hi)
        from_lo = np.zeros(msg) if s.lo >= 0 else None
        from_hi = np.zeros(msg) if s.hi >= 0 else None
        if s.lo == rank:  # one periodic slab: its own boundary layers are its ghosts
            from_lo[:], from_hi[:] = to_hi, to_lo
        else:
            reqs = []
            # tag 0: a message travelling up (to_hi -> the upper rank's
            # from_lo), tag 1: travelling down (to_lo -> the lower rank's from_hi)
            if s.hi >= 0:
                reqs.append(dist.isend(torch.from_numpy(to_hi), dst=s.hi, tag=0))
            if s.lo >= 0:
                reqs.append(dist.isend(torch.from_numpy(to_lo), dst=s.lo, tag=1))
            if s.lo >= 0:
                dist.recv(torch.from_numpy(from_lo), src=s.lo, tag=0)
            if s.hi >= 0:
                dist.recv(torch.from_numpy(from_hi), src=s.hi, tag=1)
            for r in reqs:
                r.wait()
        lbm.lbm_slab_unpack(s, state, Nloc, from_lo, from_hi)
        o.set_pops(state[lib_of_ora], state[Q + lib_of_ora])
        o.step(1)
    rho, u, T = o.moments()
    o.close()
    own = slice(3 * lc, (3 + s.end - s.begin) * lc)
    out.put((rank, s.begin, s.end, rho[own], u[:, own], T[own]))
    dist.barrier()
    dist.destroy_process_group()


def _single_domain(lattice, shape, bc_axis, steps, seed):
    from oracle import oracle as ora
    D = len(shape)
    bc = (P,) * (D - 1) + (bc_axis,)
    o = ora.Oracle(lattice, 1.4, 0.6, 0.7, shape, bc=bc)
    o.init(*_fields(shape, seed))
    o.step(steps)
    res = o.moments()
    o.close()
    return res


CASES = [
    # lattice, shape, split-axis boundary, world size
    (0, (20, 12), P, 2),
    (0, (17, 11), ZG, 3),
    (0, (9, 8), P, 1),
    (1, (6, 5, 9), P, 3),
    (1, (5, 4, 8), ZG, 2),
]


@pytest.mark.parametrize("lattice,shape,bc_axis,world", CASES)
def test_slabs_stitch_to_the_single_domain(lattice, shape, bc_axis, world):
    steps, seed = 6, 31
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, lattice, shape, bc_axis, steps, seed, q))
             for r in range(world)]
    for p in procs:
        p.start()
    parts = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    rho, u, T = _single_domain(lattice, shape, bc_axis, steps, seed)
    D = len(shape)
    lc = int(np.prod(shape[:-1]))
    for rank, b, e, r_, u_, T_ in parts:
        sl = slice(b * lc, e * lc)
        assert np.array_equal(r_, rho[sl]), rank
        assert np.array_equal(T_, T[sl]), rank
        assert np.array_equal(u_, u[:, sl]), rank
    assert sum(e - b for _, b, e, *_ in parts) == shape[-1]


def test_plan_rejects_thin_slabs_and_bad_ranks():
    from paper_1608_06345_gb300 import lbm
    with pytest.raises(lbm.LbmError):
        lbm.lbm_slab_plan(0, (10, 8, 1), True, 3, 0)   # 8 layers over 3 ranks: a slab of 2
    with pytest.raises(lbm.LbmError):
        lbm.lbm_slab_plan(0, (10, 9, 1), True, 3, 3)   # rank out of range
    from oracle import oracle as ora
    s = lbm.lbm_slab_plan(1, (4, 5, 12), False, 2, 1)
    assert (s.begin, s.end, s.lo, s.hi, s.layer_cells) == (6, 12, 0, -1, 20)
    assert tuple(s.local_n) == (4, 5, 12)
    # a message carries, per layer cell, g and h of the velocities with
    # c_z >= 1, >= 2 and >= 3 (counted on the oracle's own velocity set)
    c, _, _ = ora.lattice_info(ora.D3Q107)
    assert s.msg_values == 2 * 20 * sum(int(np.sum(c[:, 2] >= k)) for k in (1, 2, 3))
