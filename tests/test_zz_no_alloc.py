"""lbm_conserved_noalloc: conservation totals of a raw device state, computed
with a static scratch array instead of any allocation.

Who needs it: callers that cannot call cudaMalloc when they want the totals
(a serving pool that has reserved the whole device budget, or code that keeps
populations in its own arena without a library instance).  The test checks
the new entry point through the C ABI against lbm_conserved on the same
state, within the 1e-13 relative tolerance of the other conservation tests,
on two calls in a row (the second after more steps, so the shared scratch is
reused).  This file sorts last so that a run stopping at the first failure
has already run every other test; it also passes on its own in a fresh
process."""
import numpy as np
import pytest

import lbm_inputs as li

pytestmark = pytest.mark.gpu

TOL = 1e-13


def device_state(solver):
    """The solver's raw state (layout of lbm_get_state) copied into a fresh
    CUDA tensor: the caller's own device buffer."""
    import torch

    from paper_1608_06345_gb300 import lbm
    raw = np.zeros(lbm.lbm_raw_state_bytes(solver.h), dtype=np.uint8)
    lbm.lbm_get_state(solver.h, raw)
    return torch.from_numpy(raw).cuda()


# (300, 50) spans 4 blocks of 4096 cells with a partial last block; 4096^2 is
# the maximum, 4096 full blocks
@pytest.mark.parametrize("lat,shape,prec", [(0, (300, 7), 0), (1, (40, 6, 5), 0), (0, (257, 9), 1),
                                            (0, (300, 7), 2), (1, (20, 6, 5), 3), (0, (300, 50), 1),
                                            (1, (30, 20, 25), 0), (0, (4096, 4096), 2)])
def test_noalloc_totals_match_lbm_conserved_twice(lat, shape, prec):
    import torch

    from paper_1608_06345_gb300 import lbm
    D = len(shape)
    N = int(np.prod(shape))
    gamma = 1.4
    s = lbm.Solver(lat, gamma, 0.6, 0.6, shape, prec=prec, rho0=0.9, T0=1.1)
    s.init(*li.random_fields(N, D, seed=N))
    stream = torch.cuda.current_stream().cuda_stream
    for steps in (3, 4):
        s.step(steps)
        ref = s.conserved()
        state = device_state(s)
        torch.cuda.synchronize()
        got = lbm.lbm_conserved_noalloc(lat, prec, gamma, state, N, N, stream=stream, rho0=0.9, T0=1.1)
        scale = np.array([abs(ref[0])] * (1 + D) + [abs(ref[-1])])
        assert np.all(np.abs(got - ref) <= TOL * scale), (got, ref)


def test_noalloc_rejects_sizes_above_its_maximum():
    from paper_1608_06345_gb300 import lbm
    too_many = 4096 * 4096 + 1
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_conserved_noalloc(0, 1, 1.4, 1 << 20, too_many, too_many)
    assert ei.value.code == lbm.LBM_EINVAL
    assert "maximum" in str(ei.value)


def _state_and_args():
    from paper_1608_06345_gb300 import lbm
    s = lbm.Solver(0, 1.4, 0.6, 0.6, (64, 4), prec=1)
    s.init(*li.random_fields(256, 2, seed=1))
    return s, device_state(s)


def test_noalloc_rejects_a_misaligned_state():
    """A state pointer off its 4-byte storage word is refused on the host,
    before anything is launched."""
    import torch

    from paper_1608_06345_gb300 import lbm
    s, state = _state_and_args()
    torch.cuda.synchronize()
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_conserved_noalloc(0, 1, 1.4, state.data_ptr() + 2, 256, 256)
    assert ei.value.code == lbm.LBM_EINVAL and "aligned" in str(ei.value)


def test_noalloc_rejects_host_memory():
    """A host pointer is refused on the host (cudaPointerGetAttributes); the
    host buffer covers the whole extent all the same."""
    from paper_1608_06345_gb300 import lbm
    host = np.zeros(2 * 37 * 256, dtype=np.float32)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_conserved_noalloc(0, 1, 1.4, host.ctypes.data, 256, 256)
    assert ei.value.code == lbm.LBM_EINVAL


def test_binding_rejects_a_short_tensor():
    import torch

    from paper_1608_06345_gb300 import lbm
    short = torch.zeros(2 * 37 * 256 - 1, dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_conserved_noalloc(0, 1, 1.4, short, 256, 256)
    assert ei.value.code == lbm.LBM_EINVAL

