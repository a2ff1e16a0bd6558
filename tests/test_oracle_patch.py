"""The full-size parity tests (tests/test_gpu_fullsize.py) compare the GPU
with the oracle run on a patch of the grid: after K steps the central cells
of a patch that reaches 3K cells beyond them depend on nothing outside it
(|c_i| <= 3 per axis).  This checks that construction on the CPU against the
oracle run on the whole periodic grid: the central cells must agree bitwise,
since each cell's arithmetic sees the same pulled values in both runs."""
import numpy as np
import pytest

import lbm_inputs as li
from oracle import oracle as ora
from tests.test_gpu_fullsize import gpu_block, oracle_patch


@pytest.mark.parametrize("lat,shape,K,M", [(0, (40, 36), 4, 5), (1, (20, 18, 22), 2, 3)])
def test_patch_equals_the_whole_grid(lat, shape, K, M):
    D = len(shape)
    fields = li.fourier_fields(shape, seed_u=3, seed_rho=4, seed_T=5 if D == 3 else None, kmax=2)
    o = ora.Oracle(lat, 1.4, 0.6, 0.7, shape, bc=(ora.PERIODIC,) * 3)
    o.init(*fields)
    o.step(K)
    whole = gpu_block(shape, o.moments(), K, M)
    o.close()
    part = oracle_patch(lat, shape, fields, 1.4, 0.6, 0.7, K, M)
    for a, b in zip(whole, part):
        assert np.array_equal(a, b)
