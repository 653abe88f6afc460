"""pm_cell_sort_static: the cell sort for callers that cannot allocate device memory.

Some hosts hand all GPU memory to their own fixed pool, or drive the library from
plain C / Fortran with no device allocator; they cannot provide the scratch buffer
pm_cell_sort asks for.  pm_cell_sort_static keeps that scratch in a fixed array
inside the library instead.  This test checks, through the C ABI, that it returns
exactly what pm_cell_sort returns (and what the oracle's cell keys and stable order are), on two calls in a row with different sizes (so
stale contents of the shared array would show), and that it refuses meshes above
its 64^3-cell limit.  It lives in its own file so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import inputs
from oracle import cic
from tests.gpu_util import lib, to_dev, to_host, torch

pytestmark = pytest.mark.gpu
FP32, FP64 = 0, 1


def _both(pm, xs, count, prec, n):
    keys_a = torch.empty(count, dtype=torch.int32, device="cuda")
    order_a = torch.empty(count, dtype=torch.int32, device="cuda")
    scratch = torch.empty(pm.pm_cell_sort_scratch_size(count, n), dtype=torch.uint8, device="cuda")
    pm.pm_cell_sort(to_dev(xs), count, prec, n, keys_a, order_a, scratch)
    keys_b = torch.full((count,), -1, dtype=torch.int32, device="cuda")
    order_b = torch.full((count,), -1, dtype=torch.int32, device="cuda")
    pm.pm_cell_sort_static(to_dev(xs), count, prec, n, keys_b, order_b)
    torch.cuda.synchronize()
    return (to_host(keys_a), to_host(order_a)), (to_host(keys_b), to_host(order_b))


def test_static_cell_sort_matches_scratch_version_on_consecutive_calls():
    pm = lib()
    cases = [(inputs.lattice_order_ticks(81, 32, 1.5, n_mesh=64), FP32, 64),
             (inputs.ticks_to_fractions(inputs.clustered_ticks(82, 20_001)), FP64, 16)]
    for xs, prec, n in cases:
        count = xs.shape[1]
        (ka, oa), (kb, ob) = _both(pm, xs, count, prec, n)
        np.testing.assert_array_equal(kb, ka)
        np.testing.assert_array_equal(ob, oa)
        # and both equal the oracle's cell keys and stable order, bit for bit
        np.testing.assert_array_equal(kb.astype(np.int64), cic.cell_keys(xs, n))
        np.testing.assert_array_equal(ob.astype(np.int64), cic.cell_order(xs, n))


def test_static_cell_sort_refuses_meshes_above_its_limit():
    pm = lib()
    x = to_dev(inputs.uniform_ticks(83, 100))
    keys = torch.empty(100, dtype=torch.int32, device="cuda")
    with pytest.raises(pm.PMError) as e:
        pm.pm_cell_sort_static(x, 100, FP32, 128, keys, None)
    assert e.value.status == 1
