"""The grouping entry point for callers that cannot allocate device memory.

ltpc_group_cells_noalloc keeps its counters in a fixed device array of the
library instead of asking for scratch space.  Checked here against the
context-based grouping (ltpc_grouping) on two calls in a row with different
inputs, so the second call also shows that the shared array is cleared.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import numpy as np
import pytest

from paper_2508_06771_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_06771_gb300 import build as B
    from paper_2508_06771_gb300 import ltpc
    B.build()
    ltpc.load_library()
    return ltpc


def _reference_grouping(L, wl):
    col = L.Collider.from_workload(wl, precision=L.F64)
    col.load_workload(wl)
    cs, perm, counts = col.grouping()
    col.close()
    return cs, perm


def _same_grouping(cs_a, perm_a, cs_b, perm_b):
    assert np.array_equal(cs_a, cs_b)
    for j in range(cs_a.size - 1):
        a, b = int(cs_a[j]), int(cs_a[j + 1])
        assert np.array_equal(np.sort(perm_a[a:b]), np.sort(perm_b[a:b])), j


def test_noalloc_grouping_matches_context_grouping_twice(L):
    import torch
    cases = [W.ragged(M=300, mean_ppc=150, seed=21, shuffled=True),
             W.ragged(M=57, mean_ppc=900, seed=22, shuffled=True)]   # fewer cells than the first call
    for wl in cases:
        cell = torch.as_tensor(wl["cell"], dtype=torch.int32, device="cuda")
        cs, perm = L.group_cells_noalloc(cell, wl["M"])
        rcs, rperm = _reference_grouping(L, wl)
        _same_grouping(cs, perm, rcs, rperm)


def test_noalloc_rejects_bad_sizes_and_ids(L):
    import torch
    cell = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(L.LtpcError) as ei:
        L.group_cells_noalloc(cell, L.NOALLOC_MAX_CELLS + 1)
    assert ei.value.code == L.EINVAL
    cell[3] = 9
    with pytest.raises(L.LtpcError) as ei:
        L.group_cells_noalloc(cell, 5)
    assert ei.value.code == L.EINVAL
