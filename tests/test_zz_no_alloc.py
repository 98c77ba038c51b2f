"""The grouping entry point for callers that cannot allocate device memory.

ltpc_group_cells_noalloc keeps its counters in a fixed device array of the
library instead of asking for scratch space.  Checked here against the
context-based grouping (ltpc_grouping) and against the oracle's grouping
(counts, offsets, and each cell's set of ids) on two calls in a row with
different inputs, so the second call also shows that the shared array is
cleared; and with out-of-range ids in an array long enough that every thread
runs many loop iterations.  This file sorts last so that a run stopping at the
first failure has already run every other test.
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


def _matches_oracle(orc, cell, M, cs, perm, valid=None):
    idx = np.arange(cell.size) if valid is None else np.nonzero(valid)[0]
    ocounts, ocs, operm = orc.group(cell[idx], M)
    assert np.array_equal(cs.astype(np.uint64), ocs)
    assert np.array_equal(np.diff(cs.astype(np.int64)), ocounts.astype(np.int64))
    for j in range(M):
        a, b = int(ocs[j]), int(ocs[j + 1])
        assert np.array_equal(np.sort(perm[a:b]), idx[operm[a:b]]), j


def test_noalloc_grouping_matches_context_grouping_twice(L, orc):
    import torch
    cases = [W.ragged(M=300, mean_ppc=150, seed=21, shuffled=True),
             W.ragged(M=57, mean_ppc=900, seed=22, shuffled=True)]   # fewer cells than the first call
    for wl in cases:
        cell = torch.as_tensor(wl["cell"], dtype=torch.int32, device="cuda")
        cs, perm = L.group_cells_noalloc(cell, wl["M"])
        rcs, rperm = _reference_grouping(L, wl)
        _same_grouping(cs, perm, rcs, rperm)
        _matches_oracle(orc, wl["cell"], wl["M"], cs, perm)


def test_noalloc_bad_ids_many_loop_iterations(L, orc):
    """Two million ids (several grid-stride iterations per thread) with out-of-range ids
    scattered through them: EINVAL, and then a clean call groups correctly."""
    import torch
    rng = np.random.default_rng(77)
    M, n = 1000, 2_000_000
    cell = rng.integers(0, M, n).astype(np.int32)
    bad_at = np.array([1, 33, 64, 999_999, 1_234_567, n - 1])
    bad = cell.copy()
    bad[bad_at] = [-1, M, -9, M + 5, 2 ** 31 - 1, M]
    with pytest.raises(L.LtpcError) as ei:
        L.group_cells_noalloc(torch.as_tensor(bad, device="cuda"), M)
    assert ei.value.code == L.EINVAL
    cs, perm = L.group_cells_noalloc(torch.as_tensor(cell, device="cuda"), M)
    _matches_oracle(orc, cell, M, cs, perm)


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
