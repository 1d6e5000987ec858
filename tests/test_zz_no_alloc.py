"""The allocation-free cell sort (sdm_cell_sort_noalloc) against the
allocating one (sdm_cell_sort), through the C ABI, two calls in a row.

Some callers cannot allocate device memory while they run: code being
captured into a CUDA graph, stream-ordered regions where a cudaMalloc would
synchronise the device, and services whose memory pools are sized once at
start-up.  The variant serves them from one fixed device array; this file
checks that it gives the same grouping as the allocating entry point and
that the second call is not disturbed by what the first left in the shared
scratch.  It is named to run last in a session."""
import numpy as np
import pytest

from paper_1310_1905_gb300 import sdm

pytestmark = pytest.mark.gpu


def _run(fn, torch, cell, n_cells):
    n = len(cell)
    d_cell = torch.tensor(cell, dtype=torch.int32, device="cuda")
    d_perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    d_off = torch.full((n_cells + 1,), -1, dtype=torch.int32, device="cuda")
    fn(d_cell, n_cells, d_perm, d_off)
    torch.cuda.synchronize()
    return d_perm.cpu().numpy()[:n], d_off.cpu().numpy()


def _same_grouping(a, b):
    perm_a, off_a = a
    perm_b, off_b = b
    assert np.array_equal(off_a, off_b)           # integers: exact
    for c in range(len(off_a) - 1):               # order inside a cell is free
        s = slice(off_a[c], off_a[c + 1])
        assert np.array_equal(np.sort(perm_a[s]), np.sort(perm_b[s]))


def test_noalloc_matches_allocating_sort_twice():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    # first call: the 2D case's size; second call: fewer cells and particles,
    # so stale counts from the first call would show up
    for n, n_cells in ((360000, 5625), (50001, 1001)):
        cell = rng.integers(0, n_cells, size=n).astype(np.int32)
        ref = _run(sdm.sdm_cell_sort, torch, cell, n_cells)
        got = _run(sdm.sdm_cell_sort_noalloc, torch, cell, n_cells)
        _same_grouping(got, ref)
        assert got[1][-1] == n


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    d_cell = torch.zeros(4, dtype=torch.int32, device="cuda")
    d_perm = torch.empty(4, dtype=torch.int32, device="cuda")
    d_off = torch.empty(2, dtype=torch.int32, device="cuda")
    with pytest.raises(sdm.SdmError) as e:
        sdm.sdm_cell_sort_noalloc(d_cell, (1 << 19) + 1, d_perm, d_off)
    assert e.value.status == 1 and "cells" in str(e.value)
