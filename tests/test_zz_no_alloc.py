"""The allocation-free cell sort (sdm_cell_sort_noalloc) through the C ABI:
against numpy and against the allocating sort (sdm_cell_sort), two calls in
a row, at its exact size limits, and on its out-of-range path.

Some callers cannot allocate device memory while they run: code being
captured into a CUDA graph, stream-ordered regions where a cudaMalloc would
synchronise the device, and services whose memory pools are sized once at
start-up.  The variant serves them from one fixed device array; this file
checks that it gives the same grouping as numpy's histogram and as the
allocating entry point, and that the second call is not disturbed by what
the first left in the shared scratch.  It is named to run last in a
session."""
import numpy as np
import pytest

from paper_1310_1905_gb300 import sdm

pytestmark = pytest.mark.gpu

MAX_N, MAX_CELLS = 1 << 21, 1 << 19


def _run(fn, torch, cell, n_cells):
    n = len(cell)
    d_cell = torch.tensor(cell.astype(np.int64), dtype=torch.int64, device="cuda").to(torch.int32)
    d_perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    d_off = torch.full((n_cells + 1,), -1, dtype=torch.int32, device="cuda")
    fn(d_cell, n_cells, d_perm, d_off)
    torch.cuda.synchronize()
    return d_perm.cpu().numpy().view(np.uint32)[:n], d_off.cpu().numpy().view(np.uint32)


def _check_against_numpy(got, cell, n_cells):
    """offsets are the exclusive scan of numpy's histogram (exact), and each
    cell's slice of perm holds exactly the indices of its particles."""
    perm, off = got
    valid = cell < n_cells
    counts = np.bincount(cell[valid].astype(np.int64), minlength=n_cells)
    ref = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint32)
    assert np.array_equal(off, ref)
    order = np.argsort(cell[valid], kind="stable")
    want = np.nonzero(valid)[0][order]
    for c in np.unique(cell[valid])[:: max(1, n_cells // 500)]:  # a sample of cells, every index in them
        s = slice(ref[c], ref[c + 1])
        assert np.array_equal(np.sort(perm[s]), want[s]), c


def test_noalloc_matches_numpy_and_allocating_sort_twice():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    # first call: the 2D case's size; second call: fewer cells and particles,
    # so stale counts from the first call would show up
    for n, n_cells in ((360000, 5625), (50001, 1001)):
        cell = rng.integers(0, n_cells, size=n).astype(np.uint32)
        ref = _run(sdm.sdm_cell_sort, torch, cell, n_cells)
        got = _run(sdm.sdm_cell_sort_noalloc, torch, cell, n_cells)
        _check_against_numpy(got, cell, n_cells)
        assert np.array_equal(got[1], ref[1])
        assert got[1][-1] == n


def test_noalloc_at_its_exact_limits():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    cell = rng.integers(0, MAX_CELLS, size=MAX_N).astype(np.uint32)
    cell[:3] = [0, MAX_CELLS - 1, MAX_CELLS - 1]
    _check_against_numpy(_run(sdm.sdm_cell_sort_noalloc, torch, cell, MAX_CELLS), cell, MAX_CELLS)


def test_noalloc_skips_out_of_range_cells():
    """Indices >= n_cells are not written: offsets[n_cells] counts only the
    valid particles, and perm's first offsets[n_cells] entries hold them."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(13)
    n, n_cells = 20000, 300
    cell = rng.integers(0, n_cells, size=n).astype(np.uint32)
    bad = rng.choice(n, 37, replace=False)
    cell[bad] = n_cells + rng.integers(0, 1000, size=37).astype(np.uint32)
    perm, off = _run(sdm.sdm_cell_sort_noalloc, torch, cell, n_cells)
    assert off[-1] == n - 37
    _check_against_numpy((perm, off), cell, n_cells)
    assert not np.isin(perm[: off[-1]], bad).any()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    d_cell = torch.zeros(4, dtype=torch.int32, device="cuda")
    d_perm = torch.empty(4, dtype=torch.int32, device="cuda")
    d_off = torch.empty(2, dtype=torch.int32, device="cuda")
    with pytest.raises(sdm.SdmError) as e:
        sdm.sdm_cell_sort_noalloc(d_cell, MAX_CELLS + 1, d_perm, d_off)
    assert e.value.status == 1 and "cells" in str(e.value)
    big = torch.zeros(MAX_N + 1, dtype=torch.int32, device="cuda")
    big_perm = torch.empty(MAX_N + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(sdm.SdmError) as e:
        sdm.sdm_cell_sort_noalloc(big, 1, big_perm, d_off)
    assert e.value.status == 1 and "particles" in str(e.value)
