"""The standalone counting sort by cell (regrouping step) through the C ABI,
against a numpy reference: offsets exact, each cell's set of particles
exact (the order inside a cell is unspecified)."""
import numpy as np
import pytest

from paper_1310_1905_gb300 import sdm

pytestmark = pytest.mark.gpu


def reference(cell, n_cells):
    counts = np.bincount(cell, minlength=n_cells)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return offsets


def check(cell, n_cells, perm, offsets):
    ref_off = reference(cell, n_cells)
    assert np.array_equal(offsets.astype(np.int64), ref_off)
    order = np.argsort(cell, kind="stable")
    for c in np.nonzero(np.diff(ref_off))[0]:
        got = np.sort(perm[ref_off[c]:ref_off[c + 1]])
        assert np.array_equal(got, order[ref_off[c]:ref_off[c + 1]])


@pytest.mark.parametrize("n,n_cells", [(0, 5), (1, 1), (1000, 7), (360000, 5625), (100003, 2049)])
def test_cell_sort(n, n_cells):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(n + n_cells)
    cell = rng.integers(0, n_cells, size=n).astype(np.int32)
    d_cell = torch.tensor(cell, device="cuda")
    d_perm = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    d_off = torch.empty(n_cells + 1, dtype=torch.int32, device="cuda")
    sdm.sdm_cell_sort(d_cell[:n] if n else d_cell, n_cells, d_perm, d_off)
    check(cell, n_cells, d_perm.cpu().numpy()[:n], d_off.cpu().numpy())


def test_cell_sort_rejects_out_of_range():
    torch = pytest.importorskip("torch")
    d_cell = torch.tensor([0, 3, 9], dtype=torch.int32, device="cuda")
    d_perm = torch.empty(3, dtype=torch.int32, device="cuda")
    d_off = torch.empty(5, dtype=torch.int32, device="cuda")
    with pytest.raises(sdm.SdmError) as e:
        sdm.sdm_cell_sort(d_cell, 4, d_perm, d_off)
    assert e.value.status == 1
