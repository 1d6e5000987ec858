"""Domain decomposition of the super-droplet state across ranks: the host-side
exchange step of the multi-GPU design (one GPU per rank, contiguous slabs of
cells in x).  Coalescence, condensation and the diagnostics are cell-local;
only advection and sedimentation move super-droplets across a slab boundary,
so a step needs one exchange of the leavers between neighbouring slabs, after
the transport and before the counting sort.

This module holds that exchange on the host over torch.distributed (gloo or
nccl): which rank owns a position, the packing of the leavers into two
blocks (the floating-point attributes as float64, multiplicities and ids as
int64, so that every integer travels exactly), the swap with the two
neighbours and the unpacking.  The library's sdm_export_leavers and
sdm_import move the super-droplets between a context and these blocks.
"""
from __future__ import annotations

import numpy as np

FLOATS = ("rw2", "rd3", "kappa", "x", "y", "z")
INTS = ("N", "uid")
ATTRS = INTS + FLOATS


def slab_of(x: np.ndarray, X: float, world: int) -> np.ndarray:
    """Owner rank of each x position in [0, X): equal slabs in x."""
    r = np.floor(np.asarray(x, np.float64) / X * world).astype(np.int64)
    return np.clip(r, 0, world - 1)


def pack(state: dict, sel: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """The selected super-droplets as an (n, 2) int64 block (N, uid) and an
    (n, 6) float64 block (r_w^2, r_d^3, kappa, x, y, z); absent attributes
    travel as zeros.  Multiplicities up to 2^63 - 1 travel exactly."""
    n = int(np.count_nonzero(sel))
    ints = np.zeros((n, len(INTS)), np.int64)
    floats = np.zeros((n, len(FLOATS)), np.float64)
    for k, a in enumerate(INTS):
        if a in state:
            v = np.asarray(state[a])[sel]
            assert n == 0 or int(v.max()) < 2 ** 63, "integers must fit int64"
            ints[:, k] = v.astype(np.int64)
    for k, a in enumerate(FLOATS):
        if a in state:
            floats[:, k] = np.asarray(state[a])[sel]
    return ints, floats


def unpack(ints: np.ndarray, floats: np.ndarray, like: dict) -> dict:
    """Attributes from packed blocks, in the dtypes of ``like``."""
    out = {a: ints[:, k].astype(np.asarray(like[a]).dtype) for k, a in enumerate(INTS) if a in like}
    out.update({a: floats[:, k].astype(np.asarray(like[a]).dtype) for k, a in enumerate(FLOATS) if a in like})
    return out


def concat(a: dict, b: dict) -> dict:
    return {k: np.concatenate([a[k], b[k]]) for k in a}


def exchange(state: dict, X: float, group=None) -> tuple[dict, int, int]:
    """Send every super-droplet whose x left this rank's slab to its owner
    (a neighbour: a transport step moves a super-droplet by less than one
    slab) and append the ones received.  Returns the new state and the
    counts sent and received.  Collective over the group: every rank calls
    it once per step."""
    import torch
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    if world == 1:
        return state, 0, 0
    owner = slab_of(state["x"], X, world)
    left, right = (rank - 1) % world, (rank + 1) % world
    stay = owner == rank
    to_left = (owner == left) & ~stay
    to_right = (owner == right) & ~stay & ~to_left
    assert np.all(stay | to_left | to_right), "a super-droplet moved by more than one slab in one step"
    recv = []
    for dst, sel in ((left, to_left), (right, to_right)):
        src = right if dst == left else left
        ints, floats = (torch.from_numpy(b) for b in pack(state, sel))
        n_out = torch.tensor([ints.shape[0]], dtype=torch.int64)
        n_in = torch.zeros(1, dtype=torch.int64)
        # sizes first, then the blocks; paired send/recv in rank order avoids a deadlock with gloo
        ops = [dist.P2POp(dist.isend, n_out, dst, group), dist.P2POp(dist.irecv, n_in, src, group)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        m = int(n_in.item())
        ibuf = torch.empty((m, len(INTS)), dtype=torch.int64)
        fbuf = torch.empty((m, len(FLOATS)), dtype=torch.float64)
        ops = []
        if ints.shape[0]:
            ops += [dist.P2POp(dist.isend, ints, dst, group), dist.P2POp(dist.isend, floats, dst, group)]
        if m:
            ops += [dist.P2POp(dist.irecv, ibuf, src, group), dist.P2POp(dist.irecv, fbuf, src, group)]
        for r in dist.batch_isend_irecv(ops) if ops else []:
            r.wait()
        recv.append((ibuf.numpy(), fbuf.numpy()))
    kept = {k: np.asarray(v)[stay] for k, v in state.items()}
    for ib, fb in recv:
        kept = concat(kept, unpack(ib, fb, state))
    return kept, int(np.count_nonzero(~stay)), int(sum(ib.shape[0] for ib, _ in recv))
