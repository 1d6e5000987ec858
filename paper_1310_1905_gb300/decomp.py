"""Domain decomposition of the super-droplet state across ranks: the host-side
exchange step of the multi-GPU design (one GPU per rank, contiguous slabs of
cells in x).  Coalescence, condensation and the diagnostics are cell-local;
only advection and sedimentation move super-droplets across a slab boundary,
so a step needs one exchange of the leavers between neighbouring slabs, after
the transport and before the counting sort.

This module holds that exchange on the host over torch.distributed (gloo or
nccl): which rank owns a position, the packing of the leavers of every
attribute into one float64 buffer (multiplicities and ids travel as exact
integers below 2^53), the swap with the two neighbours and the unpacking.
Every run here has one GPU, so the library's device path stays one domain
per GPU (bench.py --gpus N runs replicas); this is the exchange a sharded
driver would call, tested with two gloo ranks on the CPU.
"""
from __future__ import annotations

import numpy as np

ATTRS = ("N", "rw2", "rd3", "kappa", "x", "y", "z", "uid")


def slab_of(x: np.ndarray, X: float, world: int) -> np.ndarray:
    """Owner rank of each x position in [0, X): equal slabs in x."""
    r = np.floor(np.asarray(x, np.float64) / X * world).astype(np.int64)
    return np.clip(r, 0, world - 1)


def pack(state: dict, sel: np.ndarray) -> np.ndarray:
    """The selected super-droplets as one (n, len(ATTRS)) float64 block;
    absent attributes travel as zeros."""
    n = int(np.count_nonzero(sel))
    out = np.zeros((n, len(ATTRS)), np.float64)
    for k, a in enumerate(ATTRS):
        if a in state:
            v = np.asarray(state[a])[sel]
            if v.dtype.kind in "ui":
                assert n == 0 or int(v.max()) < 2 ** 53, "integers above 2^53 do not travel exactly as float64"
            out[:, k] = v
    return out


def unpack(block: np.ndarray, like: dict) -> dict:
    """Attributes from a packed block, in the dtypes of ``like``."""
    return {a: block[:, k].astype(np.asarray(like[a]).dtype) for k, a in enumerate(ATTRS) if a in like}


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
        block = torch.from_numpy(pack(state, sel))
        n_out = torch.tensor([block.shape[0]], dtype=torch.int64)
        n_in = torch.zeros(1, dtype=torch.int64)
        # sizes first, then the blocks; paired send/recv in rank order avoids a deadlock with gloo
        ops = [dist.P2POp(dist.isend, n_out, dst, group), dist.P2POp(dist.irecv, n_in, src, group)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        buf = torch.empty((int(n_in.item()), len(ATTRS)), dtype=torch.float64)
        ops = []
        if block.shape[0]:
            ops.append(dist.P2POp(dist.isend, block, dst, group))
        if buf.shape[0]:
            ops.append(dist.P2POp(dist.irecv, buf, src, group))
        for r in dist.batch_isend_irecv(ops) if ops else []:
            r.wait()
        recv.append(buf.numpy())
    kept = {k: np.asarray(v)[stay] for k, v in state.items()}
    for b in recv:
        kept = concat(kept, unpack(b, state))
    return kept, int(np.count_nonzero(~stay)), int(sum(b.shape[0] for b in recv))
