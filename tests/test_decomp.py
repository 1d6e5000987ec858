"""The exchange step of the multi-GPU design (paper_1310_1905_gb300.decomp)
on CPU gloo ranks: x-slabs per rank, a transport step that moves
super-droplets by less than half a slab (periodic in x), then one exchange;
afterwards every super-droplet sits on the rank that owns its x, none is lost
or duplicated, and every attribute arrives unchanged."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

X, Z, N_SD = 1500.0, 1500.0, 4000


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def global_state(seed=0):
    rng = np.random.default_rng(seed)
    # multiplicities up to 2^62: above 2^53 they would not travel exactly as float64
    return dict(N=rng.integers(1, 2 ** 62, N_SD, dtype=np.int64).astype(np.uint64),
                rw2=rng.uniform(1e-14, 1e-8, N_SD), rd3=rng.uniform(1e-24, 1e-21, N_SD),
                kappa=np.full(N_SD, 0.61), x=rng.uniform(0, X, N_SD), z=rng.uniform(0, Z, N_SD),
                uid=np.arange(N_SD, dtype=np.uint32))


def moved(state, world, seed=1):
    rng = np.random.default_rng(seed)
    out = dict(state)
    out["x"] = np.mod(state["x"] + rng.uniform(-0.5, 0.5, N_SD) * X / world, X)
    return out


def _rank(rank, world, port, q):
    import torch.distributed as dist
    from paper_1310_1905_gb300 import decomp
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = global_state()
        mine = decomp.slab_of(g["x"], X, world) == rank
        local = moved({k: v for k, v in g.items()}, world)
        local = {k: v[mine] for k, v in local.items()}
        new, sent, got = decomp.exchange(local, X)
        q.put((rank, {k: v.copy() for k, v in new.items()}, sent, got))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_routes_every_super_droplet_to_its_owner(world):
    import torch.multiprocessing as mp
    from paper_1310_1905_gb300 import decomp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = moved(global_state(), world)
    seen = np.zeros(N_SD, np.int64)
    total_sent = total_got = 0
    for rank, st, sent, got in res:
        total_sent += sent
        total_got += got
        assert np.all(decomp.slab_of(st["x"], X, world) == rank)
        uid = st["uid"].astype(np.int64)
        seen[uid] += 1
        for k in ("N", "rw2", "rd3", "kappa", "x", "z"):
            assert np.array_equal(st[k], ref[k][uid]), k
    assert np.all(seen == 1)
    assert total_sent == total_got > 0
