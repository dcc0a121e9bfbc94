"""Host logic of the slab decomposition (no GPU): the slab plan (sizes,
neighbours, periodic wrap, the minimum of H cells per slab) and the halo
exchange through torch.distributed with the gloo backend on host tensors,
world sizes 2 and 3, periodic and bounded.  Every rank holds its slab of one
seeded global state; after the exchange each halo must equal the planes the
undivided grid has there.  Rendezvous on 127.0.0.1."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import paper_2109_14340_gb300 as T  # noqa: E402


def test_slab_plan():
    plan = T.slab_plan(37, 3, 5, False)
    assert [(a, b) for a, b, _, _ in plan] == [(0, 13), (13, 25), (25, 37)]
    assert [(lo, hi) for _, _, lo, hi in plan] == [(None, 1), (0, 2), (1, None)]
    plan = T.slab_plan(36, 2, 5, True)
    assert [(lo, hi) for _, _, lo, hi in plan] == [(1, 1), (0, 0)]
    assert [(lo, hi) for _, _, lo, hi in T.slab_plan(40, 4, 4, True)] == \
        [(3, 1), (0, 2), (1, 3), (2, 0)]
    for n, parts, H in ((256, 8, 5), (100, 7, 6), (64, 16, 4)):
        plan = T.slab_plan(n, parts, H, True)
        sizes = [b - a for a, b, _, _ in plan]
        assert sum(sizes) == n and max(sizes) - min(sizes) <= 1 and min(sizes) >= H
        assert all(plan[k][1] == plan[k + 1][0] for k in range(parts - 1))
    with pytest.raises(ValueError):
        T.slab_plan(9, 2, 5, True)              # a slab smaller than the halo


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


NC, NZ, M, H = 5, 23, 6, 5          # components, slab-axis cells, cells per plane, halo


def global_state():
    g = np.random.Generator(np.random.PCG64(777))
    return torch.from_numpy(g.standard_normal((NC, NZ * M)))


def _rank(rank, world, port, periodic, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import paper_2109_14340_gb300 as T
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        plan = T.slab_plan(NZ, world, H, periodic)
        a0, a1, lo, hi = plan[rank]
        Ug = global_state()
        U = Ug[:, a0 * M:a1 * M].contiguous()
        hl = torch.full((NC, H * M), np.nan, dtype=torch.float64)
        hh = torch.full((NC, H * M), np.nan, dtype=torch.float64)
        T.exchange_halos_dist(U, a1 - a0, M, H, hl, hh, lo, hi)
        ok = True
        full = Ug.view(NC, NZ, M)
        if lo is not None:
            planes = [(a0 - H + q) % NZ for q in range(H)]
            ok &= torch.equal(hl.view(NC, H, M), full[:, planes, :])
        else:
            ok &= bool(torch.isnan(hl).all())
        if hi is not None:
            planes = [(a1 + q) % NZ for q in range(H)]
            ok &= torch.equal(hh.view(NC, H, M), full[:, planes, :])
        else:
            ok &= bool(torch.isnan(hh).all())
        out.put((rank, bool(ok)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, True), (2, False), (3, True), (3, False)])
def test_halo_exchange_gloo(world, periodic):
    port = free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, periodic, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [r for r, _ in res] == list(range(world))
    assert all(ok for _, ok in res), res
