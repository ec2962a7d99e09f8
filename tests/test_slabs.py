"""Row-slab decomposition, host side, on CPU: partition, routing, assembly, and the
cut-row exchange and gradient sum between gloo ranks (2 and 3 processes, periodic or not).

The exchange moves each rank's cut rows (send_lo: its first row, send_hi: its last) into
its neighbours' halo rows: send_hi -> the rank above's recv_lo, send_lo -> the rank
below's recv_hi; on a periodic grid the last and the first rank are neighbours.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def slabs():
    from paper_1704_03172_gb300 import build
    build.build()
    from paper_1704_03172_gb300 import slabs
    return slabs


def test_partition_tiles_the_rows(slabs):
    for ny, n in ((10, 3), (4096, 8), (7, 7), (1000, 6), (33, 1)):
        b = slabs.partition(ny, n)
        assert len(b) == n and b[0][0] == 0 and b[-1][1] == ny
        assert all(b[k][1] == b[k + 1][0] for k in range(n - 1))
        h = [y1 - y0 for y0, y1 in b]
        assert max(h) - min(h) <= 1 and min(h) >= 1
    with pytest.raises(ValueError):
        slabs.partition(3, 4)


def test_owner_routing_and_assembly(slabs):
    b = slabs.partition(50, 4)                   # 13, 13, 12, 12 rows
    assert [slabs.owner(y, b) for y in (0, 12, 13, 25, 26, 37, 38, 49)] == [0, 0, 1, 1, 2, 2, 3, 3]
    rec = np.array([[3, 0], [4, 13], [5, 12], [6, 49], [7, 26], [8, 13]], np.int32)
    routes = slabs.route_receivers(rec, b)
    assert [list(idx) for idx, _ in routes] == [[0, 2], [1, 5], [4], [3]]
    assert routes[1][1].tolist() == [[4, 0], [8, 0]]
    assert routes[3][1].tolist() == [[6, 11]]
    nt = 5
    full = np.arange(nt * len(rec), dtype=np.float32).reshape(nt, len(rec))
    parts = [full[:, idx] for idx, _ in routes]
    np.testing.assert_array_equal(slabs.assemble_traces(parts, routes, len(rec), nt), full)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, periodic, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1704_03172_gb300 import slabs
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws)
    n = 37
    send_lo = torch.full((n,), rank * 10.0 + 1)
    send_hi = torch.full((n,), rank * 10.0 + 2)
    recv_lo = torch.full((n,), -1.0)
    recv_hi = torch.full((n,), -1.0)
    for _ in range(3):   # repeated exchanges stay matched
        slabs.exchange(send_lo, send_hi, recv_lo, recv_hi, rank, ws, periodic)
    g = torch.full((4, 3), float(rank + 1))
    slabs.allreduce_gradient(g)
    out.put((rank, float(recv_lo[0]), float(recv_lo[-1]), float(recv_hi[0]), float(recv_hi[-1]),
             float(g[0, 0])))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ws,periodic", [(2, False), (2, True), (3, False), (3, True)])
def test_exchange_and_gradient_sum_between_gloo_ranks(slabs, ws, periodic):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, periodic, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, lo0, lo1, hi0, hi1, gsum in res:
        below, above = slabs.neighbours(rank, ws, periodic)
        exp_lo = -1.0 if below is None else below * 10.0 + 2     # the rank below's last row
        exp_hi = -1.0 if above is None else above * 10.0 + 1     # the rank above's first row
        assert (lo0, lo1) == (exp_lo, exp_lo), (rank, lo0, exp_lo)
        assert (hi0, hi1) == (exp_hi, exp_hi), (rank, hi0, exp_hi)
        assert gsum == ws * (ws + 1) / 2


def test_single_rank_exchange_wraps_a_periodic_grid(slabs):
    import torch
    a, b = torch.tensor([1.0, 2.0]), torch.tensor([3.0, 4.0])
    rl, rh = torch.zeros(2), torch.zeros(2)
    slabs.exchange(a, b, rl, rh, 0, 1, True)
    assert rl.tolist() == [3.0, 4.0] and rh.tolist() == [1.0, 2.0]
    rl.zero_()
    slabs.exchange(a, b, rl, rh, 0, 1, False)
    assert rl.tolist() == [0.0, 0.0]
