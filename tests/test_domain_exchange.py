"""The halo exchange of the slab decomposition (paper_2112_14640_gb300.domain)
on CPU: real gloo process groups of 2 and 3 ranks send each slab's first time
slice to its lower neighbour and its last slice to its upper neighbour on a
periodic ring; every rank must receive its lower neighbour's last slice and
its upper neighbour's first slice.  Also the slab bounds and the folding of
the global boundary phase into the slab links (host logic, no GPU)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_2112_14640_gb300 import domain
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first = torch.full((5,), 10.0 * rank + 1)     # this slab's first owned slice
    last = torch.full((7,), 10.0 * rank + 2)      # ... and its last (another size: a half-spinor slice)
    recv_lo, recv_hi = domain.exchange(first, last, world, rank)
    out[rank] = (recv_lo.tolist(), recv_hi.tolist())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_exchange_ring(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        got = dict(out)
    for r in range(world):
        recv_lo, recv_hi = got[r]
        prev, nxt = (r - 1) % world, (r + 1) % world
        assert recv_lo == [10.0 * prev + 2] * 7      # lower neighbour's last slice -> lower ghost
        assert recv_hi == [10.0 * nxt + 1] * 5       # upper neighbour's first slice -> upper ghost


def _rank_reduce(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_2112_14640_gb300 import domain
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank's partial dot products (N_v = 3 RHS) of the slabs it holds
    parts = [torch.tensor([1.0, 2.0, 3.0], dtype=torch.float64) * (rank + 1),
             torch.tensor([0.5, 0.0, -1.0], dtype=torch.float64)]
    out[rank] = domain._reduce_sum(parts[:1], world, None).tolist()
    out[10 + rank] = parts[0].tolist()   # the input is not modified in place
    dist.barrier()
    dist.destroy_process_group()


def test_distributed_cg_reductions_are_summed_over_ranks():
    """The per-RHS partial reductions of the slab CG are all-reduced over the
    ranks (gloo, world size 2); in-process slabs are summed locally."""
    import torch
    from paper_2112_14640_gb300 import domain
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_reduce, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        got = dict(out)
    for r in range(world):
        assert got[r] == [3.0, 6.0, 9.0]                  # (1 + 2) x [1, 2, 3]
        assert got[10 + r] == [1.0 * (r + 1), 2.0 * (r + 1), 3.0 * (r + 1)]
    a, b = torch.tensor([1.0, 2.0]), torch.tensor([3.0, -1.0])
    assert domain._reduce_sum([a, b], 1, None).tolist() == [4.0, 1.0]
    assert a.tolist() == [1.0, 2.0]


def test_single_slab_exchanges_with_itself():
    import torch
    from paper_2112_14640_gb300 import domain
    a, b = torch.ones(3), torch.zeros(3)
    lo, hi = domain.exchange(a, b, 1, 0)
    assert lo is b and hi is a


def test_slab_bounds_links_and_vectors():
    from paper_2112_14640_gb300 import domain
    from paper_2112_14640_gb300 import inputs as I
    assert [domain.slab_bounds(10, 3, r) for r in range(3)] == [(0, 3), (3, 6), (6, 10)]
    with pytest.raises(ValueError):
        domain.slab_bounds(4, 5, 0)
    dims = (2, 2, 2, 6)
    U = I.gauge_field(dims, 3, 0.4, 5)
    bc = (1, 1, 1, -1)
    for world in (1, 2, 3):
        covered = []
        for r in range(world):
            t0, t1 = domain.slab_bounds(6, world, r)
            Ul = domain.slab_links(U, bc, world, r)
            assert Ul.shape[0] == t1 - t0 + 2
            for i, t in enumerate(range(t0 - 1, t1 + 1)):
                g = t % 6
                want = U[g].copy()
                if g == 5:
                    want[..., 3, :, :] *= -1          # the global antiperiodic phase, on U_t at t = N_t - 1
                assert np.array_equal(Ul[i], want)
            covered += list(range(t0, t1))
            v = I.source(dims, 3, 2, 7)
            vl = domain.slab_vector(v, world, r)
            assert np.array_equal(vl[1:-1], v[t0:t1]) and np.array_equal(vl[0], v[(t0 - 1) % 6])
        assert covered == list(range(6))
