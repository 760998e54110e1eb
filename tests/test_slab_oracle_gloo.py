"""y-slab decomposition of one lattice, checked on the reference oracle with two gloo ranks on
CPU (no GPU): each rank advances its own rows plus an H-row halo on each side that has a
neighbour, everything farther away poisoned with NaN, and after every k steps receives the
neighbours' own rows into its halo over torch.distributed.  With H >= 7 k (the rows one step
reaches: streaming 1, the fourth-order stencils of Eqs. 9 and 12 2 + 2, the two solid layers of
Eq. 15 2) every rank's own rows equal the undivided oracle's bit for bit; with too small a halo
the poison reaches them.  The partition and the neighbour order are the package's host logic
(paper_2203_04508_gb300.slab); the arithmetic is the oracle's alone."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import scenarios as S
from paper_2203_04508_gb300.slab import neighbours, shard_instances, slab_rows

STEPS = 60


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case(walls):
    """96 x 72 with two cylinders (one crossing the middle of the lattice, where the slabs
    meet) carrying drops of opposite wettability; walled or periodic in y."""
    return S.Scenario(name="slab", nx=96, ny=72, walls=walls, T_over_Tc=0.6, coll=S.COLL_MRT, tau=0.8,
                      cx=[30.37, 67.61], cy=[36.41, 14.83], r=[9.3, 7.2],
                      dmu_w=[S.theta_to_dmu(60.0), S.theta_to_dmu(120.0)],
                      x0=[30.37, 67.61], y0=[36.41 + 9.3, 14.83 + 7.2], r0=[7.0, 5.5])


def _rows_mod(lo, hi, ny, periodic):
    rows = np.arange(lo, hi)
    return rows % ny if periodic else rows[(rows >= 0) & (rows < ny)]


def _worker(rank, world, port, walls, halo, k, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from harness import make_oracle
    O.set_threads(2)
    sc = _case(walls)
    ny, nx = sc.ny, sc.nx
    y0, y1 = slab_rows(ny, world, halo)[rank]
    below, above = neighbours(rank, world, bool(walls))
    o = make_oracle(sc)
    keep = np.zeros(ny, bool)
    keep[_rows_mod(y0 - halo, y1 + halo, ny, not walls)] = True
    for _ in range(STEPS // k):
        f = o.populations()
        f[:, ~keep, :] = np.nan          # this rank has nothing beyond its halo
        o.set_populations(f)
        o.step(k)
        f = o.populations()
        # own rows next to each edge go to that neighbour; its own rows come back into the halo
        top = torch.from_numpy(np.ascontiguousarray(f[:, y1 - halo:y1, :]))
        bot = torch.from_numpy(np.ascontiguousarray(f[:, y0:y0 + halo, :]))
        from_below = torch.empty_like(top)
        from_above = torch.empty_like(top)
        works = []
        if above is not None:
            works.append(dist.isend(top, above, tag=0))
        if below is not None:
            works += [dist.irecv(from_below, below, tag=0), dist.isend(bot, below, tag=1)]
        if above is not None:
            works.append(dist.irecv(from_above, above, tag=1))
        for w in works:
            w.wait()
        if below is not None:
            f[:, _rows_mod(y0 - halo, y0, ny, not walls), :] = from_below.numpy()
        if above is not None:
            f[:, _rows_mod(y1, y1 + halo, ny, not walls), :] = from_above.numpy()
        o.set_populations(f)
    q.put((rank, y0, y1, o.populations()[:, y0:y1, :].copy()))
    dist.destroy_process_group()


def _run(walls, halo, k):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, walls, halo, k, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from harness import make_oracle
    ref = make_oracle(_case(walls))
    ref.step(STEPS)
    f_ref = ref.populations()
    return [(f, f_ref[:, y0:y1, :]) for _, y0, y1, f in res]


@pytest.mark.parametrize("walls,halo,k", [(1, 8, 1), (0, 8, 1), (0, 16, 2)])
def test_two_oracle_slabs_equal_the_undivided_oracle(walls, halo, k):
    for f, f_ref in _run(walls, halo, k):
        assert np.array_equal(f, f_ref)


def test_a_halo_shorter_than_one_step_reaches_is_not_enough():
    assert not all(np.array_equal(f, f_ref, equal_nan=True) for f, f_ref in _run(1, 4, 1))


def test_partition_host_logic():
    assert slab_rows(4096, 4, 8) == [(0, 1024), (1024, 2048), (2048, 3072), (3072, 4096)]
    assert slab_rows(10, 3, 3) == [(0, 3), (3, 7), (7, 10)]
    with pytest.raises(ValueError):
        slab_rows(20, 4, 8)
    assert neighbours(0, 3, True) == (None, 1) and neighbours(2, 3, True) == (1, None)
    assert neighbours(0, 3, False) == (2, 1) and neighbours(2, 3, False) == (1, 0)
    assert neighbours(0, 1, False) == (0, 0) and neighbours(0, 1, True) == (None, None)
    parts = shard_instances([5, 3, 3, 2, 1, 1], 2)
    assert sorted(sum(parts, [])) == list(range(6))
    loads = [sum([5, 3, 3, 2, 1, 1][k] for k in p) for p in parts]
    assert loads == [7, 8] or loads == [8, 7]
