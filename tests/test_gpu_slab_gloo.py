"""y-slab decomposition with one process per slab: two gloo ranks (spawned processes, both on
cuda:0) each advance their slab of one lattice and exchange halos through torch.distributed
with page-locked host copies (paper_2203_04508_gb300.slab.DistSlab).  No kernel waits on
another rank: each message is complete before the receiving rank's next launch.  After the run
the ranks' own rows must equal the undivided lattice's bit for bit, and the all-reduced mass
its mass."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    import scenarios as S
    return S.Scenario(name="slab2", nx=160, ny=120, walls=1, T_over_Tc=0.6, coll=S.COLL_MRT, tau=0.8,
                      cx=[40.37, 100.61], cy=[59.41, 30.83], r=[10.3, 8.2],
                      dmu_w=[S.theta_to_dmu(60.0), S.theta_to_dmu(120.0)],
                      x0=[40.37, 100.61], y0=[59.41 + 10.3, 30.83 + 8.2], r0=[8.0, 6.5])


def _worker(rank, world, port, steps, q):
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    for p in (os.path.dirname(here), here):
        if p not in sys.path:
            sys.path.insert(0, p)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2203_04508_gb300.slab import DistSlab
    sc = _case()
    ds = DistSlab(sc.physics(), rank, world, halo=8)
    ds.init_droplets(sc.droplets())
    ds.step(steps)
    M = ds.mass()
    q.put((rank, ds.slab.y0, ds.slab.populations().copy(), M))
    dist.destroy_process_group()


def test_two_gloo_ranks_on_one_gpu_equal_the_undivided_lattice():
    import torch
    import torch.multiprocessing as mp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_04508_gb300 import build
    build.build()
    steps = 40
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    from harness import make_lattice
    whole = make_lattice(_case(), fp64=False)
    whole.step(steps)
    f = np.concatenate([r[2] for r in res], axis=1)
    assert np.array_equal(f, whole.populations())
    M, M0, _ = whole.mass()
    for _, _, _, (Ms, M0s, _) in res:
        assert Ms == pytest.approx(M, rel=1e-12) and M0s == pytest.approx(M0, rel=1e-12)
