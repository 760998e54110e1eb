"""y-slab decomposition of one lattice on the GPU (lbm_create_slab, lbm_slab_pack/unpack):
after n steps the slabs' own rows hold exactly the populations of the undivided lattice (bit for
bit), for walled and periodic lattices, cylinders cut by the slab edges, FP32 and FP64, both
force models, several slabs and a halo refreshed every k steps; the slabs' masses and Eq. 18
sums add up to the undivided lattice's.  The slabs here are held by one process on one GPU and
exchange their halos by device copies (SlabGroup); test_zz_slab_gloo.py runs two processes
that exchange through torch.distributed."""
import numpy as np
import pytest

import scenarios as S
from harness import make_lattice

pytestmark = pytest.mark.gpu

PP = dict(force_model=S.FORCE_PSEUDO, k=1.0, kappa=0.0, T_over_Tc=0.7)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_04508_gb300 import build
    build.build()


def case(walls=1, **over):
    """160 x 120 with three cylinders, two of them crossing the lines where slabs meet, drops of
    both wettabilities on them."""
    base = dict(name="slab", nx=160, ny=120, walls=walls, T_over_Tc=0.6, coll=S.COLL_MRT, tau=0.8,
                cx=[40.37, 100.61, 130.2], cy=[59.41, 30.83, 88.5], r=[10.3, 8.2, 9.1],
                dmu_w=[S.theta_to_dmu(60.0), S.theta_to_dmu(120.0), 0.0],
                x0=[40.37, 100.61, 130.2], y0=[59.41 + 10.3, 30.83 + 8.2, 88.5 + 9.1], r0=[8.0, 6.5, 7.0])
    base.update(over)
    return S.Scenario(**base)


def run_pair(sc, n_slabs, fp64, steps, halo=8, k=1):
    import paper_2203_04508_gb300 as G
    from paper_2203_04508_gb300.slab import SlabGroup
    prec = G.LBM_FP64 if fp64 else G.LBM_FP32
    whole = make_lattice(sc, fp64=fp64)
    whole.step(steps)
    grp = SlabGroup(sc.physics(), n_slabs, halo=halo, precision=prec, steps_per_exchange=k)
    grp.init_droplets(sc.droplets())
    grp.step(steps)
    return whole, grp


@pytest.mark.parametrize("walls,n,fp64", [(1, 2, False), (1, 3, False), (0, 2, False), (0, 3, True), (1, 2, True),
                                          (0, 1, False)])
def test_slabs_equal_the_undivided_lattice(walls, n, fp64):
    sc = case(walls)
    whole, grp = run_pair(sc, n, fp64, 60)
    assert np.array_equal(grp.populations(), whole.populations())
    M, M0, dM = whole.mass()
    Ms, M0s, dMs = grp.mass()
    assert Ms == pytest.approx(M, rel=1e-12) and M0s == pytest.approx(M0, rel=1e-12)
    assert dMs == pytest.approx(dM, rel=1e-9, abs=1e-15 * M0)


def test_slabs_with_a_halo_refreshed_every_three_steps():
    sc = case(1)
    whole, grp = run_pair(sc, 3, False, 60, halo=24, k=3)
    assert np.array_equal(grp.populations(), whole.populations())


def test_slabs_with_the_pseudopotential_force():
    sc = case(1, dmu_w=[0.15, -0.15, 0.0], **PP)
    whole, grp = run_pair(sc, 2, False, 60)
    assert np.array_equal(grp.populations(), whole.populations())


def test_slab_fields_and_classes_match():
    sc = case(0)
    whole, grp = run_pair(sc, 2, False, 20)
    r, vx, vy = whole.fields()
    rs, vxs, vys = grp.fields()
    assert np.array_equal(r, rs) and np.array_equal(vx, vxs) and np.array_equal(vy, vys)
    kinds = np.concatenate([s.kind() for s in grp.slabs], axis=0)
    assert np.array_equal(kinds, whole.kind())


def test_slab_refusals():
    import paper_2203_04508_gb300 as G
    from paper_2203_04508_gb300 import LbmError
    from paper_2203_04508_gb300.slab import Slab
    sc = case(1)
    with pytest.raises(LbmError) as e:
        Slab(sc.physics(), 0, 60, halo=6)          # shorter than one step's reach
    assert e.value.status == G._abi.LBM_EINVAL
    with pytest.raises(LbmError):
        Slab(sc.physics(), 1, 60)                  # splits the bottom wall rows from their slab
    with pytest.raises(LbmError):
        Slab(sc.physics(), 56, 60)                 # owns fewer rows than it must send
    s = Slab(sc.physics(), 0, 60)
    import torch
    buf = torch.empty(s.message_bytes, dtype=torch.uint8, device="cuda")
    s.init_droplets(sc.droplets())
    with pytest.raises(LbmError) as e:
        s.pack(1, buf)                             # before the first step
    assert e.value.status == G._abi.LBM_ESTATE
    s.step(1)
    with pytest.raises(LbmError):
        s.pack(0, buf)                             # the bottom slab has no neighbour below
    s.pack(1, buf)
