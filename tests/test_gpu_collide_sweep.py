"""The collide kernel that forms the next state's density by column sweeps (collide kernel 2:
each block walks a 32-column strip up a band of tile rows and sums the populations streaming
into the rows it has finished; the strips' edge columns and the bands' edge rows are completed
by a second, small kernel) against the TMA-pipelined kernel that leaves the density to its own
pass (kind 1): the same populations, bit for bit, after runs on walled and periodic lattices,
with cylinders cut by strip and band edges, both collision operators and both equations of
state, bands of one tile row and of many, and through the graph-launched and the phase-by-phase
step."""
from __future__ import annotations

import numpy as np
import pytest

import scenarios as S
from harness import make_lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_04508_gb300 import build
    build.build()


def _cylinders(**over):
    """160 x 120 walled box, three cylinders across strip edges (x = 32 k) and drops on them."""
    base = dict(name="cyl", nx=160, ny=120, walls=1, T_over_Tc=0.6, coll=S.COLL_MRT, tau=0.8,
                cx=[31.7, 96.2, 128.4], cy=[59.41, 30.83, 88.5], r=[10.3, 8.2, 9.1],
                dmu_w=[S.theta_to_dmu(60.0), S.theta_to_dmu(120.0), 0.0],
                x0=[31.7, 96.2, 128.4], y0=[59.41 + 10.3, 30.83 + 8.2, 88.5 + 9.1], r0=[8.0, 6.5, 7.0])
    base.update(over)
    return S.Scenario(**base)


CASES = {
    # one tile row per band (more bands than tile rows would give)
    "impact_256x512": (lambda: S.c3_impact(256, 512), (1, 2, 37, 200)),
    "cylinders_walls_mrt": (lambda: _cylinders(), (1, 2, 37, 200)),
    "cylinders_walls_bgk": (lambda: _cylinders(coll=S.COLL_BGK, tau=1.0), (1, 2, 37, 200)),
    "cylinders_periodic": (lambda: _cylinders(walls=0), (1, 2, 37, 200)),
    "peng_robinson": (lambda: _cylinders(dmu_w=[0.0, 0.0, 0.0], **S.PR_PHYSICS), (1, 2, 37, 100)),
    # one strip: its left neighbour is itself
    "periodic_one_strip": (lambda: S.Scenario(name="o", nx=32, ny=64, walls=0, T_over_Tc=0.7,
                                              x0=[15.3], y0=[31.1], r0=[7.0]), (1, 2, 37, 200)),
    # bands of several tile rows
    "impact_1024x2048": (lambda: S.c3_impact(1024, 2048), (1, 2, 37)),
    "periodic_1024x512": (lambda: S.Scenario(name="p", nx=1024, ny=512, walls=0, T_over_Tc=0.7,
                                             cx=[300.3, 700.6], cy=[200.2, 350.7], r=[40.0, 30.0],
                                             dmu_w=[-0.03, 0.03], x0=[300.3, 700.6], y0=[252.2, 391.7],
                                             r0=[25.0, 20.0]), (1, 2, 37)),
    "impact_full": (lambda: S.c3_impact(), (1, 2, 37)),
}


def sweeping(lat):
    """Collide kernel 2 with the row-sweep chemical-potential pass (lattices small enough for L2
    default to the fused density + mu pass, which forms the density itself)."""
    lat.set_mu_kernel(2)
    lat.set_collide_kernel(2)
    assert lat.collide_kernel() == 2
    return lat


@pytest.mark.parametrize("name", list(CASES))
def test_sweeps_equal_the_separate_density_pass(name):
    make, runs = CASES[name]
    sc = make()
    a = sweeping(make_lattice(sc, fp64=False))
    b = make_lattice(sc, fp64=False)
    b.set_collide_kernel(1)
    assert b.collide_kernel() == 1
    for n in runs:
        a.step(n)
        b.step(n)
        fa, fb = a.populations(), b.populations()
        assert np.isfinite(fa).all()
        assert np.array_equal(fa, fb), (n, float(np.abs(fa.astype(np.float64) - fb).max()))
    Ma, M0a, dMa = a.mass()
    Mb, M0b, dMb = b.mass()
    assert Ma == Mb and M0a == M0b and dMa == dMb
    # the phase-by-phase path (profiling) runs the sweep's phases in their order
    a.profile_steps(3)
    b.profile_steps(3)
    assert np.array_equal(a.populations(), b.populations())
    a.step(5)
    b.step(5)
    assert np.array_equal(a.populations(), b.populations())


def test_switching_kernels_keeps_the_state():
    sc = S.c3_impact(256, 512)
    a = make_lattice(sc, fp64=False)
    b = make_lattice(sc, fp64=False)
    b.set_collide_kernel(1)
    a.set_mu_kernel(2)
    for k in range(6):
        a.set_collide_kernel((2, 1, 0)[k % 3])
        a.step(9)
        b.step(9)
    assert np.array_equal(a.populations(), b.populations())


def test_the_fused_chemical_potential_pass_takes_kind_1():
    """The fused density + mu pass (mu kernel 3) forms the next density itself: under it a lattice
    set to the sweeps runs kind 1, with the same values."""
    sc = S.c3_impact(256, 512)
    a = sweeping(make_lattice(sc, fp64=False))
    a.set_mu_kernel(3)
    assert a.collide_kernel() == 1
    b = sweeping(make_lattice(sc, fp64=False))
    a.step(20)
    b.step(20)
    assert np.array_equal(a.populations(), b.populations())
    a.set_mu_kernel(2)
    assert a.collide_kernel() == 2


def test_where_the_sweeps_run():
    import paper_2203_04508_gb300 as G
    # selected, never the default (kind 1 and the density pass are faster on the impact lattice)
    assert make_lattice(S.c3_impact(), fp64=False).collide_kernel() == 1
    refused = [
        make_lattice(S.small_parity(), fp64=False),                       # 131 x 97: not whole tiles
        make_lattice(_cylinders(force_model=S.FORCE_PSEUDO, k=1.0, kappa=0.0, T_over_Tc=0.7,
                                dmu_w=[0.15, -0.15, 0.0]), fp64=False),   # the pseudopotential force
        make_lattice(_cylinders(), fp64=True),                            # FP64
    ]
    for lat in refused:
        with pytest.raises(G.LbmError):
            lat.set_collide_kernel(2)


def test_a_sweep_wait_that_gives_up_is_reported():
    """A zero wait limit makes every sweeping block give up at its first tile; the next mass audit
    reports LBM_ETIMEOUT and a fresh context is unaffected."""
    import paper_2203_04508_gb300 as G
    from paper_2203_04508_gb300 import _abi
    lat = sweeping(make_lattice(S.c3_impact(256, 512), fp64=False))
    lat.step(3)
    lat.mass()
    lat.set_spin_limit(0)
    lat.step(1)
    with pytest.raises(G.LbmError) as e:
        lat.mass()
    assert e.value.args[0].startswith(f"lbm status {_abi.LBM_ETIMEOUT}")
    other = sweeping(make_lattice(S.c3_impact(256, 512), fp64=False))
    other.step(3)
    M, M0, _ = other.mass()
    assert abs(M / M0 - 1) < 1e-6
