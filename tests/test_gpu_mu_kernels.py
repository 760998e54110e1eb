"""The chemical-potential passes (Eq. 12; lbm_set_mu_kernel) -- one node a thread, row vectors,
row sweeps, and (FP32) mu formed with the next state's density in one tiled pass, finished at the
nodes next to solids and boundary nodes after the boundary phase -- give the same bits:
populations after a run on walled and periodic lattices, ragged sizes (partial vectors, partial
sweeps and tiles, lanes at warp and lattice edges), lattices narrower than two vectors, and the
large impact lattice with the TMA-pipelined collide."""
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


CASES = {
    "walls_ragged": lambda: S.small_parity(fp64=False),
    "periodic_ragged": lambda: S.Scenario(name="p", nx=61, ny=77, walls=0, T_over_Tc=0.7, cx=[30.41], cy=[26.77],
                                          r=[11.3], dmu_w=[0.0], x0=[30.4], y0=[58.0], r0=[9.0]),
    "periodic_multiple_of_4": lambda: S.Scenario(name="p4", nx=64, ny=40, walls=0, T_over_Tc=0.7,
                                                 x0=[31.0], y0=[20.5], r0=[9.0]),
    "impact": lambda: S.c3_impact(1024, 2048),
    # large enough for the column-strip form of the fused pass (a full wave of strips x bands)
    "impact_full": lambda: S.c3_impact(),
    # narrower than two vectors: every lane's outer neighbours wrap around the lattice
    "tiny_periodic": lambda: S.Scenario(name="t", nx=6, ny=9, walls=0, T_over_Tc=0.9, x0=[2.7], y0=[4.4],
                                        r0=[2.0]),
    "smallest_walled": lambda: S.Scenario(name="w", nx=5, ny=21, walls=1, T_over_Tc=0.9, x0=[2.5], y0=[10.3],
                                          r0=[2.0]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_mu_kernels_agree(name):
    sc = CASES[name]()
    steps = 37 if not name.startswith("impact") else 60
    pops = []
    for kind in (0, 1, 2, 3):
        lat = make_lattice(sc, fp64=False)
        lat.set_mu_kernel(kind)
        lat.step(steps)
        pops.append(lat.populations())
        M, M0, _ = lat.mass()
        assert abs(M / M0 - 1) < 1e-5
    assert np.array_equal(pops[0], pops[1])
    assert np.array_equal(pops[0], pops[2])
    assert np.array_equal(pops[0], pops[3])


def test_switching_to_and_from_the_fused_pass_keeps_the_state():
    sc = S.c3_impact(256, 512)
    a = make_lattice(sc, fp64=False)
    b = make_lattice(sc, fp64=False)
    b.set_mu_kernel(2)
    for k in range(4):
        a.set_mu_kernel(3 if k % 2 == 0 else 2)
        a.step(9)
        b.step(9)
    assert np.array_equal(a.populations(), b.populations())


def test_fp64_and_invalid_choices():
    import paper_2203_04508_gb300 as G
    d = make_lattice(S.small_parity(fp64=True), fp64=True)
    for fp32_only in (2, 3):
        with pytest.raises(G.LbmError):
            d.set_mu_kernel(fp32_only)
    d.set_mu_kernel(0)
    d2 = make_lattice(S.small_parity(fp64=True), fp64=True)
    d.step(11)
    d2.step(11)
    assert np.array_equal(d.populations(), d2.populations())
    f = make_lattice(S.small_parity(fp64=False), fp64=False)
    for bad in (-1, 4):
        with pytest.raises(G.LbmError):
            f.set_mu_kernel(bad)
    pp = make_lattice(S.small_parity(fp64=False).with_(force_model=S.FORCE_PSEUDO, k=1.0, kappa=0.0,
                                                       T_over_Tc=0.7, dmu_w=[0.15, -0.15]), fp64=False)
    with pytest.raises(G.LbmError):
        pp.set_mu_kernel(3)
