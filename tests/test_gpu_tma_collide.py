"""The TMA-pipelined collide kernel against the plain one (FP32): the same populations, bit for
bit, on lattices whose tiles take every path -- halos fetched by TMA, halos that wrap around a
periodic edge (plain loads), ragged right and top edges, walls and periodic boxes, both force
models -- and through both the graph-launched and the phase-by-phase step."""
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
    "impact_256x512": lambda: S.c3_impact(256, 512),
    "ragged_131x97": lambda: S.small_parity(),
    "periodic_200x150": lambda: S.Scenario(name="p", nx=200, ny=150, walls=0, T_over_Tc=0.7,
                                           cx=[70.3, 150.6], cy=[60.2, 95.7], r=[18.0, 14.0],
                                           dmu_w=[-0.03, 0.03], x0=[70.3, 150.6], y0=[84.2, 115.7],
                                           r0=[12.0, 10.0]),
    "periodic_narrow_61x53": lambda: S.Scenario(name="q", nx=61, ny=53, walls=0, cx=[30.41], cy=[26.77],
                                                r=[11.3], dmu_w=[0.0], x0=[30.41], y0=[40.0], r0=[6.0]),
    "c2_1024": lambda: S.c2_fp32_single(),
    "pseudo_ragged": lambda: S.small_parity().with_(dmu_w=[0.15, -0.15], force_model=S.FORCE_PSEUDO, k=1.0,
                                                    kappa=0.0, T_over_Tc=0.7),
}


@pytest.mark.parametrize("name", list(CASES))
def test_tma_collide_equals_the_plain_kernel(name):
    sc = CASES[name]()
    a = make_lattice(sc, fp64=False)
    b = make_lattice(sc, fp64=False)
    a.set_collide_kernel(1)
    assert a.collide_kernel() == 1
    b.set_collide_kernel(0)
    assert b.collide_kernel() == 0
    for n in (1, 2, 37, 200):
        a.step(n)
        b.step(n)
    fa, fb = a.populations(), b.populations()
    assert np.isfinite(fa).all()
    assert np.array_equal(fa, fb), float(np.abs(fa.astype(np.float64) - fb).max())
    Ma, M0a, _ = a.mass()
    Mb, M0b, _ = b.mass()
    assert Ma == Mb and M0a == M0b
    # the phase-by-phase path (profiling) runs the same kernels
    a.profile_steps(3)
    b.profile_steps(3)
    assert np.array_equal(a.populations(), b.populations())


def test_switching_back_and_forth_keeps_the_state():
    sc = S.c3_impact(256, 512)
    a = make_lattice(sc, fp64=False)
    b = make_lattice(sc, fp64=False)
    b.set_collide_kernel(0)
    for k in range(4):
        a.set_collide_kernel(k % 2)
        a.step(10)
        b.step(10)
    assert np.array_equal(a.populations(), b.populations())


def test_the_default_follows_the_lattice_size():
    """The pipeline pays off on large lattices only: the 2048 x 4096 impact lattice takes it, the
    1024 x 1024 one (about five tiles per persistent block) keeps the plain kernel."""
    assert make_lattice(S.c3_impact(), fp64=False).collide_kernel() == 1
    assert make_lattice(S.c2_fp32_single(), fp64=False).collide_kernel() == 0


def test_fp64_has_only_the_plain_kernel():
    import paper_2203_04508_gb300 as G
    lat = make_lattice(S.small_parity(fp64=True))
    assert lat.collide_kernel() == 0
    with pytest.raises(G.LbmError):
        lat.set_collide_kernel(1)


def test_a_wait_that_gives_up_is_reported():
    """With the pipelined kernel's wait limit at zero every block gives up at its first tile: it
    flags the error, waits (with the full limit) for its own copies in flight and leaves; the
    next mass audit reports LBM_ETIMEOUT, and the context keeps that status."""
    import paper_2203_04508_gb300 as G
    from paper_2203_04508_gb300 import _abi
    lat = make_lattice(S.c3_impact(256, 512), fp64=False)
    lat.set_collide_kernel(1)
    lat.step(3)
    lat.mass()
    lat.set_spin_limit(0)
    lat.step(1)
    with pytest.raises(G.LbmError) as e:
        lat.mass()
    assert e.value.args[0].startswith(f"lbm status {_abi.LBM_ETIMEOUT}")
    with pytest.raises(G.LbmError):
        lat.step(1)
    # a fresh context on the same device is unaffected
    other = make_lattice(S.c3_impact(256, 512), fp64=False)
    other.set_collide_kernel(1)
    other.step(3)
    M, M0, _ = other.mass()
    assert abs(M / M0 - 1) < 1e-6
