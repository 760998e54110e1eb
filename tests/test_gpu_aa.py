"""One population lattice in AA order (LBM_LAYOUT_AA) against the two-lattice step: the same
populations, densities, velocities, mass and Eq. 18 compensation history, bit for bit, after odd
and even step counts (the state alternates between natural and shifted slot order), on lattices
that take every path -- walls and periodic boxes, ragged edges, several cylinders, both force
models, FP32 and FP64, BGK and MRT, every boundary scheme, the TMA-pipelined collide in both of
the order's steps and the plain one -- and through the graph-launched and the phase-by-phase
step.  The AA order is an implementation choice of streaming (Eq. 5), so the values must not
change at all."""
from __future__ import annotations

import os
import tempfile

import numpy as np
import pytest

import scenarios as S
from harness import compare, make_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_04508_gb300 import build
    build.build()


def lattice(sc, fp64, layout):
    import paper_2203_04508_gb300 as G
    lat = G.Lattice(sc.physics(), precision=G.LBM_FP64 if fp64 else G.LBM_FP32, layout=layout)
    lat.init_droplets(sc.droplets())
    return lat


def same_state(a, b, what):
    fa, fb = a.populations(), b.populations()
    assert np.isfinite(fa).all(), what
    assert np.array_equal(fa, fb), (what, float(np.abs(fa.astype(np.float64) - fb).max()))
    for u, v in zip(a.fields(), b.fields()):
        assert np.array_equal(u, v), what
    assert a.mass() == b.mass(), what
    ha, hb = a.dM_history(), b.dM_history()
    assert np.array_equal(ha, hb), what


CASES = {
    "c1_fp64_bgk": (lambda: S.c1_plain_fp64(), True),
    "ragged_131x97": (lambda: S.small_parity(), False),
    "ragged_fp64": (lambda: S.small_parity(fp64=True), True),
    "impact_256x512": (lambda: S.c3_impact(256, 512), False),
    "periodic_200x150": (lambda: S.Scenario(name="p", nx=200, ny=150, walls=0, T_over_Tc=0.7,
                                            cx=[70.3, 150.6], cy=[60.2, 95.7], r=[18.0, 14.0],
                                            dmu_w=[-0.03, 0.03], x0=[70.3, 150.6], y0=[84.2, 115.7],
                                            r0=[12.0, 10.0], gy=-1e-6), False),
    "periodic_narrow_61x53": (lambda: S.Scenario(name="q", nx=61, ny=53, walls=0, cx=[30.41], cy=[26.77],
                                                 r=[11.3], dmu_w=[0.0], x0=[30.41], y0=[40.0], r0=[6.0]), False),
    "pseudo_ragged": (lambda: S.small_parity().with_(dmu_w=[0.15, -0.15], force_model=S.FORCE_PSEUDO, k=1.0,
                                                     kappa=0.0, T_over_Tc=0.7), False),
    "ibc": (lambda: S.small_parity(bc=S.BC_IBC), False),
    "mibc_fp64": (lambda: S.small_parity(bc=S.BC_MIBC, fp64=True), True),
    "hbb_bgk": (lambda: S.small_parity(bc=S.BC_HBB, coll=S.COLL_BGK), False),
}


@pytest.mark.parametrize("name", list(CASES))
def test_aa_order_equals_two_lattices(name):
    import paper_2203_04508_gb300 as G
    make, fp64 = CASES[name]
    sc = make()
    a = lattice(sc, fp64, G.LBM_LAYOUT_AB)
    b = lattice(sc, fp64, G.LBM_LAYOUT_AA)
    same_state(a, b, "initial state")
    done = 0
    for n in (1, 2, 7, 30):
        a.step(n)
        b.step(n)
        done += n
        same_state(a, b, f"after {done} steps")
    # the phase-by-phase path (profiling) runs the same kernels in the same order
    a.profile_steps(3)
    b.profile_steps(3)
    same_state(a, b, "after the profiled steps")


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("name", ["impact_512", "periodic_200x150", "pseudo_ragged"])
def test_aa_order_with_each_collide_kernel(kind, name):
    """Both steps of the AA order by the TMA-pipelined kernel (1: in place, then from the pull
    box, with tiles whose shifted rows wrap around a periodic edge read from global memory) and
    by the plain kernel (0)."""
    import paper_2203_04508_gb300 as G
    sc, fp64 = (lambda: S.c3_impact(512, 512), False) if name == "impact_512" else CASES[name]
    sc = sc()
    a = lattice(sc, False, G.LBM_LAYOUT_AB)
    b = lattice(sc, False, G.LBM_LAYOUT_AA)
    b.set_collide_kernel(kind)
    for n in (1, 4, 25):
        a.step(n)
        b.step(n)
        same_state(a, b, f"collide kernel {kind}")


def test_aa_order_halves_the_population_memory():
    import paper_2203_04508_gb300 as G
    sc = S.c3_impact(512, 1024)
    ab = G.workspace_size(sc.physics(), G.LBM_FP32, G.LBM_LAYOUT_AB)
    aa = G.workspace_size(sc.physics(), G.LBM_FP32, G.LBM_LAYOUT_AA)
    plane = sc.nx * sc.ny * 4
    # nine population planes fewer, three staging planes more
    assert ab - aa >= 6 * plane - (1 << 20), (ab, aa)


def test_aa_order_checkpoint_round_trip_at_odd_parity():
    """A checkpoint taken in the shifted order resumes the run bit for bit."""
    import paper_2203_04508_gb300 as G
    sc = S.small_parity()
    ref = lattice(sc, False, G.LBM_LAYOUT_AA)
    ref.step(11)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "aa.ckpt")
        ref.save(path)
        res = lattice(sc, False, G.LBM_LAYOUT_AA)
        res.load(path)
        same_state(ref, res, "restored")
        ref.step(9)
        res.step(9)
        same_state(ref, res, "resumed")
        # a two-lattice context of the same physics refuses the file
        other = lattice(sc, False, G.LBM_LAYOUT_AB)
        with pytest.raises(G.LbmError):
            other.load(path)


def test_aa_order_set_populations_and_readouts():
    """A state set from host arrays (staged three planes at a time), then stepped: the same as the
    two-lattice step; the column read-out and the largest speed agree in the shifted order."""
    import paper_2203_04508_gb300 as G
    sc = S.small_parity()
    a = lattice(sc, False, G.LBM_LAYOUT_AB)
    b = lattice(sc, False, G.LBM_LAYOUT_AA)
    a.step(5)
    f = a.populations()
    b.set_populations(f)
    a.set_populations(f)
    a.step(3)
    b.step(3)
    same_state(a, b, "from set populations")
    assert np.array_equal(a.column_density(60), b.column_density(60), equal_nan=True)
    assert a.max_speed() == b.max_speed()


def test_aa_order_matches_the_oracle_fp64():
    import paper_2203_04508_gb300 as G
    sc = S.small_parity(fp64=True)
    lat = lattice(sc, True, G.LBM_LAYOUT_AA)
    orc = make_oracle(sc)
    for n in (1, 4):
        lat.step(n)
        orc.step(n)
        er, ev, ef = compare(lat, orc)
        assert er <= 1e-12 and ev <= 1e-10 and ef <= 1e-12, (n, er, ev, ef)


def test_aa_order_refuses_what_needs_two_lattices():
    import paper_2203_04508_gb300 as G
    sc = S.small_parity()
    b = lattice(sc, False, G.LBM_LAYOUT_AA)
    for call in (lambda: b.set_collide_kernel(2), lambda: b.set_mu_kernel(3),
                 lambda: b.adjoint_workspace_size(10), lambda: b.objective(0)):
        with pytest.raises(G.LbmError) as e:
            call()
        assert e.value.status == G._abi.LBM_EINVAL
    phys = [S.small_parity().physics()]
    cfg, keep = G.make_config(phys[0], G.LBM_FP32, layout=G.LBM_LAYOUT_AA)
    import ctypes as C
    n = C.c_size_t()
    assert G.load().lbm_slab_workspace_size(C.byref(cfg), 0, 60, 8, C.byref(n)) == G._abi.LBM_EINVAL
