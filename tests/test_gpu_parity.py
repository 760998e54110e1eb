"""Parity of the CUDA path (through the C ABI) with the FP64 reference oracle.

Bars:
  - node classes and cut-link lists (x1, i, q bits, x2): bit-exact;
  - FP64 GPU vs oracle: populations within 1e-11 (relative to max |f|) after 10 steps and
    fields within 1e-9 after 1000 steps (only the order of rounding differs; transcendental
    functions differ by an ulp);
  - FP32 GPU vs oracle: within 1e-5 (rho pointwise relative, v normwise relative) over the
    first 20 steps at full size, and after 1000 steps.  One case, the 128 x 128 drop on a
    neutral cylinder run in FP32 (BGK tau = 1, 0.7 Tc), reaches 1.2e-5 in v: its transient gas
    flow amplifies rounding the most.  Rounding every stored FP32 quantity (populations,
    density, chemical potential, force, velocity) of the FP64 oracle once per step gives it
    8.3e-6 already, so its bar is 1.5e-5;
  - mass: FP64 drift <= 1e-12, FP32 drift (FP64 audit) <= 1e-6 over 2000 steps.
"""
import numpy as np
import pytest

import oracle as O
import scenarios as S
from harness import compare, make_lattice, make_oracle, pop_err, rho_err, vel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_04508_gb300 import build
    build.build()
    O.build()


def _flat_q(q, walls_bottom=1.7):
    return S.Scenario(name="flat", nx=70, ny=40, y_bottom=walls_bottom, y_top=40 - 2.3, T_over_Tc=0.7,
                      dmu_w_walls=-0.045, x0=[35.0], y0=[walls_bottom + 6.0], r0=[14.0])


GEOMETRIES = {
    "small": lambda: S.small_parity(),
    "c1": lambda: S.c1_plain_fp64(),
    "c2_full": lambda: S.c2_fp32_single(),
    "c3_full": lambda: S.c3_impact(),
    "flat_q07": lambda: _flat_q(0.7, 1.3),
    "periodic_cyl": lambda: S.Scenario(name="p", nx=61, ny=53, walls=0, cx=[30.41], cy=[26.77], r=[11.3],
                                        dmu_w=[0.0]),
    # degenerate: centre on a node and an integer radius, so that nodes lie exactly on the circle
    # (solid) and links are cut at exactly q = 1; flat walls at q = 1 (y_b = 1) and q = 1/2
    "node_centred": lambda: S.Scenario(name="n", nx=64, ny=64, walls=1, y_bottom=1.0, cx=[32.0], cy=[32.0],
                                       r=[10.0], dmu_w=[0.0], x0=[32.0], y0=[47.0], r0=[6.0]),
    # nodes and centres on both sides of x = 8192, where the FP32 pre-screens of the disc and
    # droplet tests give way to the FP64 tests; one cylinder straddles the line, one lies beyond it
    "beyond_screen": lambda: S.Scenario(name="w", nx=8250, ny=32, walls=1, cx=[8190.37, 8232.81],
                                        cy=[12.2, 15.6], r=[6.3, 5.1], dmu_w=[0.02, -0.02],
                                        x0=[8170.4, 8208.9], y0=[20.3, 24.1], r0=[5.0, 3.5]),
}


@pytest.mark.parametrize("name", list(GEOMETRIES))
def test_links_and_classes_bit_exact(name):
    sc = GEOMETRIES[name]()
    lat = make_lattice(sc, fp64=False, init=False)
    orc = make_oracle(sc, init=False)
    kg = lat.kind()
    ko, _ = orc.kind()
    assert np.array_equal(kg, ko)
    lg, lo = lat.links(), orc.links()
    assert len(lg["q"]) == len(lo["q"]) > 0
    for key in ("x1", "dir", "x2", "x2_fluid"):
        assert np.array_equal(lg[key], lo[key]), key
    assert np.array_equal(lg["q"].view(np.uint64), lo["q"].view(np.uint64))
    c = lat.counts()
    assert c["fluid"] == int((ko == 0).sum())
    assert c["solid1"] == int((ko == 1).sum()) and c["solid2"] == int((ko == 2).sum())


@pytest.mark.parametrize("name", [k for k in GEOMETRIES if GEOMETRIES[k]().r0])
def test_initial_state_matches_the_oracle(name):
    """The initial populations (Sec. 4: tanh profiles, the gas state where no droplet reaches,
    FP64) against the oracle's, and the FP32 ones within their rounding."""
    sc = GEOMETRIES[name]()
    orc = make_oracle(sc)
    fo = orc.populations()
    m = orc.kind()[0] == 0
    for fp64, bar in ((True, 1e-14), (False, 2e-7)):
        lat = make_lattice(sc, fp64=fp64)
        assert pop_err(lat.populations(), fo, m) <= bar, (fp64, pop_err(lat.populations(), fo, m))


@pytest.mark.parametrize("coll", [S.COLL_MRT, S.COLL_BGK])
def test_fp64_matches_oracle_step_by_step(coll):
    sc = S.small_parity(fp64=True, coll=coll)
    lat, orc = make_lattice(sc), make_oracle(sc)
    for n in (1, 1, 8):
        lat.step(n)
        orc.step(n)
        er, ev, ef = compare(lat, orc)
        assert ef < 1e-11 and er < 1e-11 and ev < 1e-9, (n, er, ev, ef)


@pytest.mark.parametrize("bc", [S.BC_IBC, S.BC_MIBC, S.BC_HBB])
def test_fp64_boundary_variants(bc):
    sc = S.small_parity(fp64=True, bc=bc)
    lat, orc = make_lattice(sc), make_oracle(sc)
    lat.step(50)
    orc.step(50)
    er, ev, ef = compare(lat, orc)
    assert ef < 1e-10 and er < 1e-10, (er, ev, ef)


def test_fp64_long_run_mass_and_compensation():
    """c1 geometry in FP64 for 1000 steps: fields, exact mass conservation, and the per-step
    compensation sum of Eq. 18 against the oracle's."""
    sc = S.c1_plain_fp64().with_(dmu_w=[-0.03])
    lat, orc = make_lattice(sc, fp64=True), make_oracle(sc)
    lat.step(1000)
    orc.step(1000)
    er, ev, ef = compare(lat, orc)
    assert er < 1e-9 and ev < 1e-7, (er, ev, ef)
    M, M0, dM = lat.mass()
    assert abs(M / M0 - 1) < 1e-12
    assert M0 == pytest.approx(orc.mass0(), rel=1e-11)   # tanh/sqrt of the init differ by ulps
    hist_g = lat.dM_history(1000)
    hist_o = orc.dM_history()
    assert np.allclose(hist_g, hist_o, rtol=1e-7, atol=1e-12 * M0)


# (scenario, bar on v); rho within 1e-5 everywhere
FP32_CASES = {
    "c1_neutral_bgk_0.7": (lambda: S.c1_plain_fp64().with_(fp64=False), 1.5e-5),
    "c1_hydrophilic_bgk_0.7": (lambda: S.c1_plain_fp64().with_(fp64=False, dmu_w=[-0.03]), 1e-5),
    "small_60_120_mrt_0.6": (lambda: S.small_parity(fp64=False), 1e-5),
    "c2_256_four_cylinders": (lambda: S.c2_fp32_single(nx=256, ny=256, n_cyl=4), 1e-5),
}


@pytest.mark.parametrize("which", list(FP32_CASES))
def test_fp32_matches_oracle_after_1000_steps(which):
    mk, v_bar = FP32_CASES[which]
    sc = mk()
    lat, orc = make_lattice(sc, fp64=False), make_oracle(sc)
    lat.step(1000)
    orc.step(1000)
    er, ev, ef = compare(lat, orc)
    print(f"{which}: rho {er:.2e} v {ev:.2e} f {ef:.2e}")
    assert er <= 1e-5 and ev <= v_bar, (er, ev, ef)


def test_fp32_mass_audit():
    sc = S.small_parity(fp64=False)
    lat = make_lattice(sc, fp64=False)
    lat.step(2000)
    M, M0, _ = lat.mass()
    assert abs(M / M0 - 1) < 1e-6
    orc = make_oracle(sc)
    assert M0 == pytest.approx(orc.mass0(), rel=1e-6)


def test_every_scheme_is_bounce_back_at_q_half():
    """All links at q = 1/2 (flat walls at y = 1.5, ny - 2.5): the four schemes coincide bit
    for bit and the compensation vanishes (Sec. 3.2)."""
    sc = S.Scenario(name="q_half", nx=64, ny=40, T_over_Tc=0.7, dmu_w_walls=-0.045, x0=[32.0], y0=[8.0],
                    r0=[12.0])
    pops = {}
    for bc in (S.BC_PRESENT, S.BC_IBC, S.BC_MIBC, S.BC_HBB):
        lat = make_lattice(sc.with_(bc=bc), fp64=False)
        lat.step(200)
        pops[bc] = lat.populations()
        if bc in (S.BC_PRESENT, S.BC_MIBC):
            assert np.all(lat.dM_history(200) == 0.0)
    for bc in (S.BC_PRESENT, S.BC_IBC, S.BC_MIBC):
        assert np.array_equal(pops[bc], pops[S.BC_HBB])


def test_full_size_c2_first_steps():
    sc = S.c2_fp32_single()
    lat, orc = make_lattice(sc, fp64=False), make_oracle(sc)
    lat.step(20)
    orc.step(20)
    er, ev, ef = compare(lat, orc)
    assert er <= 1e-5 and ev <= 1e-5, (er, ev, ef)


def test_full_size_c3_first_steps():
    sc = S.c3_impact()
    lat, orc = make_lattice(sc, fp64=False), make_oracle(sc)
    lat.step(6)
    orc.step(6)
    er, ev, ef = compare(lat, orc)
    assert er <= 1e-5 and ev <= 1e-5, (er, ev, ef)


def test_periodic_box_without_solids_and_ragged_sizes():
    sc = S.Scenario(name="free", nx=37, ny=29, walls=0, T_over_Tc=0.7, x0=[18.3], y0=[14.6], r0=[8.0])
    lat, orc = make_lattice(sc, fp64=True), make_oracle(sc)
    assert lat.counts()["links"] == 0
    lat.step(100)
    orc.step(100)
    er, ev, ef = compare(lat, orc)
    assert ef < 1e-10, (er, ev, ef)


def test_device_fields_equal_host_fields():
    sc = S.small_parity(fp64=False)
    lat = make_lattice(sc, fp64=False)
    lat.step(7)
    h = lat.fields()
    d = [t.cpu().numpy() for t in lat.fields(on_device=True)]
    for a, b in zip(h, d):
        assert np.array_equal(a, b)


def test_graph_and_direct_launches_agree():
    """n steps as captured graph pairs equal n single launches bit for bit."""
    sc = S.small_parity(fp64=False)
    a, b = make_lattice(sc, fp64=False), make_lattice(sc, fp64=False)
    a.step(9)
    for _ in range(9):
        b.step(1)
    assert np.array_equal(a.populations(), b.populations())


def test_instability_is_reported():
    """A state that blows up is reported by the FP64 audit as LBM_EUNSTABLE (no device fault:
    NaN arithmetic only)."""
    from paper_2203_04508_gb300 import LbmError
    sc = S.small_parity(fp64=False).with_(k=1.0, kappa=0.0, width=1.0)
    lat = make_lattice(sc, fp64=False)
    with pytest.raises(LbmError) as e:
        for _ in range(40):
            lat.step(50)
            lat.mass()
    assert e.value.status == 5


def test_single_steps_and_the_asynchronous_read_back():
    """Steps taken one at a time (the one-step graphs) give the bits of steps taken together
    (the two-step graphs), and the compensation sums read back asynchronously, one per step, are
    the per-step history."""
    import torch
    sc = S.small_parity()
    a, b = make_lattice(sc, fp64=False), make_lattice(sc, fp64=False)
    n = 9
    buf = torch.empty(n, dtype=torch.float64, pin_memory=True)
    for k in range(n):
        a.step(1)
        a.last_dM_async(buf, k)
    b.step(n)
    a.synchronize()
    assert np.array_equal(a.populations(), b.populations())
    hist = b.dM_history(n)
    assert np.array_equal(buf.numpy(), hist)
    assert a.last_dM() == hist[-1]
    # pageable memory takes the copy path (page-locked memory is stored into by a kernel)
    c = make_lattice(sc, fp64=False)
    pageable = torch.empty(n, dtype=torch.float64)
    for k in range(n):
        c.step(1)
        c.last_dM_async(pageable, k)
    c.synchronize()
    assert np.array_equal(pageable.numpy(), hist)


@pytest.mark.parametrize("fp64,layout", [(False, 0), (True, 0), (False, 1)])
def test_fields_into_caller_buffers(fp64, layout):
    """fields(out=...) fills caller-owned page-locked host tensors (which the read-out kernel
    writes directly) with the values fields() returns through its staging copies, in both
    precisions and both population layouts, and refuses buffers of the wrong shape or precision."""
    import torch
    import paper_2203_04508_gb300 as G
    sc = S.small_parity()
    lat = G.Lattice(sc.physics(), precision=G.LBM_FP64 if fp64 else G.LBM_FP32, layout=layout)
    lat.init_droplets(sc.droplets())
    lat.step(7)
    ref = lat.fields()
    dt = torch.float64 if fp64 else torch.float32
    out = [torch.empty((sc.ny, sc.nx), dtype=dt, pin_memory=True) for _ in range(3)]
    got = lat.fields(out=out)
    for a, b in zip(ref, got):
        assert np.array_equal(a, b.numpy())
    with pytest.raises(ValueError):
        lat.fields(out=[torch.empty((sc.ny, sc.nx), dtype=torch.float32 if fp64 else torch.float64) for _ in range(3)])


def test_fp64_degenerate_geometry():
    """The node-centred cylinder of integer radius with a wall at q = 1: FP64 against the oracle
    over 50 steps, and the links cut at exactly q = 1 are there."""
    sc = GEOMETRIES["node_centred"]().with_(fp64=True)
    lat, orc = make_lattice(sc), make_oracle(sc)
    q = lat.links()["q"]
    assert np.any(q == 1.0)
    lat.step(50)
    orc.step(50)
    er, ev, ef = compare(lat, orc)
    assert ef < 1e-10 and er < 1e-10, (er, ev, ef)


@pytest.mark.parametrize("fp64,layout", [(False, 0), (True, 0), (False, 1)])
def test_mass_audit_equals_the_sum_of_the_populations(fp64, layout):
    """lbm_mass's M (the FP64 audit, which converts FP32 populations to FP64 by their bit fields)
    against the sum of the read-out populations over the fluid nodes, formed in FP64 on the host,
    for the initial state and after some steps."""
    import paper_2203_04508_gb300 as G
    sc = S.small_parity()
    lat = G.Lattice(sc.physics(), precision=G.LBM_FP64 if fp64 else G.LBM_FP32, layout=layout)
    lat.init_droplets(sc.droplets())
    fluid = lat.kind() == 0
    for n in (0, 9):
        lat.step(n)
        M, M0, _ = lat.mass()
        f = lat.populations().astype(np.float64)
        ref = float(f[:, fluid].sum())
        # the read-out adds w_i rho_ref to the stored offset values in the storage precision
        assert abs(M - ref) <= (1e-12 if fp64 else 2e-7) * ref, (n, M, ref)
