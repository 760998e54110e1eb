"""Parity of the CUDA path with the oracle for the pseudopotential force model (the Shan-Chen
force with an EOS pseudopotential, G = -1, w = 1/3 and 1/12; CS at 0.7 Tc, k = 1).

Bars, as for the chemical-potential force: FP64 populations within 1e-11 (relative to max |f|)
step by step and 1e-10 after 50 steps of each boundary scheme; FP32 fields after 1000 steps
within 2e-5 (rho, pointwise relative, and v, normwise relative); FP32 within 1e-5
over the first steps of the full-size impact lattice; FP32 coexistence plateaus of a flat
interface within 1e-3 of the oracle's; mass of the present scheme within 1e-6 over 2000 FP32
steps."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
import scenarios as S
from harness import compare, make_lattice, make_oracle

pytestmark = pytest.mark.gpu
PP = dict(force_model=S.FORCE_PSEUDO, k=1.0, kappa=0.0, T_over_Tc=0.7)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_04508_gb300 import build
    build.build()
    O.build()


def small(fp64=False, coll=S.COLL_MRT, bc=S.BC_PRESENT):
    """Two cylinders at fractional centres with drops, one wall factor of each sign."""
    return S.small_parity(fp64=fp64, coll=coll, bc=bc).with_(dmu_w=[0.15, -0.15], **PP)


def flat(q=0.3, bc=S.BC_PRESENT, fp64=False):
    yb = 2.0 - q
    return S.Scenario(name="pp_flat", nx=96, ny=60, y_bottom=yb, coll=S.COLL_MRT, tau=0.8, bc=bc,
                      dmu_w_walls=0.15, x0=[48.0], y0=[yb + 7.5], r0=[15.0], fp64=fp64, **PP)


@pytest.mark.parametrize("coll", [S.COLL_MRT, S.COLL_BGK])
def test_fp64_matches_oracle_step_by_step(coll):
    sc = small(fp64=True, coll=coll)
    lat, orc = make_lattice(sc), make_oracle(sc)
    for n in (1, 1, 8):
        lat.step(n)
        orc.step(n)
        er, ev, ef = compare(lat, orc)
        assert ef < 1e-11 and er < 1e-11 and ev < 1e-9, (n, er, ev, ef)


@pytest.mark.parametrize("bc", [S.BC_PRESENT, S.BC_IBC, S.BC_MIBC, S.BC_HBB])
def test_fp64_boundary_schemes_on_a_flat_wall(bc):
    sc = flat(0.3, bc, fp64=True)
    lat, orc = make_lattice(sc), make_oracle(sc)
    lat.step(50)
    orc.step(50)
    er, ev, ef = compare(lat, orc)
    assert ef < 1e-10 and er < 1e-10, (er, ev, ef)


@pytest.mark.parametrize("case", ["small", "flat_q0.3"])
def test_fp32_matches_oracle_after_1000_steps(case):
    sc = small() if case == "small" else flat(0.3)
    lat, orc = make_lattice(sc, fp64=False), make_oracle(sc)
    lat.step(1000)
    orc.step(1000)
    er, ev, ef = compare(lat, orc)
    print(f"{case}: rho {er:.2e} v {ev:.2e} f {ef:.2e}")
    assert er <= 2e-5 and ev <= 2e-5, (er, ev, ef)


def test_fp32_full_size_impact_first_steps():
    sc = S.c3_impact().with_(dmu_w=[0.15], **PP)
    lat, orc = make_lattice(sc, fp64=False), make_oracle(sc)
    lat.step(6)
    orc.step(6)
    er, ev, ef = compare(lat, orc)
    assert er <= 1e-5 and ev <= 1e-5, (er, ev, ef)


def test_fp32_flat_interface_coexistence_matches_the_oracle():
    """A periodic liquid slab (BGK tau = 1, 30000 steps): the FP32 plateaus against the
    oracle's (which satisfy the exact discrete pressure balance of this force)."""
    nx, ny, steps = 5, 64, 30000
    sc = S.Scenario(name="pp_slab", nx=nx, ny=ny, walls=0, coll=S.COLL_BGK, tau=1.0, **PP)
    o = O.Oracle(O.OracleConfig(**sc.physics()))
    info = o.eos_info()
    y = np.arange(ny)
    phi = 0.5 * (np.tanh((y - ny / 4) / 2.5) - np.tanh((y - 3 * ny / 4) / 2.5))
    rho = info["rho_g"] + (info["rho_l"] - info["rho_g"]) * phi
    o.set_state(np.repeat(rho, nx), np.zeros(nx * ny), np.zeros(nx * ny))
    o.step(steps)
    ro = o.fields()[0]
    lat = make_lattice(sc, fp64=False, init=False)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    lat.set_populations((w[:, None, None] * np.broadcast_to(rho[:, None], (ny, nx))[None]).astype(np.float32))
    lat.step(steps)
    rg = lat.fields()[0].astype(np.float64)
    for yy in (0, ny // 2):
        assert rg[yy, 2] == pytest.approx(ro[yy, 2], rel=1e-3), (yy, rg[yy, 2], ro[yy, 2])
    assert ro[ny // 2, 2] / ro[0, 2] > 30


def test_fp32_mass_with_the_present_scheme():
    sc = small()
    lat = make_lattice(sc, fp64=False)
    lat.step(2000)
    M, M0, _ = lat.mass()
    assert abs(M / M0 - 1) < 1e-6, M / M0 - 1


def test_reverse_mode_rejects_the_pseudopotential_force():
    import paper_2203_04508_gb300 as G
    lat = make_lattice(small(fp64=True))
    with pytest.raises(G.LbmError):
        lat.adjoint_workspace_size(10, 5)
