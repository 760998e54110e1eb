"""The paper's own drops with Peng-Robinson (Eqs. 10-11 with its constants a = 2/49,
b = 2/21, R = 1, omega = 0.344; T = 0.7 Tc, kappa^ = 0.01), FP32 on the GPU:

* parity of the PR path with the oracle: FP64 populations step by step (present scheme and
  IBC, flat wall at q = 0.3 and a cylinder), FP32 fields after 1000 steps, and the first
  steps of both full-size cases;
* Sec. 4.1 at full size (500 x 300, r0 = 50, 20000 steps, q = 0.1 ... 1.0, 60 and 120 deg):
  the present scheme keeps the mass constant at every q, IBC makes the drop shrink on the
  hydrophilic wall and grow on the hydrophobic one, except at q = 1/2 where both are
  halfway bounce-back;
* Sec. 4.2 at full size (500 x 600, R = 100, r0 = 70; 20000 steps at 60 deg, 25000 at
  120 deg): the same on a curved substrate.

Mass is the FP64 audit over fluid nodes; the present scheme's FP32 bar (2e-6 over 20000
steps) covers the collision's rounding, which the audit sees at ~1e-7 here."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
import scenarios as S
from harness import compare, make_lattice, make_oracle

pytestmark = pytest.mark.gpu
QS = [0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 1.0]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_04508_gb300 import build
    build.build()
    O.build()


def small_flat(bc, fp64):
    return S.e1_flat_drop(0.3, 60.0, bc, nx=96, ny=60, r0=15.0).with_(fp64=fp64)


def small_curved(bc, fp64):
    return S.e2_curved_drop(120.0, bc, nx=100, ny=120, R=20.0, r0=14.0).with_(fp64=fp64)


@pytest.mark.parametrize("bc", [S.BC_PRESENT, S.BC_IBC])
@pytest.mark.parametrize("case", [small_flat, small_curved])
def test_pr_fp64_matches_oracle_step_by_step(case, bc):
    sc = case(bc, True)
    lat, orc = make_lattice(sc), make_oracle(sc)
    for n in (1, 9, 90):
        lat.step(n)
        orc.step(n)
        er, ev, ef = compare(lat, orc)
        assert ef < 1e-10 and er < 1e-10 and ev < 1e-8, (n, er, ev, ef)


@pytest.mark.parametrize("case", [small_flat, small_curved])
def test_pr_fp32_matches_oracle_after_1000_steps(case):
    sc = case(S.BC_PRESENT, False)
    lat, orc = make_lattice(sc), make_oracle(sc)
    lat.step(1000)
    orc.step(1000)
    er, ev, ef = compare(lat, orc)
    print(f"{sc.name}: rho {er:.2e} v {ev:.2e} f {ef:.2e}")
    assert er <= 5e-5 and ev <= 1.5e-4, (er, ev, ef)


@pytest.mark.parametrize("sc", [S.e1_flat_drop(0.3, 60.0), S.e2_curved_drop(120.0)], ids=["e1", "e2"])
def test_full_size_first_steps(sc):
    lat, orc = make_lattice(sc, fp64=False), make_oracle(sc)
    lat.step(10)
    orc.step(10)
    er, ev, ef = compare(lat, orc)
    assert er <= 1e-5 and ev <= 1e-5, (er, ev, ef)


def mass_trace(sc, every=1000):
    """M / M0 - 1 every `every` steps over the scenario's step count (FP32)."""
    lat = make_lattice(sc, fp64=False)
    out = []
    for _ in range(sc.steps // every):
        lat.step(every)
        M, M0, _ = lat.mass()
        out.append(M / M0 - 1.0)
    return np.array(out)


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_e1_flat_substrate_mass_over_q(theta):
    sign = -1.0 if theta < 90.0 else 1.0
    for q in QS:
        present = mass_trace(S.e1_flat_drop(q, theta, S.BC_PRESENT))
        ibc = mass_trace(S.e1_flat_drop(q, theta, S.BC_IBC))
        print(f"theta {theta} q {q}: present {present[-1]:+.2e}  ibc {ibc[-1]:+.3e}")
        # measured: present |M/M0 - 1| <= 5.5e-7 at every q; IBC -0.87 (q = 0.4, 0.6) to
        # -0.975 (q = 1) at 60 deg, +1.15 to +2.31 at 120 deg
        assert np.isfinite(present).all() and np.abs(present).max() < 2e-6, (q, present)
        if q == 0.5:
            assert np.array_equal(ibc, present)
        else:
            assert np.isfinite(ibc).all()
            assert sign * ibc[-1] > 0.5, (q, ibc[-1])


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_e2_curved_substrate_mass(theta):
    present = mass_trace(S.e2_curved_drop(theta, S.BC_PRESENT))
    ibc = mass_trace(S.e2_curved_drop(theta, S.BC_IBC))
    print(f"theta {theta}: present {present[-1]:+.2e}  ibc {ibc[-1]:+.3e}")
    # measured: present 6e-8 / -2e-8; IBC -0.92 at 60 deg after 20000 steps (the paper: down
    # to about 2 % of the initial mass) and +0.88 at 120 deg after 25000 (the paper: above 180 %)
    assert np.isfinite(present).all() and np.abs(present).max() < 2e-6, present
    if theta < 90.0:
        assert ibc[-1] < -0.8, ibc
    else:
        assert ibc[-1] > 0.6, ibc
