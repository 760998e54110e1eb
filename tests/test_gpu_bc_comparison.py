"""The paper's comparison of boundary schemes (Sec. 4.3, 4.4), on reduced-size drops, FP32 GPU:

* the compensating mass Delta M of Eq. 18 per step: with the present scheme (Eqs. 16-17 with
  the F_i term) it only corrects the interpolation error and decays to almost nothing; with
  MIBC (interpolation without F_i, plus Eq. 18) it must also absorb the nonideal effect and
  stays large every step;
* spurious currents next to a flat wall at an offset q: the present scheme is at the level of
  halfway bounce-back, MIBC several times above it; at q = 1/2 the schemes coincide;
* on a curved substrate the present scheme keeps the mass (IBC and MIBC do not survive this
  set-up, see the design notes).

Each case is a sessile drop (CS, 0.6 T_c, MRT tau = 0.8) run for 10000 steps; the bars are
the orders of magnitude the paper reports, with the measured values in the comments."""
from __future__ import annotations

import numpy as np
import pytest

import scenarios as S

pytestmark = pytest.mark.gpu
STEPS = 10000


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_04508_gb300 import build
    build.build()


def run(sc):
    """(per-step Delta M history, M / M0, max |v| over fluid nodes) after STEPS steps."""
    import paper_2203_04508_gb300 as G
    lat = G.Lattice(sc.physics(), precision=G.LBM_FP32)
    lat.init_droplets(sc.droplets())
    hist = []
    for _ in range(STEPS // 1000):
        lat.step(1000)
        hist.append(lat.dM_history(1000))
    M, M0, _ = lat.mass()
    r, vx, vy = lat.fields()
    fl = lat.kind() == 0
    return np.concatenate(hist), M / M0, float(np.hypot(vx, vy)[fl].max())


def flat_drop(bc, q, theta):
    return S.Scenario(name="flat_drop", nx=160, ny=100, walls=1, y_bottom=1.0 + q, T_over_Tc=0.6,
                      coll=S.COLL_MRT, tau=0.8, bc=bc, dmu_w_walls=S.theta_to_dmu(theta),
                      x0=[80.0], y0=[13.0 + q], r0=[25.0])


@pytest.mark.parametrize("theta", [60.0, 120.0])
@pytest.mark.parametrize("q", [0.2, 0.8])
def test_present_scheme_compensates_little_and_keeps_spurious_currents_low(q, theta):
    present = run(flat_drop(S.BC_PRESENT, q, theta))
    mibc = run(flat_drop(S.BC_MIBC, q, theta))
    hbb = run(flat_drop(S.BC_HBB, q, theta))
    # late Delta M per step: present ~1e-6, MIBC 0.17-0.65 (measured)
    late_p, late_m = np.abs(present[0][-1000:]).mean(), np.abs(mibc[0][-1000:]).mean()
    assert late_m > 0.05
    assert late_p < 1e-3 * late_m
    # both compensate the mass
    assert abs(present[1] - 1) < 1e-5 and abs(mibc[1] - 1) < 1e-5
    # spurious currents: present ~= halfway bounce-back, MIBC 3-5x higher (measured)
    assert present[2] < 1.1 * hbb[2]
    assert present[2] < 0.5 * mibc[2]


def test_schemes_coincide_at_q_half():
    runs = [run(flat_drop(bc, 0.5, 60.0)) for bc in (S.BC_PRESENT, S.BC_MIBC, S.BC_HBB)]
    for h, m, v in runs:
        assert np.all(h == 0.0)
    assert runs[0][1] == runs[1][1] == runs[2][1]
    assert runs[0][2] == runs[1][2] == runs[2][2]


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_present_scheme_keeps_the_mass_on_a_curved_substrate(theta):
    """A drop r = 28 on a cylinder r = 40 (E2/E3 scaled by 0.4): mass constant to 1e-5 with a
    compensation far below one per step -- at most 0.03-0.05 early, about 1.2-1.6e-3 per step
    over the last thousand steps (measured), where the curved wall keeps a residual
    interpolation error that a flat wall at one q does not."""
    R, r0 = 40.0, 28.0
    cx, cy = 100.37, 2.0 + R + 0.61
    sc = S.Scenario(name="curved_drop", nx=200, ny=240, walls=1, T_over_Tc=0.6, coll=S.COLL_MRT, tau=0.8,
                    bc=S.BC_PRESENT, cx=[cx], cy=[cy], r=[R], dmu_w=[S.theta_to_dmu(theta)],
                    x0=[cx], y0=[cy + R + 0.5 * r0], r0=[r0])
    hist, ratio, vmax = run(sc)
    assert np.isfinite(hist).all() and np.isfinite(vmax)
    assert abs(ratio - 1) < 1e-5
    assert np.abs(hist).max() < 0.1
    assert np.abs(hist[-1000:]).mean() < 5e-3
