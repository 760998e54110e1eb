"""Drop impact on a cylinder and the film on its top (Sec. 4.5), FP32 on the GPU.

* lbm_column_density: the field read-out's densities bit for bit, the oracle's within FP64
  rounding (FP32: the 1e-5 bar of the first steps), NaN at solid nodes, bounds refused;
* at full size (600 x 1200, cylinder R = 100, drop D = 200, CS 0.6 Tc, MRT tau = 0.8, gravity
  from the Bond number with the oracle-measured surface tension, drop launched at 0.02 lu/step:
  Re = U_i D / nu ~ 50, We ~ 10):
  - the kinematic early-time law h* = 1 - t*: measured within 0.05 up to t* = 0.3 (the film's
    top then starts to lag: 0.057 at t* = 0.34 on the hydrophilic wall);
  - the film thins from t* = 0.5 through 1 to 1.5 (means over +-0.1 in t*);
  - on the hydrophilic cylinder (Bo 2.2, 60 deg) the film at t* = 1.5 ... 2.5 lies within a
    factor 3 of the intermediate law 0.15 t*^-2 (measured 2.4 ... 1.2: at this Reynolds number
    the viscous film stays thicker than the high-Re experiments the law was fitted to);
  - mass conserved to 1e-6.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as O
import scenarios as S
from harness import make_lattice, make_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_04508_gb300 import build
    build.build()
    O.build()


@pytest.mark.parametrize("fp64", [True, False])
def test_column_density_matches_the_oracle(fp64):
    sc = S.small_parity(fp64=fp64)
    lat, orc = make_lattice(sc), make_oracle(sc)
    lat.step(25)
    orc.step(25)
    ro = orc.fields()[0]
    rg = lat.fields()[0]
    kind, _ = orc.kind()
    for x in (0, 17, int(sc.cx[0]), sc.nx - 1):
        col = lat.column_density(x)
        solid = kind[:, x] != 0
        assert np.all(np.isnan(col[solid])) and np.all(np.isfinite(col[~solid]))
        # the same sum as the field read-out, to the bit; against the oracle within the FP64
        # rounding, or the FP32 bar of the first steps
        assert np.array_equal(col[~solid], rg[~solid, x].astype(np.float64))
        err = np.abs(col[~solid] - ro[~solid, x]) / ro[~solid, x]
        assert err.max() < (1e-12 if fp64 else 1e-5), err.max()
    part = lat.column_density(5, 10, 7)
    assert np.array_equal(part, lat.column_density(5)[10:17], equal_nan=True)


def test_column_outside_the_lattice_is_refused():
    import paper_2203_04508_gb300 as G
    lat = make_lattice(S.small_parity())
    for args in ((-1, 0, 5), (lat.nx, 0, 5), (0, lat.ny - 2, 5), (0, 0, 0)):
        with pytest.raises(G.LbmError):
            lat.column_density(*args)


def film(bo, theta, steps=30000, every=100):
    import paper_2203_04508_gb300 as G
    from paper_2203_04508_gb300.film import FilmProbe
    sc = S.e5_impact(bo, theta)
    lat = G.Lattice(sc.physics(), precision=G.LBM_FP32)
    lat.init_droplets(sc.droplets())
    info = lat.eos_info()
    probe = FilmProbe(lat, sc.cx[0], sc.cy[0] + sc.r[0], info["rho_g"], info["rho_l"], 2 * sc.r0[0])
    for k in range(0, steps, every):
        probe.sample(k)
        lat.step(every)
    M, M0, _ = lat.mass()
    return probe.result(), M / M0 - 1


@pytest.mark.parametrize("bo,theta", [(2.2, 60.0), (4.0, 150.0)])
def test_film_thickness_on_the_cylinder_top(bo, theta):
    res, drift = film(bo, theta)
    assert abs(drift) < 1e-6
    assert res["impact"] and 0.018 < res["U_i"] < 0.032 and abs(res["h_i"] / 200.0 - 1) < 0.03
    ts, hs = res["tstar"], res["hstar"]
    early = (ts >= 0.05) & (ts <= 0.3)
    assert early.sum() >= 5
    assert np.abs(hs[early] - (1 - ts[early])).max() < 0.06
    # the film thins (window means: capillary ripples make single samples wobble)
    means = [hs[(ts >= a - 0.1) & (ts <= a + 0.1)].mean() for a in (0.5, 1.0, 1.5)]
    assert means[0] > means[1] > means[2], means
    if theta < 90.0:
        mid = (ts >= 1.5) & (ts <= 2.5)
        ratio = hs[mid] / (0.15 * ts[mid] ** -2)
        assert np.all((ratio > 1 / 3) & (ratio < 3)), ratio
