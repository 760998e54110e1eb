"""FP32 against FP64 on the GPU through a drop impact: the half-size impact lattice (1024 x 2048,
cylinder r = 150, drop r = 50 falling at 0.05 lu/step under gravity, CS 0.6 Tc, MRT), 6000 steps
in each precision, the drop's lower and upper interface read on the line through the cylinder
centre (mid-density crossings above the cylinder) every 1000 steps.  The FP32 path stores offset
populations and sums the Eq. 18 compensation in FP64; its interfaces must follow the FP64 ones
and both must keep the mass."""
from __future__ import annotations

import math

import numpy as np
import pytest

import scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_04508_gb300 import build
    build.build()


def series(precision, sc, steps, every):
    import paper_2203_04508_gb300 as G
    from paper_2203_04508_gb300.film import FilmProbe
    lat = G.Lattice(sc.physics(), precision=precision)
    lat.init_droplets(sc.droplets())
    info = lat.eos_info()
    probe = FilmProbe(lat, sc.cx[0], sc.cy[0] + sc.r[0], info["rho_g"], info["rho_l"], 2 * sc.r0[0])
    for k in range(0, steps + 1, every):
        probe.sample(k)
        if k < steps:
            lat.step(every)
    M, M0, _ = lat.mass()
    return np.array(probe.bottom), np.array(probe.top), M / M0 - 1


def test_fp32_interfaces_follow_fp64_through_an_impact():
    import paper_2203_04508_gb300 as G
    sc = S.c3_impact(1024, 2048)
    b32, t32, m32 = series(G.LBM_FP32, sc, 6000, 1000)
    b64, t64, m64 = series(G.LBM_FP64, sc, 6000, 1000)
    print("bottom", b32 - b64, "top", t32 - t64, "mass", m32, m64)
    assert np.all(np.isfinite(t32)) and np.all(np.isfinite(b32))
    assert np.abs(t32 - t64).max() < 0.5 and np.abs(b32 - b64).max() < 0.5
    assert abs(m32) < 1e-6 and abs(m64) < 1e-12
