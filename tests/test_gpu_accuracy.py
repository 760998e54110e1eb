"""Accuracy of the FP32 (and FP64) CUDA path on the full-size workloads, against values the
FP64 reference oracle gave on the same seeded inputs (tests/golden/accuracy_refs.json, written
by tests/golden/make_accuracy_refs.py, which runs the oracle only).

  c2 (1024 x 1024, 16 drops on cylinders, FP32):
    - after 1000 steps, rho (pointwise relative) and v = u + F/(2 rho) (relative to the
      largest speed on the lattice) at 1024 seeded nodes, half of them in interfaces.  Measured
      1.8e-5 and 1.4e-5: the oracle with every quantity the step stores rounded to FP32 once
      per step (populations, density, chemical potential, force, velocity) reaches 1.8e-5 in
      rho by itself, so the bars are 2.5e-5 and 2e-5;
    - at 5000, 10000 and 20000 steps, the steady-state measures: every drop's liquid density,
      the gas density and every contact angle within 1e-3 relative (the steady-state
      accuracy asked of the FP32 path); the mass change within 1e-6 of the oracle's.
  c3 (2048 x 4096 drop impact, FP32): the drop's lower and upper interface on the line
    through the cylinder centre every 100 steps up to 500 (1e-3 lu), the mass change (1e-6),
    and rho, v after 500 steps at 1024 seeded nodes (5e-5 and 1e-5; measured 3.6e-5 and 6.7e-6).
  c5 (512 x 512, 4000 steps, checkpoints every 200): J and its gradient with respect to the
    wall chemical potentials and the cylinder centre against the oracle's complex-step
    derivatives: FP64 within 1e-8, FP32 within 1e-4 relative.
"""
import json
import os

import numpy as np
import pytest

import scenarios as S
from diagnostics import droplet_report, isoline_crossings_column, report_errors, sampled_errors
from harness import make_lattice

pytestmark = pytest.mark.gpu

REFS = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "accuracy_refs.json")))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_04508_gb300 import build
    build.build()


def c2_report(lat, sc, info):
    r, _, _ = lat.fields()
    d = sc.droplets()
    rep = droplet_report(r.astype(np.float64), lat.kind() == 0, info["rho_g"], info["rho_l"],
                         sc.cx, sc.cy, sc.r, d["x0"], d["y0"], d["r0"])
    M, M0, _ = lat.mass()
    rep["mass_change"] = M / M0 - 1
    return rep


def test_c2_fields_after_1000_fp32_steps():
    sc = S.c2_fp32_single()
    lat = make_lattice(sc, fp64=False)
    lat.step(1000)
    er, ev = sampled_errors(*lat.fields(), REFS["c2"]["fields_1000"])
    print(f"c2 1000 steps: rho {er:.2e} v {ev:.2e}")
    assert er <= 2.5e-5 and ev <= 2e-5, (er, ev)


def test_c2_steady_state_measures_fp32():
    sc = S.c2_fp32_single()
    lat = make_lattice(sc, fp64=False)
    info = lat.eos_info()
    done = 0
    for target in ("5000", "10000", "20000"):
        lat.step(int(target) - done)
        done = int(target)
        errs = report_errors(c2_report(lat, sc, info), REFS["c2"]["reports"][target])
        print(f"c2 {target} steps: {errs}")
        assert errs["missing"] == 0, errs
        assert errs["rho_liquid"] <= 1e-3 and errs["rho_gas"] <= 1e-3 and errs["theta"] <= 1e-3, errs
        assert errs["mass_change"] <= 1e-6, errs


def test_c3_impact_window_fp32():
    sc = S.c3_impact()
    ref = REFS["c3"]
    lat = make_lattice(sc, fp64=False)
    info = lat.eos_info()
    mid = 0.5 * (info["rho_g"] + info["rho_l"])
    xc = ref["x_line"]
    for k, st in enumerate(ref["steps"]):
        if k:
            lat.step(st - ref["steps"][k - 1])
        r, _, _ = lat.fields()
        ys = isoline_crossings_column(r[:, xc].astype(np.float64), lat.kind()[:, xc] == 0, mid,
                                      y_min=sc.cy[0] + sc.r[0] + 5.0)
        M, M0, _ = lat.mass()
        assert abs(ys[0] - ref["lower"][k]) <= 1e-3 and abs(ys[-1] - ref["upper"][k]) <= 1e-3, (st, ys)
        assert abs((M / M0 - 1) - ref["mass_change"][k]) <= 1e-6
    er, ev = sampled_errors(*lat.fields(), ref["fields_500"])
    print(f"c3 500 steps: rho {er:.2e} v {ev:.2e}")
    assert er <= 5e-5 and ev <= 1e-5, (er, ev)


def c5_gradient(fp64):
    sc = S.c5_adjoint()
    lat = make_lattice(sc, fp64=fp64)
    lat.forward_checkpointed(sc.steps, 200)
    J, seed = lat.objective(0, seed=True)
    return J, np.asarray(lat.adjoint(drho=seed), dtype=np.float64)


@pytest.mark.parametrize("fp64", [True, False])
def test_c5_gradient_against_the_oracle(fp64):
    ref = REFS["c5"]
    J, g = c5_gradient(fp64)
    cs = np.array([ref["complex_step"][k] for k in ref["order"]])
    cd = np.array([ref["central_differences"][k] for k in ref["order"]])
    e_cs = np.abs(g - cs) / np.abs(cs)
    e_cd = np.abs(g - cd) / np.abs(cd)
    print(f"c5 {'FP64' if fp64 else 'FP32'}: J {J!r} (oracle {ref['J']!r}); rel err vs complex step {e_cs}, "
          f"vs central differences {e_cd}")
    bar = 1e-8 if fp64 else 1e-4
    assert abs(J - ref["J"]) <= (1e-12 if fp64 else 1e-6) * abs(ref["J"])
    assert (e_cs <= bar).all(), e_cs
