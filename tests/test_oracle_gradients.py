"""Pins of the gradient references the adjoint is checked against.

The oracle differentiates the droplet objective J (the centre-of-mass height of the excess
density plus the wetted arc of a cylinder) by the complex step: every quantity of the step is
complex, one parameter carries an imaginary perturbation h = 1e-20, and dJ/dp = Im J / h exact to
rounding.  That machinery is pinned here against central finite differences of the real
oracle, and the closed-form derivative of a cut fraction q of Eqs. 16-17 with respect to the
cylinder centre, which the CUDA adjoint uses, is pinned against differences of the oracle's own
cut fractions."""
from __future__ import annotations

import math

import numpy as np
import pytest

import scenarios as S
from oracle import Oracle, OracleConfig, q_cylinder
from oracle.oracle import lattice as velocity_set
from harness import grad_case, oracle_J


def run_J(sc, steps, cs=None, **over):
    return oracle_J(sc, steps, cs=cs, **over)


# (parameter code of the oracle, body, key of the physics dict, index or None)
PARAMS = [(0, 0, "dmu_w", 0), (0, -1, "dmu_w_walls", None), (1, 0, "cx", 0), (2, 0, "cy", 0)]


@pytest.mark.parametrize("param", PARAMS, ids=["dmu_cyl", "dmu_walls", "cx", "cy"])
def test_complex_step_equals_central_differences(param):
    code, body, key, idx = param
    sc = grad_case()
    steps = 60
    h_cs = 1e-20
    J, Jim = run_J(sc, steps, cs=(code, body, h_cs))
    J0, _ = run_J(sc, steps)
    assert J == pytest.approx(J0, rel=1e-13), "the complex run's real part is the real run"
    g_cs = Jim / h_cs
    # small enough that no cut fraction crosses 1/2 (where Eqs. 16 and 17 meet with a kink)
    h = 1e-4
    phys = sc.physics()

    def shifted(s):
        if idx is None:
            return {key: phys[key] + s}
        v = list(phys[key])
        v[idx] += s
        return {key: v}
    Jp, _ = run_J(sc, steps, **shifted(h))
    Jm, _ = run_J(sc, steps, **shifted(-h))
    g_fd = (Jp - Jm) / (2 * h)
    assert abs(g_cs) > 1e-6, "the case must be sensitive to the parameter"
    assert g_cs == pytest.approx(g_fd, rel=2e-5, abs=1e-9)


def test_objective_is_its_definition():
    """J recomputed from the oracle's density field, its cut links and the cylinder test."""
    sc = grad_case()
    o = Oracle(OracleConfig(**sc.physics()))
    d = sc.droplets()
    o.init_droplets(d["x0"], d["y0"], d["r0"], d["width"], d["ux0"], d["uy0"])
    o.step(30)
    J, Jim = o.objective(0)
    assert Jim == 0.0
    rho = o.fields()[0]
    kind, _ = o.kind()
    eos = o.eos_info()
    rg, rl = eos["rho_g"], eos["rho_l"]
    fl = kind == 0
    y = np.broadcast_to(np.arange(sc.ny)[:, None], rho.shape)
    ex = rho - rg
    y_cm = (ex[fl] * y[fl]).sum() / ex[fl].sum()
    L = o.links()
    ex_, ey_, _, _ = velocity_set()
    _, body = o.kind()
    r = sc.r[0]
    touch = set()
    for x1, di in zip(L["x1"], L["dir"]):
        xs, ys = (x1 % sc.nx + ex_[di]) % sc.nx, (x1 // sc.nx + ey_[di]) % sc.ny
        if body[ys, xs] == 0:
            touch.add(int(x1))
    phi = np.array([(rho.flat[n] - rg) / (rl - rg) for n in sorted(touch)])
    L_wet = 2 * math.pi * r / len(touch) * phi.sum()
    assert J == pytest.approx(y_cm + L_wet, rel=1e-12)


def test_cut_fraction_centre_derivative_closed_form():
    """|x1 + q e - c| = r  =>  dq/dc = p / (p . e) with p = x1 + q e - c, against central
    differences of the oracle's cut fractions on every cut link of a circle."""
    cx, cy, r = 40.37, 31.61, 12.3
    ex_, ey_, _, _ = velocity_set()
    e = (ex_, ey_)
    h = 1e-6
    n = 0
    for x in range(20, 62):
        for y in range(12, 52):
            if (x - cx) ** 2 + (y - cy) ** 2 <= r * r:
                continue
            for d in range(1, 9):
                xs, ys = x + e[0][d], y + e[1][d]
                if (xs - cx) ** 2 + (ys - cy) ** 2 > r * r:
                    continue
                q = q_cylinder(x, y, d, cx, cy, r)
                if not (1e-3 < q < 1 - 1e-3):
                    continue
                px, py = x + q * e[0][d] - cx, y + q * e[1][d] - cy
                pe = px * e[0][d] + py * e[1][d]
                dqx = (q_cylinder(x, y, d, cx + h, cy, r) - q_cylinder(x, y, d, cx - h, cy, r)) / (2 * h)
                dqy = (q_cylinder(x, y, d, cx, cy + h, r) - q_cylinder(x, y, d, cx, cy - h, r)) / (2 * h)
                assert dqx == pytest.approx(px / pe, rel=1e-6, abs=1e-7)
                assert dqy == pytest.approx(py / pe, rel=1e-6, abs=1e-7)
                n += 1
    assert n > 80
