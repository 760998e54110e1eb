"""Builds the same seeded scenario on the CUDA library and on the reference oracle, and the
error measures the parity tests use.

Error measures (relative, so that one bar covers gas and liquid):
  rho: max over fluid nodes of |rho - rho_ref| / rho_ref (pointwise);
  v:   max over fluid nodes of |v - v_ref| / max over fluid nodes of |v_ref| (normwise, because
       the velocity is near zero in the bulk);
  f:   max over fluid nodes and directions of |f - f_ref| / max |f_ref|.
"""
from __future__ import annotations

import numpy as np

import oracle as O
import scenarios as S


def make_oracle(sc: S.Scenario, init: bool = True):
    o = O.Oracle(O.OracleConfig(**sc.physics()))
    if init and sc.r0:
        d = sc.droplets()
        o.init_droplets(d["x0"], d["y0"], d["r0"], d["width"], d["ux0"], d["uy0"])
    return o


def make_lattice(sc: S.Scenario, fp64: bool | None = None, init: bool = True, rho_ref: float = -1.0):
    import paper_2203_04508_gb300 as G
    prec = G.LBM_FP64 if (sc.fp64 if fp64 is None else fp64) else G.LBM_FP32
    lat = G.Lattice(sc.physics(), precision=prec, rho_ref=rho_ref)
    if init:
        lat.init_droplets(sc.droplets())
    return lat


def rho_err(r, r_ref, mask):
    return float(np.max(np.abs(r[mask].astype(np.float64) - r_ref[mask]) / r_ref[mask]))


def vel_err(vx, vy, vx_ref, vy_ref, mask):
    dv = np.hypot(vx[mask].astype(np.float64) - vx_ref[mask], vy[mask].astype(np.float64) - vy_ref[mask])
    return float(dv.max() / np.hypot(vx_ref[mask], vy_ref[mask]).max())


def pop_err(f, f_ref, mask):
    d = np.abs(f[:, mask].astype(np.float64) - f_ref[:, mask])
    return float(d.max() / np.abs(f_ref[:, mask]).max())


def compare(lat, orc):
    """(rho error, v error, population error) between the library and the oracle now."""
    r, vx, vy = lat.fields()
    ro, vxo, vyo = orc.fields()
    kind, _ = orc.kind()
    m = kind == 0
    return rho_err(r, ro, m), vel_err(vx, vy, vxo, vyo, m), pop_err(lat.populations(), orc.populations(), m)


# ---- gradients ---------------------------------------------------------------------------
def grad_case(**kw) -> S.Scenario:
    """64 x 56 channel between flat walls with one cylinder at a non-lattice-aligned centre and
    a droplet resting on it: J depends on the cylinder's and the walls' wettability and on
    the centre."""
    base = dict(name="grad_64x56", nx=64, ny=56, T_over_Tc=0.6, coll=S.COLL_MRT, tau=0.8,
                cx=[32.37], cy=[18.61], r=[10.0], dmu_w=[-0.02], dmu_w_walls=0.01,
                x0=[32.37], y0=[29.0], r0=[7.0], fp64=True, steps=100)
    base.update(kw)
    return S.Scenario(**base)


def oracle_J(sc: S.Scenario, steps: int, cs=None, body: int = 0, **over):
    """(J, Im J) of the oracle after `steps` steps; cs = (parameter code, body, h) runs it with
    a complex-step perturbation (code 0 wall chemical potential, 1 cx, 2 cy; body -1 is the
    flat walls)."""
    phys = sc.physics()
    phys.update(over)
    o = O.Oracle(O.OracleConfig(**phys), cs_param=cs)
    d = sc.droplets()
    o.init_droplets(d["x0"], d["y0"], d["r0"], d["width"], d["ux0"], d["uy0"])
    o.step(steps)
    return o.objective(body)


def oracle_gradient(sc: S.Scenario, steps: int, body: int = 0):
    """J and dJ/dp by the complex step on the oracle, p in the library's layout:
    [dmu_w per cylinder, dmu_w of the walls, (cx, cy) per cylinder]."""
    n = len(sc.r)
    h = 1e-20
    g = np.zeros(3 * n + 1)
    J, _ = oracle_J(sc, steps, body=body)
    for k in range(n):
        g[k] = oracle_J(sc, steps, cs=(0, k, h), body=body)[1] / h
        g[n + 1 + 2 * k] = oracle_J(sc, steps, cs=(1, k, h), body=body)[1] / h
        g[n + 2 + 2 * k] = oracle_J(sc, steps, cs=(2, k, h), body=body)[1] / h
    g[n] = oracle_J(sc, steps, cs=(0, -1, h), body=body)[1] / h
    return J, g
