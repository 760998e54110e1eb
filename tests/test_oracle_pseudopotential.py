"""Pins of the oracle's pseudopotential force model (the Shan-Chen force with a pseudopotential
built from the EOS, F = -G psi(x) sum_i w_i psi(x + e_i) e_i, G = -1, w = 1/3 and 1/12,
psi^2 = 2 (rho c_s^2 - k^2 p0(rho))), against what the mathematics fixes:

* the force of a cosine pseudopotential field equals the stencil's Fourier symbol,
  psi(x) (-A sin theta) (sin k_x (2 + cos k_y) / 3, sin k_y (2 + cos k_x) / 3), which only the
  weights 1/3, 1/12 on the right axes give;
* the force is a sum of equal and opposite pair forces, so it sums to zero on a periodic box;
* a steady flat interface conserves the discrete momentum flux through every lattice plane,
  the sum of the populations that crossed it plus the pair forces across it, and in the bulk
  liquid that flux is the EOS pressure k^2 p0;
* at tau = 1 (BGK, f~ = f^eq(rho, u + F/rho)), the D2Q9 equilibrium's half-space sums,
  sum_{e_y = +-1} f^eq = rho/6 (1 +- 3 v + 3 v^2), turn the steady flat interface into the
  local balance  P0 = k^2 p0(rho) + F^2 / (4 rho) - psi (psi_{y+1} - 2 psi + psi_{y-1}) / 4
  at every node (with u = -F/(2 rho), the physical velocity being zero).  Multiplied by
  psi'/psi and summed over one interface the last term telescopes away, which leaves the
  mechanical-stability condition of this force with the exact-difference forcing:
  sum (P0 - k^2 p0) dpsi/psi = sum F^2/(4 rho) dpsi/psi  -- the coexistence densities follow
  neither the Maxwell construction nor the plain integral sum (P0 - k^2 p0) dpsi/psi = 0;
* wettability: the wall factor's sign decides hydrophilic against hydrophobic.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O

K = 1.0


def _cfg(**kw):
    base = dict(nx=24, ny=20, walls=0, eos=O.EOS_CS, T_over_Tc=0.7, k=K, kappa=0.0, coll=O.COLL_BGK, tau=1.0,
                force_model=O.FORCE_PSEUDO)
    base.update(kw)
    return O.OracleConfig(**base)


def _psi_of(cfg, rho):
    p, _, _ = O.eos_eval(cfg, rho)
    return np.sqrt(np.maximum(0.0, 2.0 * (np.asarray(rho) / 3.0 - cfg.k ** 2 * p)))


def _rho_for_psi(cfg, target, lo=0.02, hi=0.3):
    """Density whose pseudopotential is `target` (bisection; psi grows with rho there)."""
    a = np.full_like(target, lo)
    b = np.full_like(target, hi)
    for _ in range(200):
        m = 0.5 * (a + b)
        below = _psi_of(cfg, m) < target
        a = np.where(below, m, a)
        b = np.where(below, b, m)
    return 0.5 * (a + b)


def test_force_of_a_cosine_field_is_the_stencils_fourier_symbol():
    cfg = _cfg()
    nx, ny = cfg.nx, cfg.ny
    kx, ky = 2 * np.pi * 2 / nx, 2 * np.pi * 3 / ny
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    theta = kx * X + ky * Y
    psi0, A = float(_psi_of(cfg, [0.1])[0]), 0.02
    target = psi0 + A * np.cos(theta)
    rho = _rho_for_psi(cfg, target.ravel()).reshape(ny, nx)
    o = O.Oracle(cfg)
    o.set_state(rho.ravel(), np.zeros(nx * ny), np.zeros(nx * ny))
    o.fields()
    psi, fx, fy = o.mu_force()
    assert np.abs(psi - target).max() < 1e-12
    sx = np.sin(kx) * (2 + np.cos(ky)) / 3
    sy = np.sin(ky) * (2 + np.cos(kx)) / 3
    ex_fx = psi * (-A * np.sin(theta)) * sx
    ex_fy = psi * (-A * np.sin(theta)) * sy
    assert np.abs(fx - ex_fx).max() < 1e-14
    assert np.abs(fy - ex_fy).max() < 1e-14


def test_pair_forces_sum_to_zero_on_a_periodic_box():
    cfg = _cfg(nx=17, ny=13)
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.01, 0.35, cfg.nx * cfg.ny)
    o = O.Oracle(cfg)
    o.set_state(rho, np.zeros_like(rho), np.zeros_like(rho))
    o.fields()
    _, fx, fy = o.mu_force()
    scale = np.abs(fy).max()
    assert scale > 1e-3
    assert abs(fx.sum()) < 1e-13 * scale * fx.size and abs(fy.sum()) < 1e-13 * scale * fy.size


def _slab(coll, tau, steps=30000, nx=5, ny=64):
    cfg = _cfg(nx=nx, ny=ny, coll=coll, tau=tau)
    o = O.Oracle(cfg)
    info = o.eos_info()
    y = np.arange(ny)
    phi = 0.5 * (np.tanh((y - ny / 4) / 2.5) - np.tanh((y - 3 * ny / 4) / 2.5))
    rho = info["rho_g"] + (info["rho_l"] - info["rho_g"]) * phi
    o.set_state(np.repeat(rho, nx), np.zeros(nx * ny), np.zeros(nx * ny))
    o.step(steps)
    r = o.fields()[0][:, 0]
    psi, fx, fy = o.mu_force()
    return cfg, o, r, psi[:, 0], fx, fy[:, 0]


def _plane_flux(o, psi):
    """Momentum flux through the plane between rows y and y+1 of a steady flat interface:
    the populations that crossed it in the last streaming plus the pair forces across it
    (-G/2 psi_y psi_{y+1} per column, G = -1)."""
    f = o.populations()[:, :, 0]
    ex, ey, _, _ = O.lattice()
    ny = f.shape[1]
    y = np.arange(ny)
    yp = (y + 1) % ny
    up = [i for i in range(9) if ey[i] == 1]
    dn = [i for i in range(9) if ey[i] == -1]
    return f[up][:, yp].sum(0) + f[dn][:, y].sum(0) - 0.5 * psi * psi[yp]


@pytest.mark.parametrize("coll,tau,steps", [(O.COLL_BGK, 1.0, 30000), (O.COLL_MRT, 0.8, 60000)])
def test_flat_interface_conserves_the_momentum_flux(coll, tau, steps):
    cfg, o, r, psi, fx, fy = _slab(coll, tau, steps)
    ny = r.size
    assert r[ny // 2] / r[0] > 30                        # two phases
    assert np.abs(fx).max() < 1e-15
    # the 1D reduction of the stencil: F_y = psi (psi_{y+1} - psi_{y-1}) (1/3 + 2/12)
    assert np.abs(fy - psi * (np.roll(psi, -1) - np.roll(psi, 1)) / 2).max() < 1e-15
    pi = _plane_flux(o, psi)
    assert pi.max() - pi.min() < 1e-14
    p, _, _ = O.eos_eval(cfg, [r[ny // 2]])
    assert pi.mean() == pytest.approx(cfg.k ** 2 * p[0], rel=1e-10, abs=1e-16)


def test_tau_one_local_pressure_balance_and_mechanical_stability():
    cfg, o, r, psi, fx, F = _slab(O.COLL_BGK, 1.0)
    ny = r.size
    P0 = _plane_flux(o, psi).mean()
    p, _, _ = O.eos_eval(cfg, r)
    kp = cfg.k ** 2 * p
    lap = np.roll(psi, -1) - 2 * psi + np.roll(psi, 1)
    balance = P0 - kp - F ** 2 / (4 * r) + psi * lap / 4
    assert np.abs(balance).max() < 1e-14 * max(1.0, r.max())
    half = slice(0, ny // 2)
    dpsi = (np.roll(psi, -1) - np.roll(psi, 1)) / 2
    lhs = np.sum(((P0 - kp) * dpsi / psi)[half])
    rhs = np.sum((F ** 2 / (4 * r) * dpsi / psi)[half])
    assert lhs == pytest.approx(rhs, rel=1e-9)
    assert abs(lhs) > 1e-4                               # the exact-difference term matters
    info = o.eos_info()
    assert abs(r[0] / info["rho_g"] - 1) > 0.2           # not the Maxwell gas density


@pytest.mark.parametrize("c_w,side", [(0.15, "philic"), (-0.15, "phobic")])
def test_wall_factor_sign_decides_the_wetting(c_w, side):
    from diagnostics import contact_angle_flat
    nx, ny = 120, 60
    cfg = O.OracleConfig(nx=nx, ny=ny, walls=1, y_bottom=1.5, eos=O.EOS_CS, T_over_Tc=0.7, k=K, kappa=0.0,
                         coll=O.COLL_MRT, tau=0.8, dmu_w_walls=c_w, force_model=O.FORCE_PSEUDO)
    o = O.Oracle(cfg)
    o.init_droplets([nx / 2], [11.5], [18.0], 5.0)
    o.step(4000)
    r, _, _ = o.fields()
    kind, _ = o.kind()
    theta = contact_angle_flat(r, kind == 0, r[ny - 6, 5], r[12, nx // 2], 1.5)
    assert (theta < 80) if side == "philic" else (theta > 100), theta
    assert abs(o.mass() / o.mass0() - 1) < 1e-11
