"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds plain data only -- grid sizes, cylinder and droplet placements, physical
parameters -- and none of the method's arithmetic: the reference oracle and the CUDA library
each derive everything else (coexistence densities, chemical potentials, cut links) on their
own.

Workloads follow the paper's set-ups (a sessile drop on a flat or cylindrical wetting
substrate, Sec. 4.1-4.2, and a drop falling onto a cylinder, Sec. 4.5), at the sizes of the
benchmark configurations:

  c1  128x128 FP64, one cylinder r=20 at (64.3, 40.7), droplet r=15, BGK tau=1, CS T=0.7 Tc
  c2  1024x1024 FP32, 16 cylinders r in [40, 80] at seed-random non-lattice-aligned centres,
      droplets r = 0.8 r_cyl, MRT nu=0.1, CS T=0.6 Tc, wettability offsets for 30..150 deg
  c3  2048x4096 FP32 drop impact: cylinder r=300 at the bottom centre, droplet r=100 150 lu
      above it falling at 0.05 lu/step under gravity 1e-6, MRT tau=0.8, CS T=0.6 Tc
  c4  256 instances, square grids 128..768, T in [0.6, 0.8] Tc (batched)
  c5  512x512 MRT, droplet r=40 on a cylinder r=80 (gradients)

The model constants the paper leaves open are fixed here for every workload: the mesh
scaling k = 0.25 and the gradient coefficient kappa^ = 0.05 of Eq. 12, and the initial
interface width W = 5 of Eq. 19.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List

import numpy as np

EOS_NONE, EOS_CS, EOS_PR = 0, 1, 2
FORCE_CHEMPOT, FORCE_PSEUDO = 0, 1
COLL_BGK, COLL_MRT = 0, 1
BC_PRESENT, BC_IBC, BC_MIBC, BC_HBB = 0, 1, 2, 3

K_MESH = 0.25
KAPPA = 0.05
WIDTH = 5.0
# Contact angle versus the offset of the wall chemical potential from its saturation value
# (mesh units; positive offsets make the wall hydrophobic), measured with the reference oracle
# on a flat substrate at T = 0.6 Tc: the monotone part of tests/golden/contact_angle_table.json
# (written by tests/golden/make_contact_angle_table.py).  Angles outside 18.8..146.4 deg are
# clamped to the table's ends.
DMU_TABLE = (-0.09, -0.06, -0.045, -0.03, -0.015, 0.0, 0.015, 0.03, 0.06, 0.09, 0.12)
THETA_TABLE = (18.836, 38.122, 54.453, 68.068, 79.213, 88.991, 97.843, 105.979, 120.462, 133.284, 146.438)
# The same for Peng-Robinson with the paper's constants (Eqs. 10-11) at T = 0.7 Tc,
# kappa^ = 0.01: tests/golden/contact_angle_table_pr.json, monotone over 11.4..139.8 deg.
DMU_TABLE_PR = (-0.1, -0.08, -0.06, -0.05, -0.04, -0.03, -0.02, -0.01, 0.0, 0.01, 0.02, 0.03, 0.04, 0.05,
                0.06, 0.08, 0.1)
THETA_TABLE_PR = (11.351, 21.262, 40.91, 51.789, 61.062, 69.114, 76.463, 83.316, 89.75, 95.833, 101.635,
                  107.195, 112.535, 117.659, 122.548, 131.517, 139.753)


@dataclass
class Scenario:
    name: str
    nx: int
    ny: int
    walls: int = 1
    y_bottom: float = 1.5
    y_top: float = -1.0            # -1: ny - 2.5
    eos: int = EOS_CS
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    T_over_Tc: float = 0.7
    omega: float = 0.344
    k: float = K_MESH
    kappa: float = KAPPA
    coll: int = COLL_MRT
    tau: float = 0.8
    s_e: float = 1.64
    s_eps: float = 1.54
    s_q: float = 1.7
    s_nu: float = -1.0             # -1: 1 / tau
    gx: float = 0.0
    gy: float = 0.0
    bc: int = BC_PRESENT
    cx: List[float] = field(default_factory=list)
    cy: List[float] = field(default_factory=list)
    r: List[float] = field(default_factory=list)
    dmu_w: List[float] = field(default_factory=list)
    dmu_w_walls: float = 0.0
    force_model: int = FORCE_CHEMPOT
    # droplets (Eq. 19)
    x0: List[float] = field(default_factory=list)
    y0: List[float] = field(default_factory=list)
    r0: List[float] = field(default_factory=list)
    ux0: List[float] = field(default_factory=list)
    uy0: List[float] = field(default_factory=list)
    width: float = WIDTH
    steps: int = 1000
    fp64: bool = False

    @property
    def y_top_value(self) -> float:
        return self.y_top if self.y_top > 0 else self.ny - 2.5

    @property
    def s_nu_value(self) -> float:
        return self.s_nu if self.s_nu > 0 else 1.0 / self.tau

    def physics(self) -> dict:
        """Fields shared by the oracle configuration and the library configuration."""
        keys = ("nx", "ny", "walls", "y_bottom", "eos", "a", "b", "R", "T_over_Tc", "omega",
                "k", "kappa", "coll", "tau", "s_e", "s_eps", "s_q", "gx", "gy", "bc", "cx",
                "cy", "r", "dmu_w", "dmu_w_walls", "force_model")
        d = {k: getattr(self, k) for k in keys}
        d["y_top"] = self.y_top_value
        d["s_nu"] = self.s_nu_value
        return d

    def droplets(self) -> dict:
        n = len(self.r0)
        return dict(x0=list(self.x0), y0=list(self.y0), r0=list(self.r0),
                    ux0=list(self.ux0) if self.ux0 else [0.0] * n,
                    uy0=list(self.uy0) if self.uy0 else [0.0] * n, width=self.width)

    def with_(self, **kw) -> "Scenario":
        return replace(self, **kw)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny


def theta_to_dmu(theta_deg: float, eos: int = EOS_CS) -> float:
    """Wall chemical-potential offset giving (about) the contact angle theta_deg: CS at
    0.6 Tc, or PR at 0.7 Tc with kappa^ = 0.01."""
    if eos == EOS_PR:
        return float(np.interp(theta_deg, THETA_TABLE_PR, DMU_TABLE_PR))
    return float(np.interp(theta_deg, THETA_TABLE, DMU_TABLE))


# ---------------------------------------------------------------------------------------
def c1_plain_fp64() -> Scenario:
    """128x128, one cylinder, droplet resting on top, BGK tau=1, CS 0.7 Tc, neutral wall."""
    return Scenario(name="c1_128x128_fp64", nx=128, ny=128, T_over_Tc=0.7, coll=COLL_BGK, tau=1.0,
                    cx=[64.3], cy=[40.7], r=[20.0], dmu_w=[0.0],
                    x0=[64.3], y0=[60.7], r0=[15.0], steps=2000, fp64=True)


def _place_cylinders(rng, nx, ny, n, rmin, rmax, clearance, drop_frac):
    """Rejection sampling of n non-overlapping cylinder+droplet pairs with fractional centres."""
    out = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > 200000:
            raise RuntimeError("could not place cylinders")
        r = float(rng.uniform(rmin, rmax))
        rd = drop_frac * r
        cx = float(rng.uniform(r + clearance, nx - r - clearance))
        cy = float(rng.uniform(r + clearance, ny - r - 2 * rd - clearance))
        fx, fy = cx % 1.0, cy % 1.0
        if min(fx, 1 - fx, abs(fx - 0.5), fy, 1 - fy, abs(fy - 0.5)) < 0.05:
            continue
        ok = True
        for (ox, oy, orr, ord_) in out:
            # cylinder discs and droplet discs (droplet centred at cy + r) kept apart
            for (ax, ay, ar) in ((cx, cy, r), (cx, cy + r, rd)):
                for (bx, by, br) in ((ox, oy, orr), (ox, oy + orr, ord_)):
                    if math.hypot(ax - bx, ay - by) < ar + br + clearance:
                        ok = False
        if ok:
            out.append((cx, cy, r, rd))
    return out


def c2_fp32_single(seed: int = 2203, nx: int = 1024, ny: int = 1024, n_cyl: int = 16) -> Scenario:
    """16 cylinders r in [40, 80] with droplets r = 0.8 r, contact angles 30..150 deg."""
    rng = np.random.default_rng(seed)
    scale = min(nx, ny) / 1024.0
    cyl = _place_cylinders(rng, nx, ny, n_cyl, 40 * scale, 80 * scale, 8.0 * max(scale, 0.5), 0.8)
    thetas = rng.uniform(30.0, 150.0, size=n_cyl)
    return Scenario(name=f"c2_{nx}x{ny}_fp32", nx=nx, ny=ny, T_over_Tc=0.6, coll=COLL_MRT, tau=0.8,
                    s_nu=1.0 / 0.8,
                    cx=[c[0] for c in cyl], cy=[c[1] for c in cyl], r=[c[2] for c in cyl],
                    dmu_w=[theta_to_dmu(t) for t in thetas],
                    x0=[c[0] for c in cyl], y0=[c[1] + c[2] for c in cyl], r0=[c[3] for c in cyl],
                    steps=20000)


def c3_impact(nx: int = 2048, ny: int = 4096, theta: float = 60.0) -> Scenario:
    """Drop impact on a cylinder: r_cyl=300 at the bottom centre, droplet r=100 150 lu above."""
    s = nx / 2048.0
    rc, rd = 300.0 * s, 100.0 * s
    cx, cy = nx / 2 + 0.3, rc + 10.7 * s
    return Scenario(name=f"c3_impact_{nx}x{ny}_fp32", nx=nx, ny=ny, T_over_Tc=0.6, coll=COLL_MRT, tau=0.8,
                    gy=-1e-6, cx=[cx], cy=[cy], r=[rc], dmu_w=[theta_to_dmu(theta)],
                    x0=[cx], y0=[cy + rc + 150.0 * s + rd], r0=[rd], ux0=[0.0], uy0=[-0.05],
                    steps=10000)


def c4_batch(seed: int = 4, n: int = 256, nmin: int = 128, nmax: int = 768) -> List[Scenario]:
    """Independent droplet-on-cylinder instances of seed-random square sizes."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        N = int(rng.integers(nmin, nmax + 1))
        rc = float(rng.uniform(0.15, 0.3)) * N
        rd = float(rng.uniform(0.5, 1.0)) * rc
        rd = min(rd, (N - 2 * rc - 20) / 2.0)
        cx = N / 2 + float(rng.uniform(-0.45, 0.45))
        cy = 4.0 + rc + float(rng.uniform(0.05, 0.95))
        Tr = float(rng.uniform(0.6, 0.8))
        th = float(rng.uniform(30.0, 150.0))
        out.append(Scenario(name=f"c4_{k}_{N}", nx=N, ny=N, T_over_Tc=Tr, coll=COLL_MRT, tau=0.8,
                            cx=[cx], cy=[cy], r=[rc], dmu_w=[theta_to_dmu(th)],
                            x0=[cx], y0=[cy + rc], r0=[rd], steps=5000))
    return out


def c5_adjoint() -> Scenario:
    return Scenario(name="c5_adjoint_512", nx=512, ny=512, T_over_Tc=0.6, coll=COLL_MRT, tau=0.8,
                    cx=[256.37], cy=[150.61], r=[80.0], dmu_w=[0.0],
                    x0=[256.37], y0=[230.61], r0=[40.0], steps=4000)


def small_parity(seed: int = 7, nx: int = 131, ny: int = 97, fp64: bool = False, coll: int = COLL_MRT,
                 bc: int = BC_PRESENT, T_over_Tc: float = 0.6) -> Scenario:
    """Small ragged grid (not a multiple of any tile) with two cylinders, one of each
    wettability sign, and droplets on them: spans several tiles and a ragged tail."""
    rng = np.random.default_rng(seed)
    cyl = _place_cylinders(rng, nx, ny, 2, 10.0, 14.0, 6.0, 0.8)
    return Scenario(name=f"small_{nx}x{ny}", nx=nx, ny=ny, T_over_Tc=T_over_Tc, coll=coll, tau=0.8,
                    bc=bc, cx=[c[0] for c in cyl], cy=[c[1] for c in cyl], r=[c[2] for c in cyl],
                    dmu_w=[theta_to_dmu(60.0), theta_to_dmu(120.0)],
                    x0=[c[0] for c in cyl], y0=[c[1] + c[2] for c in cyl], r0=[c[3] for c in cyl],
                    fp64=fp64, steps=1000)


# Surface tension of the CS model at 0.6 Tc (k = 0.25, kappa^ = 0.05), measured with the
# reference oracle by the Laplace law (tests/golden/surface_tension.json, written by
# tests/golden/make_surface_tension.py); it sets the Bond number of the drop-impact runs.
SIGMA_CS06 = 0.004918094961305327
RHO_G_CS06, RHO_L_CS06 = 0.0030814585387010035, 0.4062041397690057   # Maxwell densities, same file

# ---- the paper's own drops (Sec. 4.1-4.2), Peng-Robinson with the constants of Eqs. 10-11 --
PR_PHYSICS = dict(eos=EOS_PR, a=2 / 49, b=2 / 21, R=1.0, omega=0.344, T_over_Tc=0.7, kappa=0.01)


def e1_flat_drop(q: float, theta: float, bc: int = BC_PRESENT, nx: int = 500, ny: int = 300,
                 r0: float = 50.0) -> Scenario:
    """A drop of radius r0 on a flat substrate whose wall cuts the first fluid row's links at
    q (0 < q <= 1): the wall line is y_b = 2 - q, halfway bounce-back at the top, periodic in
    x; its centre is half a radius above the wall (Sec. 4.1: 500 x 300, r0 = 50)."""
    if not 0.0 < q <= 1.0:
        raise ValueError("q must lie in (0, 1]")
    yb = 2.0 - q
    return Scenario(name=f"e1_flat_q{q:.1f}_th{theta:.0f}", nx=nx, ny=ny, walls=1, y_bottom=yb,
                    coll=COLL_MRT, tau=0.8, bc=bc, dmu_w_walls=theta_to_dmu(theta, EOS_PR),
                    x0=[nx / 2], y0=[yb + 0.5 * r0], r0=[r0], steps=20000, **PR_PHYSICS)


def e2_curved_drop(theta: float, bc: int = BC_PRESENT, nx: int = 500, ny: int = 600,
                   R: float = 100.0, r0: float = 70.0) -> Scenario:
    """A drop of radius r0 resting on a cylinder of radius R at a non-lattice-aligned centre
    (Sec. 4.2: 500 x 600, R = 100, r0 = 70; 20000 steps at 60 deg, 25000 at 120 deg); flat
    neutral walls at the bottom and top."""
    s = nx / 500.0
    cx, cy = nx / 2 + 0.37, 180.0 * s + 0.61
    return Scenario(name=f"e2_curved_th{theta:.0f}", nx=nx, ny=ny, walls=1, coll=COLL_MRT, tau=0.8,
                    bc=bc, cx=[cx], cy=[cy], r=[R], dmu_w=[theta_to_dmu(theta, EOS_PR)],
                    x0=[cx], y0=[cy + R + 0.5 * r0], r0=[r0],
                    steps=20000 if theta < 90.0 else 25000, **PR_PHYSICS)


def e5_impact(bo: float = 4.0, theta: float = 150.0, nx: int = 600, ny: int = 1200, R: float = 100.0,
              r0: float = 100.0, U0: float = 0.02, gap: float = 20.0, tau: float = 0.8) -> Scenario:
    """A drop falling onto a cylinder (Sec. 4.5: 600 x 1200, cylinder R = 100, drop D = 200, Bond
    numbers 2.2 / 4.0 / 14.5, contact angles 60 and 150 deg): CS at 0.6 Tc, gravity from
    Bo = g (rho_l - rho_g) D^2 / sigma with the oracle-measured sigma, the drop starting `gap`
    above the cylinder and moving down at U0, neutral flat walls at the bottom and top."""
    D = 2.0 * r0
    g = bo * SIGMA_CS06 / ((RHO_L_CS06 - RHO_G_CS06) * D * D)
    cx, cy = nx / 2 + 0.37, R + 60.61
    return Scenario(name=f"e5_impact_bo{bo:g}_th{theta:.0f}", nx=nx, ny=ny, walls=1, T_over_Tc=0.6, coll=COLL_MRT,
                    tau=tau, gy=-g, cx=[cx], cy=[cy], r=[R], dmu_w=[theta_to_dmu(theta)],
                    x0=[cx], y0=[cy + R + gap + r0], r0=[r0], ux0=[0.0], uy0=[-U0], steps=30000)


ALL = {"c1": c1_plain_fp64, "c2": c2_fp32_single, "c3": c3_impact, "c5": c5_adjoint}
