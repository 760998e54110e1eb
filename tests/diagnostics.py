"""Post-processing of density fields used by the tests (not part of either compute path).

The contact angle of a sessile drop is measured the usual way for diffuse-interface
simulations: points of the mid-density isoline rho = (rho_l + rho_g)/2 are located by linear
interpolation along grid rows and columns, points closer than `skip` lattice units to the
substrate are discarded, a circle is fitted to the rest by linear least squares, and the
angle between the substrate and the circle is taken through the liquid.
"""
from __future__ import annotations

import math

import numpy as np


def isoline_points(rho: np.ndarray, level: float, mask: np.ndarray | None = None):
    """(x, y) crossings of `level` between horizontally or vertically adjacent valid nodes."""
    ny, nx = rho.shape
    valid = np.ones_like(rho, bool) if mask is None else mask
    pts = []
    a, b = rho[:, :-1], rho[:, 1:]
    va = valid[:, :-1] & valid[:, 1:]
    s = va & ((a - level) * (b - level) < 0)
    ys, xs = np.nonzero(s)
    t = (level - a[ys, xs]) / (b[ys, xs] - a[ys, xs])
    pts.append(np.stack([xs + t, ys.astype(float)], 1))
    a, b = rho[:-1, :], rho[1:, :]
    va = valid[:-1, :] & valid[1:, :]
    s = va & ((a - level) * (b - level) < 0)
    ys, xs = np.nonzero(s)
    t = (level - a[ys, xs]) / (b[ys, xs] - a[ys, xs])
    pts.append(np.stack([xs.astype(float), ys + t], 1))
    return np.concatenate(pts, 0)


def fit_circle(p: np.ndarray):
    """Algebraic least-squares circle: x^2 + y^2 + D x + E y + F = 0."""
    x, y = p[:, 0], p[:, 1]
    A = np.stack([x, y, np.ones_like(x)], 1)
    rhs = -(x * x + y * y)
    (D, E, F), *_ = np.linalg.lstsq(A, rhs, rcond=None)
    xc, yc = -D / 2, -E / 2
    return xc, yc, math.sqrt(xc * xc + yc * yc - F)


def contact_angle_flat(rho, fluid_mask, rho_g, rho_l, y_wall, skip=3.0, x_range=None):
    """Angle (degrees, through the liquid) of a drop sitting on the flat wall y = y_wall."""
    pts = isoline_points(rho, 0.5 * (rho_g + rho_l), fluid_mask)
    pts = pts[pts[:, 1] > y_wall + skip]
    if x_range is not None:
        pts = pts[(pts[:, 0] >= x_range[0]) & (pts[:, 0] <= x_range[1])]
    xc, yc, R = fit_circle(pts)
    c = (y_wall - yc) / R
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))


def contact_angle_cylinder(rho, fluid_mask, rho_g, rho_l, cx, cy, rc, skip=3.0, window=None):
    """Angle (degrees, through the liquid) of a drop sitting on top of a cylinder.

    The drop's isoline (points farther than `skip` from the cylinder and within `window` of
    the drop) is fitted by a circle (xd, yd, rd); the two circles meet at distance d between
    centres, and the angle through the liquid between them satisfies
    d^2 = rc^2 + rd^2 - 2 rc rd cos(pi - theta).
    """
    pts = isoline_points(rho, 0.5 * (rho_g + rho_l), fluid_mask)
    dist = np.hypot(pts[:, 0] - cx, pts[:, 1] - cy)
    pts = pts[dist > rc + skip]
    if window is not None:
        (x0, y0, rw) = window
        pts = pts[np.hypot(pts[:, 0] - x0, pts[:, 1] - y0) < rw]
    xd, yd, rd = fit_circle(pts)
    d = math.hypot(xd - cx, yd - cy)
    c = (rc * rc + rd * rd - d * d) / (2 * rc * rd)
    # c = cos(pi - theta)
    return 180.0 - math.degrees(math.acos(max(-1.0, min(1.0, c))))


def max_speed(vx, vy, mask):
    s = np.sqrt(vx * vx + vy * vy)
    return float(s[mask].max())


def droplet_report(rho, fluid_mask, rho_g, rho_l, cx, cy, rc, x0, y0, r0, erode=4):
    """Steady-state measures of drops resting on cylinders, for comparing two runs of the same
    workload (both compute paths are measured by this one function).

    Returns per drop k (initially centred at (x0[k], y0[k]) with radius r0[k] on cylinder k):
      rho_liquid[k]: median density of the drop's liquid core (nodes above the mid density,
                     `erode` nodes inside its interface);
      theta[k]:      contact angle through the liquid (contact_angle_cylinder on the drop's own
                     part of the mid-density isoline);
    and rho_gas: median density of the gas away from every interface and solid.  The drop on
    cylinder k is the largest connected liquid region touching it (within 3 lu of its
    circle); NaN where no liquid touches the cylinder."""
    from scipy import ndimage

    mid = 0.5 * (rho_g + rho_l)
    liquid = fluid_mask & (rho > mid)
    gas = fluid_mask & (rho <= mid)
    core_l = ndimage.binary_erosion(liquid, iterations=erode, border_value=1)
    core_g = ndimage.binary_erosion(gas, iterations=erode, border_value=1)
    labels, n = ndimage.label(liquid)
    ny, nx = rho.shape
    Y, X = np.mgrid[0:ny, 0:nx]
    pts = isoline_points(rho, mid, fluid_mask)
    out = {"rho_gas": float(np.median(rho[core_g])), "rho_liquid": [], "theta": []}
    sizes = np.bincount(labels.reshape(-1))
    for k in range(len(cx)):
        ring = (X - cx[k]) ** 2 + (Y - cy[k]) ** 2 <= (rc[k] + 3.0) ** 2
        ids = np.unique(labels[ring & liquid])
        if ids.size == 0:
            out["rho_liquid"].append(float("nan"))
            out["theta"].append(float("nan"))
            continue
        lab = ids[np.argmax(sizes[ids])]
        comp = labels == lab
        out["rho_liquid"].append(float(np.median(rho[comp & core_l])))
        near = ndimage.binary_dilation(comp, iterations=2)
        ix = np.clip(np.rint(pts[:, 0]).astype(int), 0, nx - 1)
        iy = np.clip(np.rint(pts[:, 1]).astype(int), 0, ny - 1)
        own = pts[near[iy, ix]]
        dist = np.hypot(own[:, 0] - cx[k], own[:, 1] - cy[k])
        own = own[dist > rc[k] + 3.0]
        if len(own) < 8:
            out["theta"].append(float("nan"))
            continue
        xd, yd, rd = fit_circle(own)
        d = math.hypot(xd - cx[k], yd - cy[k])
        c = (rc[k] ** 2 + rd * rd - d * d) / (2 * rc[k] * rd)
        out["theta"].append(180.0 - math.degrees(math.acos(max(-1.0, min(1.0, c)))))
    return out


def isoline_crossings_column(col, fluid, level, y_min=-1.0):
    """Positions y (linear interpolation) where the density profile `col` along one grid
    column crosses `level` between two fluid nodes, above y_min, bottom to top."""
    a, b = col[:-1], col[1:]
    ok = fluid[:-1] & fluid[1:] & ((a - level) * (b - level) < 0)
    ys = np.nonzero(ok)[0]
    pos = ys + (level - a[ys]) / (b[ys] - a[ys])
    return [float(p) for p in pos if p > y_min]


def sampled_errors(rho, vx, vy, rec):
    """(rho error, v error) of fields (ny, nx) at the nodes of a record of the oracle's fields
    {nodes, rho, vx, vy, max_speed}: rho pointwise relative, v relative to the largest speed."""
    idx = np.asarray(rec["nodes"])
    r, u, v = (np.asarray(a).reshape(-1)[idx].astype(np.float64) for a in (rho, vx, vy))
    er = np.max(np.abs(r - rec["rho"]) / np.asarray(rec["rho"]))
    ev = np.max(np.hypot(u - rec["vx"], v - rec["vy"])) / rec["max_speed"]
    return float(er), float(ev)


def report_errors(rep, ref):
    """Largest relative differences of two droplet_report results (drops that exist in both),
    and the difference of their mass changes."""
    def rel(a, b, lo=-np.inf, hi=np.inf):
        a, b = np.asarray(a, float), np.asarray(b, float)
        ok = np.isfinite(a) & np.isfinite(b) & (b > lo) & (b < hi)
        return float((np.abs(a[ok] - b[ok]) / np.abs(b[ok])).max()) if ok.any() else float("nan")
    # an angle of 0 or 180 degrees is a circle fit that failed (a drop spread into a film or
    # wrapped around its cylinder), not an angle: those drops are left out
    return {"rho_liquid": rel(rep["rho_liquid"], ref["rho_liquid"]),
            "rho_gas": rel([rep["rho_gas"]], [ref["rho_gas"]]),
            "theta": rel(rep["theta"], ref["theta"], 1.0, 179.0),
            "missing": int(np.sum(np.isfinite(ref["theta"]) != np.isfinite(rep["theta"]))),
            "mass_change": float(abs(rep["mass_change"] - ref["mass_change"]))}
