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
