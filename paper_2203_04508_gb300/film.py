"""Film thickness on top of a cylinder during a drop impact (Sec. 4.5 of the paper).

The film thickness h_f is the depth of liquid above the cylinder's top, normalised as
h* = h_f / h_i by the drop's height h_i at the instant of impact t_i, against the time
t* = (t - t_i) U_i / D, with U_i the drop's speed at impact and D its diameter.  The laws the
paper compares with are h* = 1 - t* at early times and h* = 0.15 t*^-2 at intermediate times.

The probe reads one column of density through the library (lbm_column_density), the vertical
line through the cylinder's top, so a sample costs one small kernel and a few kilobytes.  On
that line it locates the liquid runs by the mid density (rho_g + rho_l) / 2, linearly
interpolated between nodes: the drop's lowest and highest interface, and, once the liquid
touches the wall, the film's upper interface.
"""
from __future__ import annotations

import math
from typing import List, Optional

import numpy as np

# the literature laws quoted in Sec. 4.5
def early_law(tstar):
    return 1.0 - np.asarray(tstar)


def intermediate_law(tstar):
    return 0.15 * np.asarray(tstar, dtype=np.float64) ** -2


def crossings(col: np.ndarray, level: float):
    """Interpolated positions where the column crosses `level`, as (y, rising) pairs: rising
    means liquid above the crossing.  Solid nodes (NaN) break the column."""
    out = []
    for j in range(1, len(col)):
        a, b = col[j - 1], col[j]
        if not (math.isfinite(a) and math.isfinite(b)):
            continue
        if (a - level) * (b - level) < 0.0 or (b == level and a != level):
            y = (j - 1) + (a - level) / (a - b)
            out.append((y, b > a))
    return out


class FilmProbe:
    """Samples the liquid on the line x = const above a wall at height y_wall (the cylinder's top
    surface, cy + r).  Call sample(t) while the lattice advances, then result()."""

    def __init__(self, lat, x: int, y_wall: float, rho_g: float, rho_l: float, diameter: float,
                 y_top: Optional[int] = None):
        self.lat = lat
        self.x = int(round(x))
        self.y_wall = float(y_wall)
        self.y0 = int(math.floor(self.y_wall)) + 1          # first node above the wall
        self.y1 = int(y_top) if y_top is not None else lat.ny - 3
        self.level = 0.5 * (rho_g + rho_l)
        self.D = float(diameter)
        self.t: List[float] = []
        self.bottom: List[float] = []   # lowest interface of the liquid above the wall (nan: none)
        self.top: List[float] = []      # highest interface
        self.h: List[float] = []        # film thickness: liquid from the wall up (0: not touching)

    def sample(self, t: float):
        col = self.lat.column_density(self.x, self.y0, self.y1 - self.y0)
        cr = crossings(col, self.level)
        touching = math.isfinite(col[0]) and col[0] > self.level
        falls = [y for y, up in cr if not up]   # liquid below, gas above
        rises = [y for y, up in cr if up]
        top = self.y0 + max(falls) if falls else float("nan")
        if touching:
            bottom = self.y_wall
            h = (self.y0 + min(falls) - self.y_wall) if falls else float("nan")
        else:
            bottom = self.y0 + min(rises) if rises else float("nan")
            h = 0.0
        self.t.append(float(t))
        self.bottom.append(bottom)
        self.top.append(top)
        self.h.append(h)

    def result(self) -> dict:
        """t_i, U_i, h_i and the normalised series (t*, h*) after impact.  The instant of impact is
        where the drop's lower interface, extrapolated from the last two samples before contact,
        reaches the wall; U_i is its speed over those samples and h_i the drop's height then."""
        t = np.asarray(self.t)
        h = np.asarray(self.h)
        b = np.asarray(self.bottom)
        top = np.asarray(self.top)
        k = int(np.argmax(h > 0)) if np.any(h > 0) else -1
        if k < 2:
            return {"impact": False}
        U = (b[k - 2] - b[k - 1]) / (t[k - 1] - t[k - 2])
        ti = t[k - 1] + (b[k - 1] - self.y_wall) / U if U > 0 else t[k]
        hi = np.interp(ti, t[k - 2:k + 1], top[k - 2:k + 1]) - self.y_wall
        after = t >= ti
        return {"impact": True, "t_i": float(ti), "U_i": float(U), "h_i": float(hi),
                "tstar": (t[after] - ti) * U / self.D, "hstar": h[after] / hi}
