"""Host logic of the run diagnostics, on stand-in lattices (no GPU):

* monitor.Monitor.record: the JSON-lines record (step, M, drift, dM, max |v|, NaN flag, ms per
  step, MLUPS) from the lattice's audit, the written line equal to the kept record, the
  non-finite audit turning into a NaN-flagged record, other errors passed on;
* film.crossings: linearly interpolated level crossings, exact on linear ramps, broken by solid
  (NaN) nodes;
* film.FilmProbe: on the columns of a drop that falls at a constant speed onto a wall and keeps
  moving down as a film (the kinematic h* = 1 - t*), the impact time, speed and drop height and
  the normalised series come out exactly.
"""
from __future__ import annotations

import io
import json
import math

import numpy as np
import pytest

from paper_2203_04508_gb300 import _abi
from paper_2203_04508_gb300.film import FilmProbe, crossings, early_law, intermediate_law
from paper_2203_04508_gb300.monitor import Monitor


class AuditStub:
    nx, ny = 10, 20

    def __init__(self, status=_abi.LBM_OK, speed=0.01):
        self.status, self.speed = status, speed

    def mass(self):
        if self.status != _abi.LBM_OK:
            raise _abi.LbmError(self.status, "stand-in")
        return 2.5, 2.0, -3e-9

    def max_speed(self):
        return self.speed


def test_monitor_record_and_line(tmp_path):
    buf = io.StringIO()
    mon = Monitor(AuditStub(), buf, every=7)
    mon.steps = 21
    rec = mon.record(0.5)
    assert rec == {"step": 21, "M": 2.5, "drift": 0.25, "dM": -3e-9, "max_speed": 0.01, "nan": False,
                   "ms_per_step": 0.5, "mlups": 200 / 500.0}
    assert json.loads(buf.getvalue()) == rec
    path = tmp_path / "run.jsonl"
    mon2 = Monitor(AuditStub(), str(path), every=1)
    mon2.record(1.0)
    mon2.record(1.0)
    lines = path.read_text().splitlines()
    assert len(lines) == 2 and json.loads(lines[1]) == mon2.records[1]


def test_monitor_flags_non_finite_states():
    mon = Monitor(AuditStub(status=_abi.LBM_EUNSTABLE), None)
    rec = mon.record(1.0)
    assert rec["nan"] and mon.unstable and rec["M"] is None
    mon = Monitor(AuditStub(speed=float("nan")), None)
    rec = mon.record(1.0)
    assert rec["nan"] and mon.unstable and rec["M"] == 2.5
    with pytest.raises(_abi.LbmError):
        Monitor(AuditStub(status=_abi.LBM_ECUDA), None).record(1.0)
    with pytest.raises(ValueError):
        Monitor(AuditStub(), None, every=0)


def test_crossings_are_exact_on_linear_ramps():
    col = np.array([0.0, 0.0, 0.5, 1.0, 1.0, 0.25, 0.0])
    cr = crossings(col, 0.4)
    assert [round(y, 12) for y, _ in cr] == [1.8, 4.8]
    assert [up for _, up in cr] == [True, False]
    # a solid node breaks the column: no crossing across it
    col2 = col.copy()
    col2[2] = np.nan
    assert [round(y, 12) for y, _ in crossings(col2, 0.4)] == [4.8]
    # a value exactly at the level counts once, on the side it is reached from
    assert len(crossings(np.array([0.0, 0.4, 1.0]), 0.4)) == 1


def test_literature_laws():
    assert np.allclose(early_law([0.0, 0.25, 1.0]), [1.0, 0.75, 0.0])
    assert np.allclose(intermediate_law([1.0, 2.0]), [0.15, 0.0375])


class FallingDrop:
    """Columns of density on x = const: a drop of height D whose bottom falls at speed U from
    b0, onto a wall at y_wall; once it touches, a film from the wall to the drop's top, which
    keeps falling at U.  Linear ramps of width 2 around every interface."""
    rho_g, rho_l = 0.1, 1.1

    def __init__(self, ny=80, y_wall=10.5, b0=30.25, D=20.0, U=0.5):
        self.nx, self.ny = 8, ny
        self.y_wall, self.b0, self.D, self.U = y_wall, b0, D, U
        self.t = 0.0

    def column_density(self, x, y0, n):
        y = np.arange(y0, y0 + n, dtype=np.float64)
        b = self.b0 - self.U * self.t
        top = b + self.D
        lo = max(b, self.y_wall)
        d = np.minimum(y - lo, top - y) if b > self.y_wall else top - y
        phi = np.clip(0.5 + d / 2.0, 0.0, 1.0)
        return self.rho_g + (self.rho_l - self.rho_g) * phi


def test_film_probe_on_a_kinematic_impact():
    lat = FallingDrop()
    probe = FilmProbe(lat, 4, lat.y_wall, lat.rho_g, lat.rho_l, lat.D)
    for k in range(26):
        lat.t = 4.0 * k
        probe.sample(lat.t)
    res = probe.result()
    assert res["impact"]
    t_i = (lat.b0 - lat.y_wall) / lat.U
    assert math.isclose(res["t_i"], t_i, rel_tol=1e-12)
    assert math.isclose(res["U_i"], lat.U, rel_tol=1e-12)
    assert math.isclose(res["h_i"], lat.D, rel_tol=1e-12)
    ts, hs = res["tstar"], res["hstar"]
    assert len(ts) == sum(4.0 * k >= t_i for k in range(26))
    live = hs > 0
    assert np.allclose(hs[live], 1.0 - ts[live], atol=1e-12)


def test_film_probe_without_impact():
    lat = FallingDrop(b0=70.0, D=5.0, U=0.1)
    probe = FilmProbe(lat, 4, lat.y_wall, lat.rho_g, lat.rho_l, lat.D)
    for k in range(5):
        lat.t = float(k)
        probe.sample(lat.t)
    assert probe.result() == {"impact": False}
