"""Run diagnostics through the C ABI: lbm_max_speed against the velocity field lbm_fields
returns (bit for bit: the same FP64 sum of squares) and against the oracle's, the JSON-lines
monitor's records against the mass audit, and a run that turns non-finite ending in a record
with the NaN flag."""
from __future__ import annotations

import io
import json

import numpy as np
import pytest

import oracle as O
import scenarios as S
from harness import make_lattice, make_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_04508_gb300 import build
    build.build()
    O.build()


def speed(vx, vy, fluid):
    a, b = vx[fluid].astype(np.float64), vy[fluid].astype(np.float64)
    return float(np.sqrt(a * a + b * b).max())


@pytest.mark.parametrize("fp64", [False, True])
def test_max_speed_is_the_fields_maximum(fp64):
    sc = S.small_parity(fp64=fp64)
    lat, orc = make_lattice(sc), make_oracle(sc)
    lat.step(60)
    orc.step(60)
    kind, _ = orc.kind()
    fluid = kind == 0
    v = lat.max_speed()
    _, vx, vy = lat.fields()
    assert v == speed(vx, vy, fluid)
    _, vxo, vyo = orc.fields()
    assert abs(v / speed(vxo, vyo, fluid) - 1) < (1e-10 if fp64 else 1e-3)
    # the read-out leaves the run's bits unchanged
    ref = make_lattice(sc)
    ref.step(80)
    lat.step(20)
    assert np.array_equal(lat.populations(), ref.populations())


def test_max_speed_on_the_pipelined_kernel_lattice():
    sc = S.c3_impact(1024, 2048)
    lat = make_lattice(sc, fp64=False)
    lat.set_collide_kernel(1)
    lat.step(200)
    _, vx, vy = lat.fields()
    fluid = lat.kind() == 0
    assert lat.max_speed() == speed(vx, vy, fluid)


def test_monitor_records():
    from paper_2203_04508_gb300.monitor import Monitor
    sc = S.small_parity(fp64=False)
    lat = make_lattice(sc)
    buf = io.StringIO()
    mon = Monitor(lat, buf, every=40)
    recs = mon.run(100)
    assert [r["step"] for r in recs] == [40, 80, 100]
    lines = [json.loads(s) for s in buf.getvalue().splitlines()]
    assert lines == recs
    M, M0, dM = lat.mass()
    last = recs[-1]
    assert last["M"] == M and last["dM"] == dM and last["drift"] == (M - M0) / M0
    assert abs(last["drift"]) < 1e-6 and not last["nan"]
    assert last["max_speed"] == lat.max_speed() and 0 < last["max_speed"] < 0.2
    assert all(r["ms_per_step"] > 0 and r["mlups"] > 0 for r in recs)


def test_monitor_stops_at_a_blow_up():
    """The instability of the parity suite (no interface energy, sharp profile): the run ends
    with a record flagged NaN before the requested steps."""
    from paper_2203_04508_gb300.monitor import Monitor
    sc = S.small_parity(fp64=False).with_(k=1.0, kappa=0.0, width=1.0)
    lat = make_lattice(sc, fp64=False)
    mon = Monitor(lat, None, every=50)
    recs = mon.run(2000)
    assert recs[-1]["nan"] and mon.unstable
    assert recs[-1]["step"] < 2000
    assert not any(r["nan"] for r in recs[:-1])
