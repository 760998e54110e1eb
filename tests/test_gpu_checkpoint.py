"""Checkpoint / resume through the C ABI (lbm_save, lbm_load): a run saved half-way and resumed
in a fresh context gives the bits of the run that went straight through (populations, mass, the
per-step compensation history); damaged files and checkpoints of another configuration are
refused with the documented status and leave the context usable."""
from __future__ import annotations

import os

import numpy as np
import pytest

import scenarios as S
from harness import make_lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_04508_gb300 import build
    build.build()


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("split", [500, 501])
def test_resume_is_bit_identical(tmp_path, fp64, split):
    sc = S.small_parity(fp64=fp64)
    n = 1000
    straight = make_lattice(sc)
    straight.step(n)
    first = make_lattice(sc)
    first.step(split)
    path = os.path.join(tmp_path, "state.ckpt")
    first.save(path)
    resumed = make_lattice(sc, init=False)
    resumed.load(path)
    resumed.step(n - split)
    assert np.array_equal(resumed.populations(), straight.populations())
    assert resumed.mass() == straight.mass()
    assert np.array_equal(resumed.dM_history(n), straight.dM_history(n))


def test_resume_with_the_tma_pipelined_kernel(tmp_path):
    """A 1024 x 2048 impact lattice stepped by the TMA-pipelined collide kernel."""
    sc = S.c3_impact(1024, 2048)
    a = make_lattice(sc, fp64=False)
    a.set_collide_kernel(1)
    a.step(300)
    path = os.path.join(tmp_path, "big.ckpt")
    a.save(path)
    a.step(200)
    b = make_lattice(sc, fp64=False, init=False)
    b.set_collide_kernel(1)
    b.load(path)
    b.step(200)
    assert np.array_equal(a.populations(), b.populations())


def test_damaged_and_foreign_checkpoints_are_refused(tmp_path):
    import paper_2203_04508_gb300 as G
    from paper_2203_04508_gb300 import _abi
    sc = S.small_parity()
    lat = make_lattice(sc)
    lat.step(20)
    path = os.path.join(tmp_path, "good.ckpt")
    lat.save(path)
    raw = open(path, "rb").read()
    cases = {"truncated": raw[: len(raw) // 2], "altered": bytearray(raw), "not a checkpoint": b"x" * len(raw)}
    cases["altered"][len(raw) // 3] ^= 0x10
    target = make_lattice(sc, init=False)
    for name, data in cases.items():
        bad = os.path.join(tmp_path, name.replace(" ", "_") + ".ckpt")
        open(bad, "wb").write(bytes(data))
        with pytest.raises(G.LbmError) as e:
            target.load(bad)
        assert e.value.args[0].startswith(f"lbm status {_abi.LBM_ECORRUPT}"), (name, e.value)
    other = make_lattice(sc.with_(dmu_w=[0.0, 0.0]), init=False)
    with pytest.raises(G.LbmError) as e:
        other.load(path)
    assert e.value.args[0].startswith(f"lbm status {_abi.LBM_EINVAL}")
    with pytest.raises(G.LbmError):
        target.load(os.path.join(tmp_path, "missing.ckpt"))
    # the refusals leave the context usable
    target.load(path)
    target.step(5)
    lat.step(5)
    assert np.array_equal(target.populations(), lat.populations())
