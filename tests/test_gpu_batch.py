"""The batched persistent step: many lattices of different sizes and physics advanced by one
cooperative kernel per call must reproduce each lattice stepped on its own, match the oracle,
and report a grid-barrier timeout instead of hanging."""
import numpy as np
import pytest

import scenarios as S
from harness import compare, make_lattice, make_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_04508_gb300 import build
    build.build()


def _mixed(fp64=False):
    """Four unlike instances: ragged sizes, two temperatures, MRT and BGK, walls and a periodic
    box, one to two cylinders."""
    return [
        S.small_parity(seed=7, fp64=fp64),
        S.small_parity(seed=11, nx=97, ny=83, fp64=fp64, T_over_Tc=0.7),
        S.c1_plain_fp64().with_(fp64=fp64, dmu_w=[-0.03]),
        S.Scenario(name="free", nx=61, ny=53, walls=0, T_over_Tc=0.8, coll=S.COLL_BGK, tau=1.0,
                   cx=[30.41], cy=[26.77], r=[9.3], dmu_w=[0.02], x0=[30.41], y0=[38.0], r0=[6.0], fp64=fp64),
    ]


def _batch(scs, fp64):
    import paper_2203_04508_gb300 as G
    b = G.Batch([sc.physics() for sc in scs], precision=G.LBM_FP64 if fp64 else G.LBM_FP32)
    b.init([sc.droplets() for sc in scs])
    return b


@pytest.mark.parametrize("fp64", [False, True])
def test_batch_equals_each_lattice_stepped_alone(fp64):
    scs = _mixed(fp64)
    b = _batch(scs, fp64)
    b.step(57)
    b.check()
    tol = 0.0 if fp64 else 1e-6
    for k, sc in enumerate(scs):
        single = make_lattice(sc, fp64=fp64)
        single.step(57)
        fb, fs = b.instances[k].populations(), single.populations()
        scale = np.abs(fs).max()
        assert np.abs(fb.astype(np.float64) - fs).max() <= max(tol, 1e-13) * scale, sc.name
        # the per-step compensation sums are cancelling sums of (f~ - f) over links: in FP32 the
        # two kernels' roundings (contracted differently by the compiler) show at 1e-6 there
        hb, hs = b.instances[k].dM_history(57), single.dM_history(57)
        assert np.allclose(hb, hs, rtol=1e-9 if fp64 else 1e-4, atol=1e-12 if fp64 else 1e-7), sc.name
        Mb, M0b, _ = b.instances[k].mass()
        assert abs(Mb / M0b - 1) < (1e-12 if fp64 else 1e-6)


@pytest.mark.parametrize("fp64", [False, True])
def test_batch_in_aa_order_equals_the_two_lattice_batch(fp64):
    """Instances that each keep one population lattice in AA order, advanced by the batched
    kernel (in-place and pulled collides, shifted-order density, the boundary moments saved in
    the second solid layer's phase): the two-lattice batch's values bit for bit, after odd and
    even step counts, in less workspace."""
    import paper_2203_04508_gb300 as G
    scs = _mixed(fp64)
    prec = G.LBM_FP64 if fp64 else G.LBM_FP32
    a = G.Batch([sc.physics() for sc in scs], precision=prec)
    c = G.Batch([sc.physics() for sc in scs], precision=prec, layout=G.LBM_LAYOUT_AA)
    assert c.workspace.numel() < a.workspace.numel()
    for b in (a, c):
        b.init([sc.droplets() for sc in scs])
    for n in (1, 4, 9):
        a.step(n)
        c.step(n)
        a.check()
        c.check()
        for k, sc in enumerate(scs):
            fa, fc = a.instances[k].populations(), c.instances[k].populations()
            assert np.array_equal(fa, fc), (sc.name, n)
            assert a.instances[k].mass() == c.instances[k].mass(), (sc.name, n)
            assert np.array_equal(a.instances[k].dM_history(), c.instances[k].dM_history()), (sc.name, n)


def test_fp64_batch_matches_the_oracle():
    scs = _mixed(True)
    b = _batch(scs, True)
    b.step(40)
    b.check()
    for k, sc in enumerate(scs):
        orc = make_oracle(sc)
        orc.step(40)
        er, ev, ef = compare(b.instances[k], orc)
        assert ef < 1e-11 and er < 1e-11, (sc.name, er, ev, ef)


def test_consecutive_calls_and_odd_step_counts():
    scs = _mixed(False)[:2]
    a, c = _batch(scs, False), _batch(scs, False)
    a.step(7)
    a.step(6)
    c.step(13)
    a.check()
    c.check()
    for k in range(2):
        assert np.array_equal(a.instances[k].populations(), c.instances[k].populations())


def test_grid_barrier_timeout_is_reported_not_hung():
    """With a zero poll budget every barrier wait gives up at once: the kernel leaves early and
    the host sees LBM_ETIMEOUT; restoring the budget and re-initialising works again."""
    from paper_2203_04508_gb300 import LbmError
    scs = _mixed(False)[:2]
    b = _batch(scs, False)
    info = b.info()
    if info["grid"] < 2:
        pytest.skip("a one-block grid never waits")
    b.set_spin_limit(0)
    b.step(3)
    with pytest.raises(LbmError) as e:
        b.check()
    assert e.value.status == 6
    b.set_spin_limit(1 << 22)
    b.init([sc.droplets() for sc in scs])
    b.step(3)
    b.check()


def test_every_tile_shape_gives_identical_results():
    """The node-tile shape is a scheduling choice only: FP64 populations after 23 steps are the
    same bits for every shape."""
    scs = _mixed(True)
    b = _batch(scs, True)
    ref = None
    for log2w in (5, 4, 6, 7, 8):
        b.set_tile(log2w)
        b.init([sc.droplets() for sc in scs])
        b.step(23)
        b.check()
        pops = [inst.populations() for inst in b.instances]
        if ref is None:
            ref = pops
        else:
            for k in range(len(scs)):
                assert np.array_equal(pops[k], ref[k]), (log2w, k)


def test_both_schedules_give_identical_results():
    """Lockstep and the two-group skewed schedule run each instance's phases in the same
    order: FP64 populations and compensation histories after 31 steps are the same bits, and
    so are the oracle's."""
    scs = _mixed(True)
    b = _batch(scs, True)
    ref = None
    for groups in (1, 2, 1):
        b.set_schedule(groups)
        b.init([sc.droplets() for sc in scs])
        b.step(31)
        b.check()
        got = [(inst.populations(), inst.dM_history(31)) for inst in b.instances]
        if ref is None:
            ref = got
        else:
            for k in range(len(scs)):
                assert np.array_equal(got[k][0], ref[k][0]), (groups, k)
                assert np.array_equal(got[k][1], ref[k][1]), (groups, k)
    b.set_schedule(2)
    b.init([sc.droplets() for sc in scs])
    b.step(40)
    b.check()
    for k, sc in enumerate(scs):
        orc = make_oracle(sc)
        orc.step(40)
        er, ev, ef = compare(b.instances[k], orc)
        assert ef < 1e-11 and er < 1e-11, (sc.name, er, ev, ef)


def test_autotune_picks_a_shape_and_the_batch_stays_correct():
    from paper_2203_04508_gb300 import LbmError
    scs = _mixed(False)
    b = _batch(scs, False)
    r = b.autotune(3)
    assert 4 <= r["log2w"] <= 8 and r["groups"] in (1, 2)
    assert all(v > 0 for v in r["ms"].values())
    tiles = {k: v for k, v in r["ms"].items() if "x" in k}
    assert r["ms"][r["tile"]] == min(tiles.values())
    sched = r["ms"]["lockstep"], r["ms"]["two groups"]
    assert sched[r["groups"] - 1] == min(sched)
    b.init([sc.droplets() for sc in scs])
    b.step(17)
    b.check()
    for k, sc in enumerate(scs):
        single = make_lattice(sc, fp64=False)
        single.step(17)
        fb, fs = b.instances[k].populations(), single.populations()
        assert np.abs(fb.astype(np.float64) - fs).max() <= 1e-6 * np.abs(fs).max(), sc.name
    with pytest.raises(LbmError):
        b.set_tile(3)
    with pytest.raises(LbmError):
        b.set_schedule(3)


def test_full_size_c4_batch_matches_single_instances():
    """The benchmark's batch -- 256 instances of 128^2..768^2, FP32, default tile and schedule --
    after 10 steps: the smallest, median and largest instance against the same lattice stepped
    on its own (the per-node arithmetic is shared, so only the compiled kernels' FP32 rounding
    may differ), and every instance's mass."""
    import torch
    scs = S.c4_batch()
    b = _batch(scs, False)
    b.step(10)
    b.check()
    order = sorted(range(len(scs)), key=lambda k: scs[k].nodes)
    for k in (order[0], order[len(order) // 2], order[-1]):
        single = make_lattice(scs[k], fp64=False)
        single.step(10)
        fb, fs = b.instances[k].populations(), single.populations()
        assert np.abs(fb.astype(np.float64) - fs).max() <= 1e-6 * np.abs(fs).max(), scs[k].name
        del single
    for k in range(len(scs)):
        M, M0, _ = b.instances[k].mass()
        assert abs(M / M0 - 1) < 1e-6, scs[k].name
    del b
    torch.cuda.empty_cache()
