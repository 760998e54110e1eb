"""Host-side checks of the CUDA library's C ABI that need no GPU: it loads, exports every
function include/lbm.h declares, validates configurations, and its own FP64 EOS set-up agrees
with the oracle's (two independent solvers: Newton on the saturation pressure versus nested
bisection)."""
import ctypes as C
import os

import numpy as np
import pytest

import scenarios as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    from paper_2203_04508_gb300 import build as B
    B.build()
    from paper_2203_04508_gb300 import _abi
    return _abi


def _create(abi, phys, precision=0):
    from paper_2203_04508_gb300.lattice import make_config
    c, keep = make_config(phys, precision)
    n = C.c_size_t()
    st = abi.load().lbm_workspace_size(C.byref(c), C.byref(n))
    ctx = C.c_void_p()
    # lbm_create does no device work: a fake, aligned, large-enough address is accepted
    st2 = abi.load().lbm_create(C.byref(c), None, C.c_void_p(1 << 20), n.value, C.byref(ctx))
    return st, st2, ctx, n.value, keep


def test_library_exports_every_declared_symbol(abi):
    lib = abi.load()
    names = abi.declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_header_is_plain_c(abi):
    """include/lbm.h is a C header (no C++ types or torch types): it compiles as C99 and as
    C++, and every call it declares is bound with the same name in the Python binding."""
    import shutil
    import subprocess
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lbm.h")
    for cc, lang, std in (("gcc", "c", "-std=c99"), ("g++", "c++", "-std=c++17")):
        if shutil.which(cc) is None:
            pytest.skip(f"{cc} not found")
        r = subprocess.run([cc, "-fsyntax-only", "-x", lang, std, "-Wall", "-Wextra", "-Werror", hdr],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
    bound = set(abi._SIGS)
    missing = [n for n in abi.declared_symbols() if n not in bound]
    assert not missing, missing


def test_workspace_and_eos_match_the_oracle(abi):
    import oracle as O
    for sc in (S.c1_plain_fp64(), S.small_parity(), S.c3_impact(256, 512)):
        st, st2, ctx, n, keep = _create(abi, sc.physics())
        assert st == 0 and st2 == 0, abi.load().lbm_last_error(ctx)
        assert n > 9 * 2 * 4 * sc.nx * sc.ny
        out = np.zeros(8)
        abi.load().lbm_eos_info(ctx, out.ctypes.data)
        abi.load().lbm_destroy(ctx)
        o = O.Oracle(O.OracleConfig(**sc.physics()))
        info = o.eos_info()
        for k, key in enumerate(("Tc", "rho_c", "T", "alpha", "rho_g", "rho_l", "mu_sat", "p_sat")):
            tol = 1e-6 if key == "rho_c" else 1e-12
            assert out[k] == pytest.approx(info[key], rel=tol, abs=1e-15), key


def test_peng_robinson_set_up_matches_the_oracle(abi):
    import oracle as O
    phys = S.small_parity().physics()
    phys.update(eos=S.EOS_PR, a=2 / 49, b=2 / 21, T_over_Tc=0.7)
    st, st2, ctx, n, keep = _create(abi, phys)
    assert st2 == 0
    out = np.zeros(8)
    abi.load().lbm_eos_info(ctx, out.ctypes.data)
    abi.load().lbm_destroy(ctx)
    _, _, info = O.eos_eval(O.OracleConfig(**phys), [1.0])
    assert out[4] == pytest.approx(info["rho_g"], rel=1e-12)
    assert out[5] == pytest.approx(info["rho_l"], rel=1e-12)


@pytest.mark.parametrize("patch", [
    dict(y_bottom=2.5), dict(y_top=10.0), dict(nx=4), dict(coll=0, tau=0.5), dict(s_nu=2.5),
    dict(cx=[1.0]), dict(eos=7), dict(bc=9), dict(k=0.0), dict(force_model=2), dict(nx=20001, ny=10000),
    dict(force_model=1, dmu_w_walls=-1.0), dict(force_model=1, dmu_w=[-1.5, 0.1]),
])
def test_invalid_configurations_are_rejected(abi, patch):
    phys = S.small_parity().physics()
    phys.update(patch)
    if "cx" in patch:
        phys.update(cy=[phys["cy"][0]], r=[phys["r"][0]], dmu_w=[0.0])
    st, st2, ctx, n, keep = _create(abi, phys)
    assert st == abi.LBM_EINVAL
    if ctx:
        abi.load().lbm_destroy(ctx)


def test_small_workspace_and_call_order(abi):
    from paper_2203_04508_gb300.lattice import make_config
    lib = abi.load()
    c, keep = make_config(S.small_parity().physics(), 0)
    n = C.c_size_t()
    assert lib.lbm_workspace_size(C.byref(c), C.byref(n)) == 0
    ctx = C.c_void_p()
    assert lib.lbm_create(C.byref(c), None, C.c_void_p(1 << 20), n.value - 256, C.byref(ctx)) == abi.LBM_ENOMEM
    lib.lbm_destroy(ctx)
    ctx = C.c_void_p()
    assert lib.lbm_create(C.byref(c), None, C.c_void_p((1 << 20) + 8), n.value, C.byref(ctx)) == abi.LBM_EINVAL
    lib.lbm_destroy(ctx)
    ctx = C.c_void_p()
    assert lib.lbm_create(C.byref(c), None, C.c_void_p(1 << 20), n.value, C.byref(ctx)) == 0
    assert lib.lbm_step(ctx, 1) == abi.LBM_ESTATE          # before lbm_build_links / lbm_init
    m = C.c_double()
    assert lib.lbm_mass(ctx, C.byref(m), None, None) == abi.LBM_ESTATE
    assert lib.lbm_max_speed(ctx, C.byref(m)) == abi.LBM_ESTATE   # before lbm_init
    assert lib.lbm_set_spin_limit(ctx, 0) == abi.LBM_ESTATE       # before lbm_build_links
    assert lib.lbm_set_mu_kernel(ctx, 1) == abi.LBM_ESTATE
    assert lib.lbm_max_speed(None, C.byref(m)) == abi.LBM_ESTATE
    lib.lbm_destroy(ctx)


def test_pseudopotential_batches_are_rejected(abi):
    """The batched kernel runs the chemical-potential force only: a batch with a
    pseudopotential instance is refused before any device work."""
    from paper_2203_04508_gb300.lattice import make_config
    lib = abi.load()
    phys = S.small_parity(T_over_Tc=0.7).physics()
    good, k1 = make_config(phys, 0)
    phys.update(force_model=1, k=1.0, kappa=0.0, dmu_w=[0.15, -0.15])
    pp, k2 = make_config(phys, 0)
    n = C.c_size_t()
    assert lib.lbm_workspace_size(C.byref(pp), C.byref(n)) == 0
    arr = (abi.lbm_config * 2)(good, pp)
    assert lib.lbm_batch_workspace_size(2, arr, C.byref(n)) == abi.LBM_EINVAL
    arr = (abi.lbm_config * 2)(good, good)
    assert lib.lbm_batch_workspace_size(2, arr, C.byref(n)) == 0


def test_the_largest_lattice_is_accepted(abi):
    """2e8 nodes (32-bit plane offsets) is the largest lattice: one node more is refused."""
    from paper_2203_04508_gb300.lattice import make_config
    lib = abi.load()
    phys = S.Scenario(name="big", nx=20000, ny=10000, walls=0).physics()
    c, keep = make_config(phys, 0)
    n = C.c_size_t()
    assert lib.lbm_workspace_size(C.byref(c), C.byref(n)) == 0
    assert n.value > 2 * 9 * 4 * 20000 * 10000
    phys.update(nx=20001)
    c, keep = make_config(phys, 0)
    assert lib.lbm_workspace_size(C.byref(c), C.byref(n)) == abi.LBM_EINVAL
