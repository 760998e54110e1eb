"""The non-allocating mass audit (lbm_mass_noalloc) agrees with lbm_mass.

lbm_mass_noalloc exists for callers that must not allocate device memory -- a host callback
or monitor, or a process whose device memory is owned by another allocator -- and keeps its
reduction scratch in a fixed array inside the library.  Here it audits the populations that
lbm_populations wrote into a device buffer, twice in a row (the second call reuses the
scratch the first one left behind), and both results must match the workspace-based audit of
the same state.  This file is collected last so that a failure here cannot hide the others.
"""
import ctypes as C

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


def _case(name):
    if name == "small":
        return S.small_parity()
    # 1024 x 512 = 524,288 nodes: twice the nodes the audit's capped grid of 1024 blocks of 256
    # threads covers in one pass, so every thread sums two strided chunks
    return S.c2_fp32_single(nx=1024, ny=512, n_cyl=4)


@pytest.mark.parametrize("case", ["small", "1024x512"])
@pytest.mark.parametrize("fp64", [False, True])
def test_noalloc_mass_matches_lbm_mass_twice(case, fp64):
    import torch
    from paper_2203_04508_gb300 import _abi
    lib = _abi.load()
    sc = _case(case)
    lat = make_lattice(sc, fp64=fp64)
    lat.step(50 if case == "small" else 20)
    M_ref, _, _ = lat.mass()
    n = sc.nx * sc.ny
    dtype = torch.float64 if fp64 else torch.float32
    f = torch.empty(9 * n, dtype=dtype, device="cuda")
    assert lib.lbm_populations(lat.ctx, C.c_void_p(f.data_ptr()), 1) == 0
    kind = torch.from_numpy(lat.kind().reshape(-1).copy()).to("cuda")
    lat.synchronize()
    prec = _abi.LBM_FP64 if fp64 else _abi.LBM_FP32
    results = []
    for _ in range(2):
        out = np.zeros(2)
        st = lib.lbm_mass_noalloc(C.c_void_p(f.data_ptr()), C.c_void_p(kind.data_ptr()), n, prec,
                                  C.c_void_p(lat.stream.cuda_stream), out.ctypes.data)
        assert st == 0
        results.append(out.copy())
    tol = 1e-12 if fp64 else 1e-6   # FP32: lbm_populations adds w_i rho_ref back in FP32
    for out in results:
        assert out[1] == 0.0
        assert out[0] == pytest.approx(M_ref, rel=tol)
    assert results[0][0] == results[1][0]


def test_noalloc_rejects_sizes_beyond_its_limit():
    from paper_2203_04508_gb300 import _abi
    lib = _abi.load()
    out = np.zeros(2)
    too_many = (1 << 30) + 1
    assert lib.lbm_mass_noalloc(C.c_void_p(256), C.c_void_p(256), too_many, 0, None, out.ctypes.data) == 1
    assert lib.lbm_mass_noalloc(C.c_void_p(256), C.c_void_p(256), 0, 0, None, out.ctypes.data) == 1


def test_noalloc_refuses_a_capturing_stream():
    """The call ends in a synchronising copy to host memory, which no capture can hold: on a
    stream that is capturing it returns LBM_ESTATE and issues nothing."""
    import torch
    from paper_2203_04508_gb300 import _abi
    lib = _abi.load()
    f = torch.zeros(9 * 64, dtype=torch.float32, device="cuda")
    kind = torch.zeros(64, dtype=torch.uint8, device="cuda")
    x = torch.zeros(4, device="cuda")
    out = np.zeros(2)
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        x.add_(1.0)
        st = lib.lbm_mass_noalloc(C.c_void_p(f.data_ptr()), C.c_void_p(kind.data_ptr()), 64, _abi.LBM_FP32,
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream), out.ctypes.data)
    assert st == _abi.LBM_ESTATE
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
    # outside the capture the same call runs
    st = lib.lbm_mass_noalloc(C.c_void_p(f.data_ptr()), C.c_void_p(kind.data_ptr()), 64, _abi.LBM_FP32, None,
                              out.ctypes.data)
    assert st == 0 and out[0] == 0.0 and out[1] == 0.0
