"""ctypes binding of the C++ reference oracle (TEST INFRASTRUCTURE ONLY).

The oracle is compiled from ``lbm_oracle.cpp`` into ``liblbm_oracle.so`` next to this file,
with ``-ffp-contract=off`` so that the cut-link fractions q come out identically on every
host.  ``build()`` compiles it; it is also compiled on first use.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(HERE, "liblbm_oracle.so")
SOURCES = [os.path.join(HERE, "lbm_oracle.cpp"), os.path.join(HERE, "lbm_oracle.hpp")]

BC_PRESENT, BC_IBC, BC_MIBC, BC_HBB = 0, 1, 2, 3
EOS_NONE, EOS_CS, EOS_PR = 0, 1, 2
FORCE_CHEMPOT, FORCE_PSEUDO = 0, 1
COLL_BGK, COLL_MRT = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain g++, OpenMP, no FMA contraction)."""
    fresh = os.path.exists(SO_PATH) and all(
        os.path.getmtime(SO_PATH) >= os.path.getmtime(s) for s in SOURCES)
    if fresh and not force:
        return SO_PATH
    tmp = SO_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, SOURCES[0]]
    subprocess.run(cmd, check=True)
    os.replace(tmp, SO_PATH)
    return SO_PATH


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(SO_PATH)
    P, D, I, LL = C.c_void_p, C.c_double, C.c_int, C.c_longlong
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    u8p = C.POINTER(C.c_uint8)
    sig = {
        "orc_last_error": (C.c_char_p, []),
        "orc_set_threads": (None, [I]),
        "orc_get_threads": (I, []),
        "orc_create": (P, [P]),
        "orc_create_cs": (P, [P, I, I, D]),
        "orc_destroy": (None, [P]),
        "orc_init_droplets": (I, [P, P]),
        "orc_set_state": (I, [P, dp, dp, dp]),
        "orc_step": (I, [P, I]),
        "orc_num_links": (LL, [P]),
        "orc_get_links": (I, [P, ip, ip, dp, ip, ip]),
        "orc_get_kind": (I, [P, u8p, ip]),
        "orc_get_f": (I, [P, dp, dp]),
        "orc_set_f": (I, [P, dp]),
        "orc_get_fields": (I, [P, dp, dp, dp]),
        "orc_get_mu_force": (I, [P, dp, dp, dp]),
        "orc_mass": (D, [P]),
        "orc_mass0": (D, [P]),
        "orc_steps_done": (LL, [P]),
        "orc_dM_history": (I, [P, dp, I]),
        "orc_eos_info": (I, [P, dp]),
        "orc_eos_eval": (I, [P, I, dp, dp, dp, dp]),
        "orc_objective": (I, [P, I, dp, dp]),
        "orc_mrt_matrices": (None, [dp, dp]),
        "orc_lattice": (None, [ip, ip, dp, ip]),
        "orc_feq": (None, [D, D, D, dp]),
        "orc_meq": (None, [D, D, D, dp]),
        "orc_collide": (I, [P, dp, D, D, dp, dp]),
        "orc_link_value": (D, [I, D, D, D, I, D, D]),
        "orc_q_cylinder": (D, [I, I, I, D, D, D]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class _CConfig(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("walls", C.c_int32),
        ("y_bottom", C.c_double), ("y_top", C.c_double),
        ("eos", C.c_int32), ("a", C.c_double), ("b", C.c_double), ("R", C.c_double),
        ("T_over_Tc", C.c_double), ("omega", C.c_double), ("k", C.c_double), ("kappa", C.c_double),
        ("coll", C.c_int32), ("tau", C.c_double), ("s_e", C.c_double), ("s_eps", C.c_double),
        ("s_q", C.c_double), ("s_nu", C.c_double), ("gx", C.c_double), ("gy", C.c_double),
        ("bc", C.c_int32), ("n_cyl", C.c_int32),
        ("cx", C.POINTER(C.c_double)), ("cy", C.POINTER(C.c_double)),
        ("r", C.POINTER(C.c_double)), ("dmu_w", C.POINTER(C.c_double)),
        ("dmu_w_walls", C.c_double), ("force_model", C.c_int32),
    ]


class _CInit(C.Structure):
    _fields_ = [("n_drop", C.c_int32), ("x0", C.POINTER(C.c_double)), ("y0", C.POINTER(C.c_double)),
                ("r0", C.POINTER(C.c_double)), ("ux0", C.POINTER(C.c_double)),
                ("uy0", C.POINTER(C.c_double)), ("width", C.c_double)]


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


@dataclass
class OracleConfig:
    """Plain-data configuration of one lattice (mirrors the oracle's C struct)."""
    nx: int
    ny: int
    walls: int = 1
    y_bottom: float = 1.5
    y_top: float = -1.0          # default: ny - 2.5
    eos: int = EOS_CS
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    T_over_Tc: float = 0.7
    omega: float = 0.344
    k: float = 1.0
    kappa: float = 0.0
    coll: int = COLL_MRT
    tau: float = 0.8
    s_e: float = 1.64
    s_eps: float = 1.54
    s_q: float = 1.7
    s_nu: float = -1.0           # default: 1 / tau
    gx: float = 0.0
    gy: float = 0.0
    bc: int = BC_PRESENT
    cx: Sequence[float] = field(default_factory=list)
    cy: Sequence[float] = field(default_factory=list)
    r: Sequence[float] = field(default_factory=list)
    dmu_w: Sequence[float] = field(default_factory=list)
    dmu_w_walls: float = 0.0
    force_model: int = 0         # 0 chemical potential (Eqs. 9, 12), 1 pseudopotential

    def to_c(self):
        keep = {k: np.ascontiguousarray(np.asarray(getattr(self, k), dtype=np.float64).reshape(-1))
                for k in ("cx", "cy", "r", "dmu_w")}
        c = _CConfig()
        for name, _ in _CConfig._fields_:
            if name in keep:
                setattr(c, name, _dptr(keep[name]))
            elif name == "n_cyl":
                c.n_cyl = len(keep["r"])
            elif name == "y_top":
                c.y_top = self.y_top if self.y_top > 0 else self.ny - 2.5
            elif name == "s_nu":
                c.s_nu = self.s_nu if self.s_nu > 0 else 1.0 / self.tau
            else:
                setattr(c, name, getattr(self, name))
        return c, keep


def _check(st):
    if st != 0:
        raise RuntimeError("oracle: " + _load().orc_last_error().decode())


class Oracle:
    """One lattice advanced by the FP64 reference implementation."""

    def __init__(self, cfg: OracleConfig, cs_param: Optional[tuple] = None):
        lib = _load()
        self.cfg = cfg
        self.nx, self.ny = cfg.nx, cfg.ny
        c, keep = cfg.to_c()
        if cs_param is None:
            h = lib.orc_create(C.byref(c))
        else:
            param, body, step = cs_param
            h = lib.orc_create_cs(C.byref(c), int(param), int(body), float(step))
        if not h:
            raise ValueError("oracle: " + lib.orc_last_error().decode())
        self._h = h
        self._lib = lib

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_destroy(h)
            self._h = None

    # ---- set-up
    def init_droplets(self, x0, y0, r0, width, ux0=None, uy0=None):
        n = len(r0)
        arrs = [np.ascontiguousarray(np.asarray(v if v is not None else np.zeros(n), dtype=np.float64))
                for v in (x0, y0, r0, ux0, uy0)]
        s = _CInit(n, *[_dptr(a) for a in arrs], float(width))
        _check(self._lib.orc_init_droplets(self._h, C.byref(s)))

    def set_state(self, rho, ux, uy):
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1)) for a in (rho, ux, uy)]
        _check(self._lib.orc_set_state(self._h, *[_dptr(a) for a in arrs]))

    def step(self, n: int = 1):
        _check(self._lib.orc_step(self._h, int(n)))

    # ---- outputs
    def links(self):
        n = self._lib.orc_num_links(self._h)
        x1 = np.zeros(n, np.int32); d = np.zeros(n, np.int32); q = np.zeros(n, np.float64)
        x2 = np.zeros(n, np.int32); x2f = np.zeros(n, np.int32)
        ip = C.POINTER(C.c_int32)
        _check(self._lib.orc_get_links(self._h, x1.ctypes.data_as(ip), d.ctypes.data_as(ip), _dptr(q),
                                       x2.ctypes.data_as(ip), x2f.ctypes.data_as(ip)))
        return {"x1": x1, "dir": d, "q": q, "x2": x2, "x2_fluid": x2f}

    def kind(self):
        n = self.nx * self.ny
        k = np.zeros(n, np.uint8); b = np.zeros(n, np.int32)
        _check(self._lib.orc_get_kind(self._h, k.ctypes.data_as(C.POINTER(C.c_uint8)),
                                      b.ctypes.data_as(C.POINTER(C.c_int32))))
        return k.reshape(self.ny, self.nx), b.reshape(self.ny, self.nx)

    def populations(self, imag: bool = False):
        n = self.nx * self.ny
        f = np.zeros(9 * n); fi = np.zeros(9 * n) if imag else None
        _check(self._lib.orc_get_f(self._h, _dptr(f), _dptr(fi) if imag else None))
        f = f.reshape(9, self.ny, self.nx)
        return (f, fi.reshape(9, self.ny, self.nx)) if imag else f

    def set_populations(self, f):
        """Overwrite the populations (shape (9, ny, nx)); step count and M0 are kept."""
        a = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1))
        assert a.size == 9 * self.nx * self.ny
        _check(self._lib.orc_set_f(self._h, _dptr(a)))

    def fields(self):
        n = self.nx * self.ny
        r = np.zeros(n); vx = np.zeros(n); vy = np.zeros(n)
        _check(self._lib.orc_get_fields(self._h, _dptr(r), _dptr(vx), _dptr(vy)))
        sh = (self.ny, self.nx)
        return r.reshape(sh), vx.reshape(sh), vy.reshape(sh)

    def mu_force(self):
        """Chemical potential and force of the state last passed through fields()."""
        n = self.nx * self.ny
        m = np.zeros(n); fx = np.zeros(n); fy = np.zeros(n)
        _check(self._lib.orc_get_mu_force(self._h, _dptr(m), _dptr(fx), _dptr(fy)))
        sh = (self.ny, self.nx)
        return m.reshape(sh), fx.reshape(sh), fy.reshape(sh)

    def mass(self) -> float:
        return self._lib.orc_mass(self._h)

    def mass0(self) -> float:
        return self._lib.orc_mass0(self._h)

    def dM_history(self):
        n = self._lib.orc_steps_done(self._h)
        out = np.zeros(n)
        _check(self._lib.orc_dM_history(self._h, _dptr(out), int(n)))
        return out

    def objective(self, body: int = 0):
        """(J, imaginary part of J) of the droplet objective for cylinder `body`."""
        re, im = C.c_double(), C.c_double()
        _check(self._lib.orc_objective(self._h, int(body), C.byref(re), C.byref(im)))
        return re.value, im.value

    def eos_info(self):
        out = np.zeros(8)
        _check(self._lib.orc_eos_info(self._h, _dptr(out)))
        keys = ("Tc", "rho_c", "T", "alpha", "rho_g", "rho_l", "mu_sat", "p_sat")
        return dict(zip(keys, out.tolist()))


def set_threads(n: int):
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return _load().orc_get_threads()


def eos_eval(cfg: OracleConfig, rho):
    """Pressure p0 and bulk chemical potential psi'(rho) of cfg's EOS, plus the EOS summary."""
    lib = _load()
    c, keep = cfg.to_c()
    r = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(-1))
    p = np.zeros_like(r); m = np.zeros_like(r); info = np.zeros(8)
    _check(lib.orc_eos_eval(C.byref(c), len(r), _dptr(r), _dptr(p), _dptr(m), _dptr(info)))
    keys = ("Tc", "rho_c", "T", "alpha", "rho_g", "rho_l", "mu_sat", "p_sat")
    return p, m, dict(zip(keys, info.tolist()))


def lattice():
    lib = _load()
    ex = np.zeros(9, np.int32); ey = np.zeros(9, np.int32); w = np.zeros(9); opp = np.zeros(9, np.int32)
    ip = C.POINTER(C.c_int32)
    lib.orc_lattice(ex.ctypes.data_as(ip), ey.ctypes.data_as(ip), _dptr(w), opp.ctypes.data_as(ip))
    return ex, ey, w, opp


def mrt_matrices():
    lib = _load()
    M = np.zeros(81); Mi = np.zeros(81)
    lib.orc_mrt_matrices(_dptr(M), _dptr(Mi))
    return M.reshape(9, 9), Mi.reshape(9, 9)


def feq(rho, ux, uy):
    out = np.zeros(9)
    _load().orc_feq(float(rho), float(ux), float(uy), _dptr(out))
    return out


def meq(rho, jx, jy):
    out = np.zeros(9)
    _load().orc_meq(float(rho), float(jx), float(jy), _dptr(out))
    return out


def collide(cfg: OracleConfig, f9, Fx, Fy):
    c, keep = cfg.to_c()
    f = np.ascontiguousarray(np.asarray(f9, dtype=np.float64))
    out = np.zeros(9); Fi = np.zeros(9)
    _check(_load().orc_collide(C.byref(c), _dptr(f), float(Fx), float(Fy), _dptr(out), _dptr(Fi)))
    return out, Fi


def link_value(bc, q, a, b2, x2_fluid, c, F):
    return _load().orc_link_value(int(bc), float(q), float(a), float(b2), int(x2_fluid), float(c), float(F))


def q_cylinder(x, y, d, cx, cy, r):
    return _load().orc_q_cylinder(int(x), int(y), int(d), float(cx), float(cy), float(r))
