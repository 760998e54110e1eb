"""ctypes binding of liblbm_gb300.so: one Python function per entry point of include/lbm.h,
with the same name and argument order (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm_gb300.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ESTATE, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_EINTERNAL, LBM_ECORRUPT = range(9)
LBM_FP32, LBM_FP64 = 0, 1
LBM_FORCE_CHEMPOT, LBM_FORCE_PSEUDO = 0, 1
LBM_LAYOUT_AB, LBM_LAYOUT_AA = 0, 1


class lbm_config(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("walls", C.c_int32),
        ("y_bottom", C.c_double), ("y_top", C.c_double),
        ("eos", C.c_int32), ("a", C.c_double), ("b", C.c_double), ("R", C.c_double),
        ("T_over_Tc", C.c_double), ("omega", C.c_double), ("k", C.c_double), ("kappa", C.c_double),
        ("coll", C.c_int32), ("tau", C.c_double), ("s_e", C.c_double), ("s_eps", C.c_double),
        ("s_q", C.c_double), ("s_nu", C.c_double), ("gx", C.c_double), ("gy", C.c_double),
        ("bc", C.c_int32), ("precision", C.c_int32), ("rho_ref", C.c_double),
        ("n_cyl", C.c_int32), ("cx", C.POINTER(C.c_double)), ("cy", C.POINTER(C.c_double)),
        ("r", C.POINTER(C.c_double)), ("dmu_w", C.POINTER(C.c_double)), ("dmu_w_walls", C.c_double),
        ("force_model", C.c_int32), ("layout", C.c_int32),
    ]


class lbm_init_spec(C.Structure):
    _fields_ = [("n_drop", C.c_int32), ("x0", C.POINTER(C.c_double)), ("y0", C.POINTER(C.c_double)),
                ("r0", C.POINTER(C.c_double)), ("ux0", C.POINTER(C.c_double)),
                ("uy0", C.POINTER(C.c_double)), ("width", C.c_double)]


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"lbm status {status}: {msg}")
        self.status = status


_lib = None
P, I32, I64, D, SZ = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
_SIGS = {
    "lbm_workspace_size": (I32, [C.POINTER(lbm_config), C.POINTER(SZ)]),
    "lbm_create": (I32, [C.POINTER(lbm_config), P, P, SZ, C.POINTER(P)]),
    "lbm_build_links": (I32, [P]),
    "lbm_slab_workspace_size": (I32, [C.POINTER(lbm_config), I32, I32, I32, C.POINTER(SZ)]),
    "lbm_create_slab": (I32, [C.POINTER(lbm_config), I32, I32, I32, P, P, SZ, C.POINTER(P)]),
    "lbm_slab_info": (I32, [P, P]),
    "lbm_slab_message_bytes": (I32, [P, C.POINTER(SZ)]),
    "lbm_slab_pack": (I32, [P, I32, P, SZ]),
    "lbm_slab_unpack": (I32, [P, I32, P, SZ]),
    "lbm_counts": (I32, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)]),
    "lbm_get_links": (I32, [P, I64, P, P, P, P, P]),
    "lbm_get_kind": (I32, [P, P]),
    "lbm_init": (I32, [P, C.POINTER(lbm_init_spec)]),
    "lbm_step": (I32, [P, I64]),
    "lbm_prepare_steps": (I32, [P, I64]),
    "lbm_fields": (I32, [P, P, P, P, I32]),
    "lbm_populations": (I32, [P, P, I32]),
    "lbm_set_populations": (I32, [P, P, I32]),
    "lbm_mass": (I32, [P, C.POINTER(D), C.POINTER(D), C.POINTER(D)]),
    "lbm_dM_history": (I32, [P, P, I64, C.POINTER(I64)]),
    "lbm_eos_info": (I32, [P, P]),
    "lbm_last_dM": (I32, [P, C.POINTER(D)]),
    "lbm_profile_steps": (I32, [P, I64, P]),
    "lbm_launches_per_step": (I32, [P, C.POINTER(I64)]),
    "lbm_set_collide_kernel": (I32, [P, I32]),
    "lbm_set_spin_limit": (I32, [P, I64]),
    "lbm_set_mu_kernel": (I32, [P, I32]),
    "lbm_max_speed": (I32, [P, P]),
    "lbm_column_density": (I32, [P, I32, I32, I32, P, I32]),
    "lbm_last_dM_async": (I32, [P, P]),
    "lbm_save": (I32, [P, C.c_char_p]),
    "lbm_load": (I32, [P, C.c_char_p]),
    "lbm_get_collide_kernel": (I32, [P, C.POINTER(I32)]),
    "lbm_batch_workspace_size": (I32, [I32, P, C.POINTER(SZ)]),
    "lbm_batch_create": (I32, [I32, P, P, P, SZ, C.POINTER(P)]),
    "lbm_batch_build_links": (I32, [P]),
    "lbm_batch_init": (I32, [P, P]),
    "lbm_batch_step": (I32, [P, I64]),
    "lbm_batch_check": (I32, [P]),
    "lbm_batch_set_spin_limit": (I32, [P, I64]),
    "lbm_batch_instance": (I32, [P, I32, C.POINTER(P)]),
    "lbm_batch_set_tile": (I32, [P, I32]),
    "lbm_batch_set_schedule": (I32, [P, I32]),
    "lbm_batch_autotune": (I32, [P, I64, C.POINTER(I32), C.POINTER(I32), P]),
    "lbm_batch_info": (I32, [P, P]),
    "lbm_batch_last_error": (C.c_char_p, [P]),
    "lbm_batch_destroy": (None, [P]),
    "lbm_mass_noalloc": (I32, [P, P, I64, I32, P, P]),
    "lbm_adjoint_workspace_size": (I32, [P, I64, I64, C.POINTER(SZ)]),
    "lbm_forward_checkpointed": (I32, [P, I64, I64, P, SZ]),
    "lbm_objective": (I32, [P, I32, C.POINTER(D), P, I32]),
    "lbm_adjoint": (I32, [P, P, P, I32, P, P]),
    "lbm_destroy": (None, [P]),
    "lbm_status_str": (C.c_char_p, [I32]),
    "lbm_last_error": (C.c_char_p, [P]),
}


def load():
    """Loads the CUDA library; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(the package has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_symbols(header=None):
    """Names of the functions declared in include/lbm.h (for export checks)."""
    import re
    header = header or os.path.join(os.path.dirname(HERE), "include", "lbm.h")
    text = open(header).read()
    return sorted(set(re.findall(r"\b(lbm_[a-zA-Z0-9_]+)\s*\(", text)))


def check(status, ctx=None):
    if status != LBM_OK:
        lib = load()
        msg = lib.lbm_last_error(ctx).decode() if ctx else lib.lbm_status_str(status).decode()
        raise LbmError(status, msg)


def __getattr__(name):
    if name in _SIGS:
        return getattr(load(), name)
    raise AttributeError(name)
