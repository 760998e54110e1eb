"""Python front end of one lattice: device workspace and stream from PyTorch, every step of
the method in the CUDA library (through the C ABI of include/lbm.h)."""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import _abi
from ._abi import check, lbm_config, lbm_init_spec

_PHYS_KEYS = ("nx", "ny", "walls", "y_bottom", "y_top", "eos", "a", "b", "R", "T_over_Tc", "omega", "k",
              "kappa", "coll", "tau", "s_e", "s_eps", "s_q", "s_nu", "gx", "gy", "bc", "dmu_w_walls")


def make_config(phys: dict, precision: int, rho_ref: float = -1.0, layout: int = _abi.LBM_LAYOUT_AB):
    """lbm_config from a plain dict of physical parameters; returns (struct, keep-alive arrays).
    layout: LBM_LAYOUT_AB (two population lattices) or LBM_LAYOUT_AA (one, updated in place)."""
    keep = {k: np.ascontiguousarray(np.asarray(phys.get(k, []), dtype=np.float64).reshape(-1))
            for k in ("cx", "cy", "r", "dmu_w")}
    c = lbm_config()
    for k in _PHYS_KEYS:
        setattr(c, k, phys[k])
    c.force_model = int(phys.get("force_model", 0))
    c.layout = int(layout)
    c.precision = precision
    c.rho_ref = rho_ref
    c.n_cyl = len(keep["r"])
    for k, a in keep.items():
        setattr(c, k, a.ctypes.data_as(C.POINTER(C.c_double)))
    return c, keep


def workspace_size(phys: dict, precision: int, layout: int = _abi.LBM_LAYOUT_AB) -> int:
    c, keep = make_config(phys, precision, layout=layout)
    n = C.c_size_t()
    check(_abi.load().lbm_workspace_size(C.byref(c), C.byref(n)))
    return n.value


class Lattice:
    """One lattice on the current CUDA device."""

    def __init__(self, phys: dict, precision: int = _abi.LBM_FP32, rho_ref: float = -1.0,
                 stream=None, build: bool = True, layout: int = _abi.LBM_LAYOUT_AB):
        import torch
        lib = _abi.load()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.lib = lib
        self.nx, self.ny = int(phys["nx"]), int(phys["ny"])
        self.precision = precision
        self.dtype = np.float64 if precision == _abi.LBM_FP64 else np.float32
        self.tdtype = torch.float64 if precision == _abi.LBM_FP64 else torch.float32
        self.layout = int(layout)
        self._cfg, self._keep = make_config(phys, precision, rho_ref, layout)
        n = C.c_size_t()
        check(lib.lbm_workspace_size(C.byref(self._cfg), C.byref(n)))
        self.workspace = torch.empty(n.value, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.Stream()
        ctx = C.c_void_p()
        st = lib.lbm_create(C.byref(self._cfg), C.c_void_p(self.stream.cuda_stream),
                            C.c_void_p(self.workspace.data_ptr()), n.value, C.byref(ctx))
        self.ctx = ctx
        if st != _abi.LBM_OK:
            msg = lib.lbm_last_error(ctx).decode() if ctx else ""
            if ctx:
                lib.lbm_destroy(ctx)
                self.ctx = None
            raise _abi.LbmError(st, msg)
        if build:
            self.build_links()

    def __del__(self):
        if getattr(self, "ctx", None):
            self.lib.lbm_destroy(self.ctx)
            self.ctx = None

    def _c(self, st):
        check(st, self.ctx)

    # ---- set-up
    def build_links(self):
        self._c(self.lib.lbm_build_links(self.ctx))

    def counts(self):
        v = [C.c_int64() for _ in range(5)]
        self._c(self.lib.lbm_counts(self.ctx, *[C.byref(x) for x in v]))
        return dict(zip(("links", "boundary_nodes", "fluid", "solid1", "solid2"), [x.value for x in v]))

    def links(self):
        n = self.counts()["links"]
        x1 = np.zeros(n, np.int32); d = np.zeros(n, np.int32); q = np.zeros(n, np.float64)
        x2 = np.zeros(n, np.int32); f2 = np.zeros(n, np.int32)
        self._c(self.lib.lbm_get_links(self.ctx, n, x1.ctypes.data, d.ctypes.data, q.ctypes.data,
                                       x2.ctypes.data, f2.ctypes.data))
        return {"x1": x1, "dir": d, "q": q, "x2": x2, "x2_fluid": f2}

    def kind(self):
        k = np.zeros((self.ny, self.nx), np.uint8)
        self._c(self.lib.lbm_get_kind(self.ctx, k.ctypes.data))
        return k

    def init(self, x0, y0, r0, width, ux0=None, uy0=None):
        n = len(r0)
        arrs = [np.ascontiguousarray(np.asarray(v if v is not None else np.zeros(n), np.float64))
                for v in (x0, y0, r0, ux0, uy0)]
        self._init_keep = arrs
        s = lbm_init_spec(n, *[a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs], float(width))
        self._c(self.lib.lbm_init(self.ctx, C.byref(s)))

    def init_droplets(self, d: dict):
        self.init(d["x0"], d["y0"], d["r0"], d["width"], d.get("ux0"), d.get("uy0"))

    # ---- time stepping
    def step(self, n: int = 1):
        self._c(self.lib.lbm_step(self.ctx, int(n)))

    def prepare_steps(self, n: int):
        """Captures the step graphs step(n) will launch, without running them (lbm_prepare_steps)."""
        self._c(self.lib.lbm_prepare_steps(self.ctx, int(n)))

    def synchronize(self):
        self.stream.synchronize()

    # ---- read-outs
    def fields(self, on_device: bool = False, out=None):
        """(rho, vx, vy) of the current state, as numpy arrays (host) or torch tensors.  `out`:
        three caller-owned host tensors of shape (ny, nx) in the lattice's precision, ideally
        page-locked, which the library fills (and which are returned)."""
        import torch
        if out is not None:
            for t in out:
                if tuple(t.shape) != (self.ny, self.nx) or t.dtype != self.tdtype or t.is_cuda or not t.is_contiguous():
                    raise ValueError("out: three contiguous host tensors of shape (ny, nx) in the lattice's precision")
            self._c(self.lib.lbm_fields(self.ctx, *[C.c_void_p(t.data_ptr()) for t in out], 0))
            return tuple(out)
        if on_device:
            out = [torch.empty((self.ny, self.nx), dtype=self.tdtype, device="cuda") for _ in range(3)]
            self.stream.wait_stream(torch.cuda.current_stream())
            self._c(self.lib.lbm_fields(self.ctx, *[C.c_void_p(t.data_ptr()) for t in out], 1))
            torch.cuda.current_stream().wait_stream(self.stream)
            return tuple(out)
        out = [np.zeros((self.ny, self.nx), self.dtype) for _ in range(3)]
        self._c(self.lib.lbm_fields(self.ctx, *[o.ctypes.data for o in out], 0))
        return tuple(out)

    def populations(self):
        f = np.zeros((9, self.ny, self.nx), self.dtype)
        self._c(self.lib.lbm_populations(self.ctx, f.ctypes.data, 0))
        return f

    def set_populations(self, f):
        """New initial state from absolute populations (9 x ny x nx, numpy array or torch
        tensor on the device)."""
        import torch
        if isinstance(f, torch.Tensor):
            t = f.detach().to(device="cuda", dtype=self.tdtype).contiguous()
            self.stream.wait_stream(torch.cuda.current_stream())
            self._c(self.lib.lbm_set_populations(self.ctx, C.c_void_p(t.data_ptr()), 1))
        else:
            a = np.ascontiguousarray(np.asarray(f, self.dtype))
            self._c(self.lib.lbm_set_populations(self.ctx, a.ctypes.data, 0))

    def mass(self):
        m, m0, dm = C.c_double(), C.c_double(), C.c_double()
        self._c(self.lib.lbm_mass(self.ctx, C.byref(m), C.byref(m0), C.byref(dm)))
        return m.value, m0.value, dm.value

    def dM_history(self, n: int = 4096):
        out = np.zeros(n)
        k = C.c_int64()
        self._c(self.lib.lbm_dM_history(self.ctx, out.ctypes.data, n, C.byref(k)))
        return out[:k.value]

    def last_dM(self) -> float:
        d = C.c_double()
        self._c(self.lib.lbm_last_dM(self.ctx, C.byref(d)))
        return d.value

    def save(self, path: str):
        """Checkpoint of the current state (see lbm_save)."""
        self._c(self.lib.lbm_save(self.ctx, str(path).encode()))

    def load(self, path: str):
        """Restores a checkpoint written by save() for the same configuration (in place of init)."""
        self._c(self.lib.lbm_load(self.ctx, str(path).encode()))

    def last_dM_async(self, out, index: int = 0):
        """Queues the last step's compensation sum into element `index` of the FP64 host tensor
        `out` (page-locked for the copy to overlap the next steps); valid after synchronize()."""
        self._c(self.lib.lbm_last_dM_async(self.ctx, C.c_void_p(out.data_ptr() + 8 * int(index))))

    def profile_steps(self, n: int):
        """Per-phase device time (ms) summed over n steps: rho, solid, mu, collide, bc."""
        ms = np.zeros(5)
        self._c(self.lib.lbm_profile_steps(self.ctx, int(n), ms.ctypes.data))
        return ms

    def eos_info(self):
        o = np.zeros(8)
        self._c(self.lib.lbm_eos_info(self.ctx, o.ctypes.data))
        return dict(zip(("Tc", "rho_c", "T", "alpha", "rho_g", "rho_l", "mu_sat", "p_sat"), o.tolist()))

    def column_density(self, x: int, y0: int = 0, n: Optional[int] = None) -> np.ndarray:
        """Density of the nodes (x, y0 .. y0+n-1) of the current state (NaN at solid nodes)."""
        n = self.ny - y0 if n is None else n
        out = np.empty(n, np.float64)
        self._c(self.lib.lbm_column_density(self.ctx, int(x), int(y0), int(n), C.c_void_p(out.ctypes.data), 0))
        return out

    def max_speed(self) -> float:
        """Largest |v| over the fluid nodes of the current state (NaN if one is not a number)."""
        v = C.c_double()
        self._c(self.lib.lbm_max_speed(self.ctx, C.byref(v)))
        return v.value

    def set_collide_kernel(self, kind: int):
        """0: the plain collide kernel; 1: the TMA-pipelined one (FP32); 2: the TMA-pipelined column
        sweeps that also form the next state's density (FP32, chemical-potential force, lattices of
        whole 32 x 8 tiles; slower on GB300, so never the default).  lbm_build_links picks 1 on large
        lattices, 0 otherwise."""
        self._c(self.lib.lbm_set_collide_kernel(self.ctx, int(kind)))

    def set_mu_kernel(self, kind: int):
        """Chemical-potential pass: 0 per node, 1 row vectors, 2 row sweeps (FP32); same bits."""
        self._c(self.lib.lbm_set_mu_kernel(self.ctx, int(kind)))

    def set_spin_limit(self, polls: int):
        """Polls before the pipelined kernel's waits give up (0: at once, to test that path)."""
        self._c(self.lib.lbm_set_spin_limit(self.ctx, int(polls)))

    def collide_kernel(self) -> int:
        k = C.c_int32()
        self._c(self.lib.lbm_get_collide_kernel(self.ctx, C.byref(k)))
        return k.value

    def launches_per_step(self) -> int:
        n = C.c_int64()
        self._c(self.lib.lbm_launches_per_step(self.ctx, C.byref(n)))
        return n.value

    # ---- objective and reverse mode
    @property
    def n_params(self) -> int:
        """Length of the parameter gradient: dmu_w per cylinder, dmu_w of the walls, (cx, cy)
        per cylinder."""
        return 3 * int(self._cfg.n_cyl) + 1

    def objective(self, body: int = 0, seed: bool = False):
        """Droplet objective J of the current state for cylinder `body`; with seed=True also
        dJ/drho (ny x nx torch tensor on the device, zero off the fluid)."""
        import torch
        J = C.c_double()
        out = None
        if seed:
            out = torch.empty((self.ny, self.nx), dtype=self.tdtype, device="cuda")
            self.stream.wait_stream(torch.cuda.current_stream())
        self._c(self.lib.lbm_objective(self.ctx, int(body), C.byref(J),
                                       C.c_void_p(out.data_ptr()) if seed else None, 1))
        return (J.value, out) if seed else J.value

    def adjoint_workspace_size(self, n: int, every: int = 0) -> int:
        b = C.c_size_t()
        self._c(self.lib.lbm_adjoint_workspace_size(self.ctx, int(n), int(every), C.byref(b)))
        return b.value

    def forward_checkpointed(self, n: int, every: int = 0):
        """Advances n steps keeping checkpoints every `every` steps (0: about sqrt(n)) in a
        device workspace held by this object until the next call."""
        import torch
        size = self.adjoint_workspace_size(n, every)
        if getattr(self, "_tape", None) is None or self._tape.numel() < size:
            self._tape = None
            self._tape = torch.empty(size, dtype=torch.uint8, device="cuda")
        self.stream.wait_stream(torch.cuda.current_stream())
        self._c(self.lib.lbm_forward_checkpointed(self.ctx, int(n), int(every),
                                                  C.c_void_p(self._tape.data_ptr()), self._tape.numel()))

    def adjoint(self, drho=None, df=None, want_df0: bool = False):
        """Reverse sweep through the last forward_checkpointed.  drho (ny x nx) and df
        (9 x ny x nx) are torch tensors of dJ/d(final state), either may be None.  Returns the
        parameter gradient (numpy, n_params) and, with want_df0, dJ/df of the first state."""
        import torch

        def dev(t, shape):
            if t is None:
                return None
            t = t.detach().to(device="cuda", dtype=self.tdtype).contiguous()
            if tuple(t.shape) != shape:
                raise ValueError(f"seed of shape {tuple(t.shape)}, expected {shape}")
            return t
        drho = dev(drho, (self.ny, self.nx))
        df = dev(df, (9, self.ny, self.nx))
        df0 = torch.empty((9, self.ny, self.nx), dtype=self.tdtype, device="cuda") if want_df0 else None
        grad = np.zeros(self.n_params)
        self.stream.wait_stream(torch.cuda.current_stream())
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        self._c(self.lib.lbm_adjoint(self.ctx, ptr(drho), ptr(df), 1, grad.ctypes.data, ptr(df0)))
        return (grad, df0) if want_df0 else grad


class _InstanceView(Lattice):
    """An instance of a Batch: an ordinary lattice context owned by the batch."""

    def __init__(self, batch, k, ctx, phys, precision):
        self.lib = batch.lib
        self.nx, self.ny = int(phys["nx"]), int(phys["ny"])
        self.precision = precision
        import torch
        self.dtype = np.float64 if precision == _abi.LBM_FP64 else np.float32
        self.tdtype = torch.float64 if precision == _abi.LBM_FP64 else torch.float32
        self.stream = batch.stream
        self.ctx = ctx
        self._batch = batch   # keeps the batch (and its workspace) alive

    def __del__(self):
        pass   # the batch owns the context

    def step(self, n: int = 1):
        raise RuntimeError("instances of a batch advance with Batch.step")


class Batch:
    """Many independent lattices advanced together by the persistent batched kernel."""

    def __init__(self, physics: list, precision: int = _abi.LBM_FP32, stream=None,
                 layout: int = _abi.LBM_LAYOUT_AB):
        import torch
        lib = _abi.load()
        self.lib = lib
        self.n = len(physics)
        self.precision = precision
        made = [make_config(p, precision, layout=layout) for p in physics]
        self._keep = made
        arr = (lbm_config * self.n)(*[m[0] for m in made])
        self._cfgs = arr
        n = C.c_size_t()
        check(lib.lbm_batch_workspace_size(self.n, arr, C.byref(n)))
        self.workspace = torch.empty(n.value, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.Stream()
        b = C.c_void_p()
        st = lib.lbm_batch_create(self.n, arr, C.c_void_p(self.stream.cuda_stream),
                                  C.c_void_p(self.workspace.data_ptr()), n.value, C.byref(b))
        self.b = b
        self._check(st)
        self._check(lib.lbm_batch_build_links(self.b))
        self.instances = []
        for k in range(self.n):
            ctx = C.c_void_p()
            self._check(lib.lbm_batch_instance(self.b, k, C.byref(ctx)))
            self.instances.append(_InstanceView(self, k, ctx, physics[k], precision))

    def __del__(self):
        if getattr(self, "b", None):
            self.instances = []
            self.lib.lbm_batch_destroy(self.b)
            self.b = None

    def _check(self, st):
        if st != _abi.LBM_OK:
            msg = self.lib.lbm_batch_last_error(self.b).decode() if getattr(self, "b", None) else ""
            raise _abi.LbmError(st, msg)

    def init(self, droplets: list):
        self._init_keep = []
        specs = (lbm_init_spec * self.n)()
        for k, d in enumerate(droplets):
            m = len(d["r0"])
            arrs = [np.ascontiguousarray(np.asarray(d.get(key) if d.get(key) is not None else np.zeros(m), np.float64))
                    for key in ("x0", "y0", "r0", "ux0", "uy0")]
            self._init_keep.append(arrs)
            specs[k] = lbm_init_spec(m, *[a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs], float(d["width"]))
        self._check(self.lib.lbm_batch_init(self.b, specs))

    def step(self, n: int = 1):
        self._check(self.lib.lbm_batch_step(self.b, int(n)))

    def check(self):
        """Synchronises; raises LbmError(LBM_ETIMEOUT) if a grid-barrier wait gave up."""
        self._check(self.lib.lbm_batch_check(self.b))

    def set_spin_limit(self, polls: int):
        self._check(self.lib.lbm_batch_set_spin_limit(self.b, int(polls)))

    def set_tile(self, log2w: int):
        """Node-tile shape of the persistent kernel: 2^log2w x 256/2^log2w (log2w in 4..8)."""
        self._check(self.lib.lbm_batch_set_tile(self.b, int(log2w)))

    def set_schedule(self, groups: int):
        """1: all instances in lockstep; 2: two node-balanced groups, the second three phases
        behind (same results, different overlap of the phases)."""
        self._check(self.lib.lbm_batch_set_schedule(self.b, int(groups)))

    def autotune(self, steps: int = 20):
        """Times every tile shape, then both schedules with the fastest shape, over `steps`
        steps each (the instances advance 14 * steps steps) and keeps the fastest; returns
        {"log2w", "tile", "groups", "ms": {tile or schedule: ms}}."""
        chosen, groups = C.c_int32(), C.c_int32()
        ms = np.zeros(7)
        self._check(self.lib.lbm_batch_autotune(self.b, int(steps), C.byref(chosen), C.byref(groups),
                                                ms.ctypes.data))
        shapes = [f"{1 << w}x{256 >> w}" for w in range(4, 9)]
        keys = shapes + ["lockstep", "two groups"]
        return {"log2w": chosen.value, "tile": shapes[chosen.value - 4], "groups": groups.value,
                "ms": {k: round(float(t), 3) for k, t in zip(keys, ms)}}

    def info(self):
        o = np.zeros(4, np.int64)
        self._check(self.lib.lbm_batch_info(self.b, o.ctypes.data))
        return {"grid": int(o[0]), "node_tiles": int(o[1]), "graph": bool(o[2]), "bc_chunks": int(o[3])}

    def synchronize(self):
        self.stream.synchronize()
