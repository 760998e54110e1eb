"""Work split over several GPUs: y-slabs of one lattice, and whole lattices of a batch.

One lattice: each rank owns a band of whole rows [y0, y1) of the global lattice and holds an
H-row halo on each side that has a neighbour (the C library's lbm_create_slab).  A step
reaches a node's state from at most 7 rows away (streaming, the fourth-order stencils of Eqs.
9 and 12, the two solid layers of Eq. 15), so with H >= 7 k the halo is refreshed every k steps
by one message per edge (lbm_slab_pack / lbm_slab_unpack: populations, density, the EOS plane
and the Eq. 18 carries of H rows), and every rank's own rows stay bit for bit those of the
undivided lattice.  The global mass and Delta M are FP64 all-reduce sums of the slabs' own.

Many lattices: whole instances are packed onto ranks by size (shard_instances); they never
exchange data.

Transports: SlabGroup exchanges between slabs held by one process (device copies on one
GPU); DistSlab exchanges with the neighbouring ranks through torch.distributed -- device
buffers with NCCL, page-locked host copies with gloo.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import _abi
from ._abi import check
from .lattice import make_config

REACH = 7             # rows a step reaches (see above); the halo must cover k steps of it


def shard_instances(sizes: Sequence[int], world: int) -> List[List[int]]:
    """Greedy bin packing of independent instances (largest first) onto `world` ranks; returns
    one sorted index list per rank.  No data moves between ranks: each advances its own."""
    order = sorted(range(len(sizes)), key=lambda k: (-sizes[k], k))
    load = [0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda j: (load[j], j))
        out[r].append(k)
        load[r] += sizes[k]
    return [sorted(v) for v in out]


def slab_rows(ny: int, n: int, halo: int) -> List[Tuple[int, int]]:
    """Even split of ny rows into n bands [y0, y1); every band with a neighbour must own at
    least `halo` rows (it sends that many)."""
    b = [round(k * ny / n) for k in range(n + 1)]
    out = [(b[k], b[k + 1]) for k in range(n)]
    if n > 1 and min(y1 - y0 for y0, y1 in out) < halo:
        raise ValueError(f"{ny} rows over {n} slabs leaves fewer than {halo} rows in a slab")
    return out


def neighbours(rank: int, n: int, walls: bool) -> Tuple[Optional[int], Optional[int]]:
    """(rank below, rank above) of a slab; None where a walled lattice ends.  A periodic
    lattice wraps around (one slab is its own neighbour)."""
    below = rank - 1 if rank > 0 else (None if walls else n - 1)
    above = rank + 1 if rank < n - 1 else (None if walls else 0)
    return below, above


class Slab:
    """The rows [y0, y1) of a global lattice (global configuration `phys`) on the current
    CUDA device, with halos of `halo` rows; lbm_* calls through the C ABI."""

    def __init__(self, phys: dict, y0: int, y1: int, halo: int = 8, precision: int = _abi.LBM_FP32,
                 rho_ref: float = -1.0, stream=None):
        import torch
        lib = _abi.load()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.lib = lib
        self.phys = phys
        self.y0, self.y1, self.halo = int(y0), int(y1), int(halo)
        self.nx = int(phys["nx"])
        self.precision = precision
        self.dtype = np.float64 if precision == _abi.LBM_FP64 else np.float32
        self._cfg, self._keep = make_config(phys, precision, rho_ref)
        n = C.c_size_t()
        check(lib.lbm_slab_workspace_size(C.byref(self._cfg), self.y0, self.y1, self.halo, C.byref(n)))
        self.workspace = torch.empty(n.value, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.Stream()
        ctx = C.c_void_p()
        st = lib.lbm_create_slab(C.byref(self._cfg), self.y0, self.y1, self.halo, C.c_void_p(self.stream.cuda_stream),
                                 C.c_void_p(self.workspace.data_ptr()), n.value, C.byref(ctx))
        self.ctx = ctx
        if st != _abi.LBM_OK:
            msg = lib.lbm_last_error(ctx).decode() if ctx else ""
            if ctx:
                lib.lbm_destroy(ctx)
                self.ctx = None
            raise _abi.LbmError(st, msg)
        info = np.zeros(10, np.int32)
        self._c(lib.lbm_slab_info(self.ctx, info.ctypes.data))
        (self.y_off, self.ny_local, self.own_lo, self.own_hi, _, eb, et, self.recv_lo_bottom,
         self.recv_lo_top, self.periodic) = [int(v) for v in info]
        self.has_edge = (bool(eb), bool(et))
        mb = C.c_size_t()
        self._c(lib.lbm_slab_message_bytes(self.ctx, C.byref(mb)))
        self.message_bytes = mb.value
        self._c(lib.lbm_build_links(self.ctx))

    def __del__(self):
        if getattr(self, "ctx", None):
            self.lib.lbm_destroy(self.ctx)
            self.ctx = None

    def _c(self, st):
        check(st, self.ctx)

    def init_droplets(self, d: dict):
        """Eq. 19 start from the drops' global positions."""
        n = len(d["r0"])
        arrs = [np.ascontiguousarray(np.asarray(d.get(k) if d.get(k) is not None else np.zeros(n), np.float64))
                for k in ("x0", "y0", "r0", "ux0", "uy0")]
        self._init_keep = arrs
        s = _abi.lbm_init_spec(n, *[a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs], float(d["width"]))
        self._c(self.lib.lbm_init(self.ctx, C.byref(s)))

    def step(self, n: int = 1):
        self._c(self.lib.lbm_step(self.ctx, int(n)))

    def pack(self, edge: int, buf):
        """Queue the message for the neighbour on `edge` (0 bottom, 1 top) into device tensor buf."""
        self._c(self.lib.lbm_slab_pack(self.ctx, int(edge), C.c_void_p(buf.data_ptr()), self.message_bytes))

    def unpack(self, edge: int, buf):
        """Queue the neighbour's message into this slab's halo on `edge`."""
        self._c(self.lib.lbm_slab_unpack(self.ctx, int(edge), C.c_void_p(buf.data_ptr()), self.message_bytes))

    def synchronize(self):
        self.stream.synchronize()

    # ---- read-outs of the own rows (global rows y0 .. y1-1)
    def populations(self):
        nl = self.nx * self.ny_local
        f = np.zeros(9 * nl, self.dtype)
        self._c(self.lib.lbm_populations(self.ctx, f.ctypes.data, 0))
        return f.reshape(9, self.ny_local, self.nx)[:, self.own_lo:self.own_hi]

    def fields(self):
        nl = self.nx * self.ny_local
        out = [np.zeros(nl, self.dtype) for _ in range(3)]
        self._c(self.lib.lbm_fields(self.ctx, *[o.ctypes.data for o in out], 0))
        return tuple(o.reshape(self.ny_local, self.nx)[self.own_lo:self.own_hi] for o in out)

    def kind(self):
        k = np.zeros((self.ny_local, self.nx), np.uint8)
        self._c(self.lib.lbm_get_kind(self.ctx, k.ctypes.data))
        return k[self.own_lo:self.own_hi]

    def mass(self):
        """(M, M0, last Delta M) of the own rows and own boundary nodes."""
        M, M0, dM = C.c_double(), C.c_double(), C.c_double()
        self._c(self.lib.lbm_mass(self.ctx, C.byref(M), C.byref(M0), C.byref(dM)))
        return M.value, M0.value, dM.value


class SlabGroup:
    """All slabs of one lattice held by one process on one GPU: the halo exchange is a device
    copy between message buffers."""

    def __init__(self, phys: dict, n: int, halo: int = 8, precision: int = _abi.LBM_FP32, rho_ref: float = -1.0,
                 steps_per_exchange: int = 1):
        import torch
        if halo < REACH * steps_per_exchange:
            raise ValueError(f"a halo of {halo} rows covers {halo // REACH} steps, not {steps_per_exchange}")
        self.walls = bool(phys["walls"])
        self.k = int(steps_per_exchange)
        rows = slab_rows(int(phys["ny"]), n, halo)
        self.slabs = [Slab(phys, y0, y1, halo, precision, rho_ref) for y0, y1 in rows]
        self.buf = [[torch.empty(s.message_bytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
                    for s in self.slabs]

    def init_droplets(self, d: dict):
        for s in self.slabs:
            s.init_droplets(d)

    def exchange(self):
        n = len(self.slabs)
        for r, s in enumerate(self.slabs):
            for e in (0, 1):
                if s.has_edge[e]:
                    s.pack(e, self.buf[r][e])
        for s in self.slabs:
            s.synchronize()
        for r, s in enumerate(self.slabs):
            below, above = neighbours(r, n, self.walls)
            # my bottom halo holds the rank below's top rows, my top halo the rank above's bottom rows
            if below is not None:
                s.unpack(0, self.buf[below][1])
            if above is not None:
                s.unpack(1, self.buf[above][0])
        for s in self.slabs:
            s.synchronize()

    def step(self, n: int):
        """n steps (a multiple of steps_per_exchange), exchanging every steps_per_exchange."""
        if n % self.k:
            raise ValueError("the step count must be a multiple of steps_per_exchange")
        for _ in range(n // self.k):
            for s in self.slabs:
                s.step(self.k)
            self.exchange()

    def populations(self):
        return np.concatenate([s.populations() for s in self.slabs], axis=1)

    def fields(self):
        parts = [s.fields() for s in self.slabs]
        return tuple(np.concatenate([p[i] for p in parts], axis=0) for i in range(3))

    def mass(self):
        ms = [s.mass() for s in self.slabs]
        return tuple(float(np.sum([m[i] for m in ms])) for i in range(3))


class DistSlab:
    """This rank's slab of one lattice, exchanging halos with the neighbouring ranks through
    torch.distributed: device buffers with NCCL, page-locked host copies otherwise (gloo)."""

    def __init__(self, phys: dict, rank: int, world: int, halo: int = 8, precision: int = _abi.LBM_FP32,
                 rho_ref: float = -1.0, steps_per_exchange: int = 1, group=None):
        import torch
        import torch.distributed as dist
        if halo < REACH * steps_per_exchange:
            raise ValueError(f"a halo of {halo} rows covers {halo // REACH} steps, not {steps_per_exchange}")
        self.rank, self.world, self.group = rank, world, group
        self.k = int(steps_per_exchange)
        self.walls = bool(phys["walls"])
        y0, y1 = slab_rows(int(phys["ny"]), world, halo)[rank]
        self.slab = Slab(phys, y0, y1, halo, precision, rho_ref)
        self.device_comm = dist.get_backend(group) == "nccl"
        mb = self.slab.message_bytes
        dev = [torch.empty(mb, dtype=torch.uint8, device="cuda") for _ in range(4)]   # send 0, 1; recv 0, 1
        self.send_dev, self.recv_dev = dev[:2], dev[2:]
        if not self.device_comm:
            self.send_host = [torch.empty(mb, dtype=torch.uint8).pin_memory() for _ in range(2)]
            self.recv_host = [torch.empty(mb, dtype=torch.uint8).pin_memory() for _ in range(2)]

    def init_droplets(self, d: dict):
        self.slab.init_droplets(d)

    def exchange(self):
        import torch
        import torch.distributed as dist
        s = self.slab
        below, above = neighbours(self.rank, self.world, self.walls)
        for e in (0, 1):
            if s.has_edge[e]:
                s.pack(e, self.send_dev[e])
        if self.device_comm:
            # NCCL runs on its own stream: it must see the packed buffers
            torch.cuda.current_stream().wait_stream(s.stream)
            send, recv = self.send_dev, self.recv_dev
        else:
            for e in (0, 1):
                if s.has_edge[e]:
                    with torch.cuda.stream(s.stream):
                        self.send_host[e].copy_(self.send_dev[e], non_blocking=True)
            s.synchronize()
            send, recv = self.send_host, self.recv_host
        # in the same order on every rank, so that two messages between one pair of ranks (a
        # periodic lattice on two ranks) are matched in order: first my top rows to the rank
        # above and my bottom halo from the rank below, then the reverse direction.  Tags name
        # the edge the message is unpacked into.
        plan = []
        if self.world == 1:
            # a periodic lattice on one rank is its own neighbour on both edges
            plan = [("copy", 1, 0), ("copy", 0, 1)] if below is not None else []
        else:
            if above is not None:
                plan.append(("send", 1, above))
            if below is not None:
                plan += [("recv", 0, below), ("send", 0, below)]
            if above is not None:
                plan.append(("recv", 1, above))
        if self.device_comm:
            ops = [dist.P2POp(dist.isend if kind == "send" else dist.irecv, (send if kind == "send" else recv)[e],
                              peer, self.group, tag=1 - e if kind == "send" else e)
                   for kind, e, peer in plan if kind != "copy"]
            if ops:
                for w in dist.batch_isend_irecv(ops):
                    w.wait()
        else:
            works = []
            for kind, e, peer in plan:
                if kind == "send":
                    works.append(dist.isend(send[e], peer, group=self.group, tag=1 - e))
                elif kind == "recv":
                    works.append(dist.irecv(recv[e], peer, group=self.group, tag=e))
            for w in works:
                w.wait()
        for kind, e_from, e_to in plan:
            if kind == "copy":
                recv[e_to].copy_(send[e_from])
        if self.device_comm:
            s.stream.wait_stream(torch.cuda.current_stream())
        else:
            for e in (0, 1):
                if s.has_edge[e]:
                    with torch.cuda.stream(s.stream):
                        self.recv_dev[e].copy_(self.recv_host[e], non_blocking=True)
        for e in (0, 1):
            if s.has_edge[e]:
                s.unpack(e, self.recv_dev[e])

    def step(self, n: int):
        if n % self.k:
            raise ValueError("the step count must be a multiple of steps_per_exchange")
        for _ in range(n // self.k):
            self.slab.step(self.k)
            self.exchange()

    def mass(self):
        """Global (M, M0, last Delta M): FP64 sums of every slab's own."""
        import torch
        import torch.distributed as dist
        m = torch.tensor(self.slab.mass(), dtype=torch.float64)
        if self.device_comm:
            m = m.cuda()
        dist.all_reduce(m, group=self.group)
        return tuple(float(v) for v in m.cpu())
