#!/usr/bin/env python3
"""Benchmark of the multiphase curved-boundary LBM step on GB300.

A "step" is one lattice Boltzmann time step of the whole hot path over the workload's
lattice: density, solid-layer densities (Eq. 15), chemical potential (Eq. 12), force +
collision + streaming, and every cut link by Eqs. 16-18.  The metric is MLUPS (million
lattice-node updates per second, all nodes counted).

Default workload: drop impact on a cylinder, 2048 x 4096 D2Q9, MRT, Carnahan-Starling EOS at
0.6 Tc, gravity, FP32 populations (0.68 GB working set, larger than the 129 MB L2, so no L2
flush is needed between steps).  `--workload c2` runs the 1024 x 1024, 16-cylinder lattice
instead, flushing L2 before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun the headline lattice is split into y-slabs, one per rank, whose halos are
exchanged over NCCL every few steps (strong scaling); rank 0 prints one JSON line.
`--impl reference` times the FP64 reference oracle on the host cores instead (rank 0 only).
Before the clock starts the graphs that the timed steps launch are captured (lbm_prepare_steps),
so that no capture happens inside the timed region; nothing is stepped by it.

Besides the contract keys the line carries: `roofline` (the collide kernel's algorithmic bytes
over its CUDA-event time, against the measured HBM copy bandwidth, with the per-phase times),
`cpu_baseline` (the oracle on the host cores), `e2e` (through the C-ABI with host buffers),
`clocks`, `fp64` (the same workload with FP64 populations: MLUPS and the FP32/FP64 speed
ratio; the drop's interface on the centre line in FP32 and FP64 over 10000 steps; the 128 x 128
FP64 case's mass change with the present scheme and IBC), `batched` (256 instances of
128^2..768^2 in one persistent launch against the same instances stepped one by one; the
autotuned tile shape; the same comparison on 1024 instances of 64^2..128^2), and `adjoint` (512 x 512, 4000 steps, checkpoint every 200: forward,
checkpointed forward and reverse-sweep times, one reverse step against one forward step, and
the gradient), and `bc_comparison` (the boundary schemes of the paper's Sec. 4.3-4.4 on
reduced-size drops: late per-step compensation and spurious currents), and `paper_runs` (the
paper's Sec. 4.1-4.2 drops at full size with Peng-Robinson: mass change of the present scheme
and IBC at every q, 40 flat-wall lattices in one batch, and the curved substrate; and Sec. 4.5's
drop impact at its three Bond numbers: the film on the cylinder's top against the h*(t*) laws), and
`pseudopotential` (the impact lattice with the pseudopotential force in place of the
chemical-potential one: step time, per-phase times, against the headline step), and `aa_layout`
(the headline lattice with one population lattice in AA order: step time, workspace, against the
two-lattice step).  `--mode kernels` / `--mode adjoint` / `--mode batch` run only the timed
step loop / only the gradient workload / only the batched kernel (for profiler captures);
`--layout 1` puts the headline lattice in AA order.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline, FP32 vs FP64 oracle; batched and adjoint cost ratio"
UNIT = "MLUPS"
# algorithmic bytes of the fused force + collision + streaming kernel: per fluid node read 9
# and write 9 FP32 populations (72 B) and read rho and mu (8 B); per lattice node its class
# byte (1 B)
COLLIDE_BYTES_PER_FLUID_NODE = 80
COLLIDE_BYTES_PER_NODE = 1
# the pseudopotential variant reads psi only (4 B) besides the populations
PSEUDO_COLLIDE_BYTES_PER_FLUID_NODE = 76
STEP_BYTES_PER_NODE = 72
# y-slabs of one lattice over several GPUs: halo refresh period (the halo is 8 rows per step)
SLAB_EXCHANGE_EVERY = 4
FALLBACK_HBM_GBS = 6800.0


def collide_kernel_name(kind, pseudo):
    force = "pseudopotential force" if pseudo else "Eq. 9 force"
    if kind == 2:
        return f"k_collide_tma ({force} + collide + stream + the next density, TMA-pipelined column sweeps)"
    if kind == 1:
        return f"k_collide_tma ({force} + collide + stream, TMA-pipelined persistent grid)"
    return f"k_collide ({force} + collide + stream, one tile per block)"


def workload_config(sc, wname, l2):
    """The workload part of the line, the same for both arms."""
    return {"workload": wname, "nodes": sc.nodes, "l2": l2}


def pseudo_impact():
    """The impact lattice with the pseudopotential force: CS at 0.7 Tc (this force model does not
    hold the Maxwell densities of 0.6 Tc), k = 1, wall factor 0.15."""
    import scenarios as S
    return S.c3_impact().with_(dmu_w=[0.15], force_model=S.FORCE_PSEUDO, k=1.0, kappa=0.0, T_over_Tc=0.7)


def workload(name):
    import scenarios as S
    if name == "c2":
        return S.c2_fp32_single(), "c2 16 droplets on cylinders 1024x1024 D2Q9 MRT CS T=0.6Tc FP32"
    if name == "c3pp":
        return pseudo_impact(), "c3 geometry 2048x4096 D2Q9 MRT, pseudopotential force, CS T=0.7Tc k=1, FP32"
    return S.c3_impact(), "c3 drop impact on a cylinder 2048x4096 D2Q9 MRT CS T=0.6Tc gravity FP32"


def run_batched(G, torch, rank, world, steps, small=False):
    """Batched workload: seed-random droplet-on-cylinder instances of 128^2..768^2 (small:
    1024 instances of 64^2..128^2), advanced together by the persistent kernel (one launch for
    all steps), against the same instances each advanced by its own lbm_step graph launches,
    issued one lattice after another (each lattice has its own stream)."""
    import scenarios as S
    scs = S.c4_batch(seed=5, n=1024, nmin=64, nmax=128) if small else S.c4_batch()
    from paper_2203_04508_gb300.slab import shard_instances
    mine = shard_instances([sc.nodes for sc in scs], world)[rank]
    scs = [scs[k] for k in mine]
    nodes = sum(sc.nodes for sc in scs)
    b = G.Batch([sc.physics() for sc in scs], precision=G.LBM_FP32)
    b.init([sc.droplets() for sc in scs])
    # the library's autotuner picks the node-tile shape on this batch, then a fresh start
    tuned = b.autotune(10)
    b.init([sc.droplets() for sc in scs])
    b.step(2)
    b.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    e1.synchronize()
    b.check()
    ms_b = e0.elapsed_time(e1)
    info = b.info()
    ws_b = b.workspace.numel()
    del b
    torch.cuda.empty_cache()
    # the same batch with one population lattice per instance in AA order (same tile shape)
    ba = G.Batch([sc.physics() for sc in scs], precision=G.LBM_FP32, layout=G.LBM_LAYOUT_AA)
    ba.init([sc.droplets() for sc in scs])
    ba.set_tile(int(tuned["log2w"]))
    ba.set_schedule(int(tuned["groups"]))
    ba.step(2)
    ba.check()
    e0.record(ba.stream)
    ba.step(steps)
    e1.record(ba.stream)
    e1.synchronize()
    ba.check()
    ms_aa = e0.elapsed_time(e1)
    ws_aa = ba.workspace.numel()
    del ba
    torch.cuda.empty_cache()
    # looping single-instance launches, same instances, same steps
    lats = []
    for sc in scs:
        lat = G.Lattice(sc.physics(), precision=G.LBM_FP32)
        lat.init_droplets(sc.droplets())
        lat.step(10)                     # warm-up: captures the eight- and two-step graphs
        lats.append(lat)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for lat in lats:
        lat.step(steps)
    for lat in lats:
        lat.synchronize()
    ms_l = (time.perf_counter() - t0) * 1e3
    del lats
    torch.cuda.empty_cache()
    return {"instances": len(scs), "nodes": nodes, "steps": steps, "ms_batched": round(ms_b, 3),
            "mlups_batched": round(nodes * steps / ms_b / 1e3, 1), "ms_looped": round(ms_l, 3),
            "mlups_looped": round(nodes * steps / ms_l / 1e3, 1), "speedup": round(ms_l / ms_b, 3),
            "persistent_grid": info["grid"], "graph_captured": info["graph"],
            "tile": tuned["tile"], "schedule": "two groups" if tuned["groups"] == 2 else "lockstep",
            "autotune_ms_per_10_steps": tuned["ms"],
            "workspace_GB": round(ws_b / 1e9, 3),
            "aa_layout": {"ms_batched": round(ms_aa, 3), "mlups_batched": round(nodes * steps / ms_aa / 1e3, 1),
                          "workspace_GB": round(ws_aa / 1e9, 3)},
            "looped_timing": "host wall clock around all instances' lbm_step calls, synchronised"}


def run_adjoint(G, torch, steps, every):
    """Gradient workload: droplet r = 40 on a cylinder r = 80 in a 512 x 512 channel (FP32).
    Times a plain forward pass, the checkpointed forward pass and the reverse sweep (segment
    recomputation included) with CUDA events on the library's stream."""
    import scenarios as S
    sc = S.c5_adjoint()
    mk = lambda: G.Lattice(sc.physics(), precision=G.LBM_FP32)

    def timed(lat, fn):
        s = lat.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        out = fn()
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1), out

    plain = mk()
    plain.init_droplets(sc.droplets())
    plain.step(20)                       # warm-up (graph capture)
    plain.init_droplets(sc.droplets())
    ms_fwd, _ = timed(plain, lambda: plain.step(steps))
    del plain
    lat = mk()
    lat.init_droplets(sc.droplets())
    lat.forward_checkpointed(2 * every, every)   # warm-up of both passes
    _, seed = lat.objective(0, seed=True)
    lat.adjoint(drho=seed)
    lat.init_droplets(sc.droplets())
    ms_ckpt, _ = timed(lat, lambda: lat.forward_checkpointed(steps, every))
    J, seed = lat.objective(0, seed=True)
    ms_adj, grad = timed(lat, lambda: lat.adjoint(drho=seed))
    ws = lat.adjoint_workspace_size(steps, every)
    del lat, seed
    torch.cuda.empty_cache()
    return {"workload": f"{sc.name}: {sc.nx}x{sc.ny}, cylinder r={sc.r[0]:g}, droplet r={sc.r0[0]:g}, FP32",
            "steps": steps, "checkpoint_every": every, "workspace_GB": round(ws / 1e9, 3),
            "ms_forward": round(ms_fwd, 3), "ms_forward_checkpointed": round(ms_ckpt, 3),
            "ms_reverse": round(ms_adj, 3),
            "cost_ratio": round((ms_ckpt + ms_adj) / ms_fwd, 3),
            # one reverse step (its share of the recomputation included) against one forward step
            "adjoint_step_over_forward_step": round(ms_adj / ms_fwd, 3),
            "reverse_MLUPS": round(sc.nodes * steps / ms_adj / 1e3, 1),
            "J": J, "dJ_ddmu_w": float(grad[0]), "dJ_dcx": float(grad[2]), "dJ_dcy": float(grad[3])}


def run_bc_comparison(G, steps):
    """The paper's comparison of boundary schemes (Sec. 4.3-4.4) on reduced-size sessile drops
    (FP32): per-step compensating mass of Eq. 18 late in the run and the largest speed (the
    spurious currents), present scheme against MIBC and halfway bounce-back on a flat wall at
    q = 0.2, and the present scheme's mass and compensation on a curved substrate."""
    import numpy as np
    import scenarios as S

    def run(sc):
        lat = G.Lattice(sc.physics(), precision=G.LBM_FP32)
        lat.init_droplets(sc.droplets())
        hist = []
        for _ in range(steps // 1000):
            lat.step(1000)
            hist.append(lat.dM_history(1000))
        M, M0, _ = lat.mass()
        r, vx, vy = lat.fields()
        fl = lat.kind() == 0
        h = np.concatenate(hist)
        return {"dM_late_mean_abs": float(np.abs(h[-1000:]).mean()), "dM_max_abs": float(np.abs(h).max()),
                "mass_drift": M / M0 - 1, "max_speed": float(np.hypot(vx, vy)[fl].max())}

    out = {"steps": steps}
    names = {S.BC_PRESENT: "present", S.BC_MIBC: "mibc", S.BC_HBB: "hbb"}
    for theta in (60.0, 120.0):
        case = {}
        for bc in (S.BC_PRESENT, S.BC_MIBC, S.BC_HBB):
            sc = S.Scenario(name="flat_drop", nx=160, ny=100, walls=1, y_bottom=1.2, T_over_Tc=0.6,
                            coll=S.COLL_MRT, tau=0.8, bc=bc, dmu_w_walls=S.theta_to_dmu(theta),
                            x0=[80.0], y0=[13.2], r0=[25.0])
            case[names[bc]] = run(sc)
        out[f"flat_q0.2_theta{int(theta)}"] = case
    R, r0 = 40.0, 28.0
    cx, cy = 100.37, 2.0 + R + 0.61
    for theta in (60.0, 120.0):
        sc = S.Scenario(name="curved_drop", nx=200, ny=240, walls=1, T_over_Tc=0.6, coll=S.COLL_MRT, tau=0.8,
                        cx=[cx], cy=[cy], r=[R], dmu_w=[S.theta_to_dmu(theta)],
                        x0=[cx], y0=[cy + R + 0.5 * r0], r0=[r0])
        out[f"curved_theta{int(theta)}_present"] = run(sc)
    return out


def run_paper_runs(G, torch):
    """The paper's own drops at full size with Peng-Robinson (Eqs. 10-11, T = 0.7 Tc), FP32:
    Sec. 4.1 -- 500 x 300, r0 = 50, q = 0.1 ... 1.0, 60 and 120 deg, present scheme and IBC,
    20000 steps, all 40 lattices in one batch (one persistent launch); Sec. 4.2 -- 500 x 600,
    R = 100, r0 = 70, 60 deg (20000 steps) and 120 deg (25000 steps), each lattice on its own.
    Reports M / M0 - 1 at the end of each run and the throughput of the runs."""
    import scenarios as S
    qs = [round(0.1 * k, 1) for k in range(1, 11)]
    names = {S.BC_PRESENT: "present", S.BC_IBC: "ibc"}
    keys = [(th, q, bc) for th in (60.0, 120.0) for q in qs for bc in names]
    scs = [S.e1_flat_drop(q, th, bc) for th, q, bc in keys]
    steps = scs[0].steps
    b = G.Batch([sc.physics() for sc in scs], precision=G.LBM_FP32)
    b.init([sc.droplets() for sc in scs])
    nodes = sum(sc.nodes for sc in scs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(b.stream)
    b.step(steps)
    e1.record(b.stream)
    e1.synchronize()
    b.check()
    ms = e0.elapsed_time(e1)
    flat = {"lattice": "500x300", "instances": len(scs), "steps": steps, "ms": round(ms, 1),
            "mlups_batched": round(nodes * steps / ms / 1e3, 1)}
    for k, (th, q, bc) in enumerate(keys):
        M, M0, _ = b.instances[k].mass()
        flat.setdefault(f"theta{int(th)}", {}).setdefault(names[bc], {})[f"q{q}"] = float(M / M0 - 1)
    del b
    torch.cuda.empty_cache()
    curved = {"lattice": "500x600"}
    for th in (60.0, 120.0):
        case = {}
        for bc in names:
            sc = S.e2_curved_drop(th, bc)
            lat = G.Lattice(sc.physics(), precision=G.LBM_FP32)
            lat.init_droplets(sc.droplets())
            e0.record(lat.stream)
            lat.step(sc.steps)
            e1.record(lat.stream)
            e1.synchronize()
            M, M0, _ = lat.mass()
            ms = e0.elapsed_time(e1)
            case[names[bc]] = {"mass_change": float(M / M0 - 1), "steps": sc.steps,
                               "mlups": round(sc.nodes * sc.steps / ms / 1e3, 1)}
            del lat
        curved[f"theta{int(th)}"] = case
    return {"eos": "PR a=2/49 b=2/21 omega=0.344, T=0.7Tc, kappa=0.01", "flat": flat, "curved": curved,
            "mass_change": "M/M0 - 1 at the end of the run (FP64 audit over fluid nodes)"}


def run_pseudopotential(G, torch, steps, ms_chempot):
    """The impact lattice (2048 x 4096, cylinder r = 300, drop r = 100 falling at 0.05 under
    gravity) with the pseudopotential force instead of the chemical-potential one: CS at
    0.7 Tc, k = 1, wall factor 0.15 (the pseudopotential model does not hold the Maxwell
    densities of the 0.6 Tc workload).  Step time from CUDA events over graph launches, the
    per-phase times, and the step time against the chemical-potential step of the headline."""
    sc = pseudo_impact()
    lat = G.Lattice(sc.physics(), precision=G.LBM_FP32)
    lat.init_droplets(sc.droplets())
    fluid = lat.counts()["fluid"]
    kname = collide_kernel_name(lat.collide_kernel(), pseudo=True)
    lat.step(20)
    lat.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(lat.stream)
    lat.step(steps)
    e1.record(lat.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    n_prof = max(10, min(100, steps // 5))
    phase_ms = lat.profile_steps(n_prof) / n_prof
    M, M0, _ = lat.mass()
    del lat
    torch.cuda.empty_cache()
    peak, peak_src = measured_peak()
    coll_bytes = PSEUDO_COLLIDE_BYTES_PER_FLUID_NODE * fluid + COLLIDE_BYTES_PER_NODE * sc.nodes
    collide_ms = float(phase_ms[3])
    achieved = coll_bytes / (collide_ms / 1e3) / 1e9
    return {"workload": "c3 geometry 2048x4096, pseudopotential force, CS T=0.7Tc, k=1, FP32",
            "roofline": {"bound": "hbm", "kernel": kname,
                         "achieved": round(achieved, 1), "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": recorded_traffic("c3pp"),
                         "algorithmic_bytes_per_launch": coll_bytes, "launch_ms": round(collide_ms, 5)},
            "steps": steps, "ms_per_step": round(ms, 5), "mlups": round(sc.nodes / ms / 1e3, 1),
            "phase_ms": {k: round(float(v), 5) for k, v in zip(("rho", "solid", "psi", "collide", "bc"), phase_ms)},
            "step_time_vs_chemical_potential": round(ms / ms_chempot, 3), "mass_drift": M / M0 - 1}


def run_aa(G, torch, sc, steps, ms_two):
    """The headline lattice with ONE population lattice in AA order (LBM_LAYOUT_AA): the in-place
    first step and the pull-push second alternate, so steps are timed in pairs.  Step time from
    CUDA events over graph launches, the workspace against the two-lattice one, and the step time
    against the two-lattice step of the headline (the values are the same bits: tests/test_gpu_aa.py)."""
    lat = G.Lattice(sc.physics(), precision=G.LBM_FP32, layout=G.LBM_LAYOUT_AA)
    lat.init_droplets(sc.droplets())
    ws = lat.workspace.numel()
    ws_two = G.workspace_size(sc.physics(), G.LBM_FP32)
    lat.step(20)
    lat.synchronize()
    steps += steps % 2
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(lat.stream)
    lat.step(steps)
    e1.record(lat.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    n_prof = max(10, min(100, steps // 5)) // 2 * 2
    phase_ms = lat.profile_steps(n_prof) / n_prof
    M, M0, _ = lat.mass()
    del lat
    torch.cuda.empty_cache()
    return {"layout": "AA (one population lattice, in place)", "steps": steps, "ms_per_step": round(ms, 5),
            "mlups": round(sc.nodes / ms / 1e3, 1), "workspace_GB": round(ws / 1e9, 4),
            "two_lattice_workspace_GB": round(ws_two / 1e9, 4),
            "phase_ms_pair_average": {k: round(float(v), 5) for k, v in
                                      zip(("rho", "solid", "mu", "collide", "bc"), phase_ms)},
            "step_time_vs_two_lattices": round(ms / ms_two, 3), "mass_drift": M / M0 - 1}


def run_film(G, torch):
    """The paper's drop impact on a cylinder (Sec. 4.5) at full size, 600 x 1200, cylinder R = 100,
    drop D = 200, for its three Bond numbers and contact angles (2.2 / 60 deg, 4.0 / 150 deg,
    14.5 / 150 deg), CS 0.6 Tc, FP32, 30000 steps each, the film on the cylinder's top sampled every
    100 steps through lbm_column_density: the impact (t_i, U_i, h_i), Re and We, h* at a few t*
    against the laws h* = 1 - t* and 0.15 t*^-2, and the throughput of the runs."""
    import numpy as np
    import scenarios as S
    from paper_2203_04508_gb300.film import FilmProbe
    out = {}
    for bo, theta in ((2.2, 60.0), (4.0, 150.0), (14.5, 150.0)):
        sc = S.e5_impact(bo, theta)
        lat = G.Lattice(sc.physics(), precision=G.LBM_FP32)
        lat.init_droplets(sc.droplets())
        info = lat.eos_info()
        probe = FilmProbe(lat, sc.cx[0], sc.cy[0] + sc.r[0], info["rho_g"], info["rho_l"], 2 * sc.r0[0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(0, sc.steps, 100):
            probe.sample(k)
            lat.step(100)
        lat.synchronize()
        dt = time.perf_counter() - t0
        res = probe.result()
        M, M0, _ = lat.mass()
        case = {"steps": sc.steps, "mass_change": M / M0 - 1,
                "mlups_with_sampling": round(sc.nodes * sc.steps / dt / 1e6, 1)}
        if res["impact"]:
            nu = (sc.tau - 0.5) / 3.0
            D = 2 * sc.r0[0]
            ts, hs = res["tstar"], res["hstar"]
            pts = {}
            for a in (0.25, 0.5, 1.0, 1.5, 2.0, 2.5):
                j = int(np.argmin(np.abs(ts - a)))
                pts[f"t*={a:g}"] = {"h*": round(float(hs[j]), 4), "1-t*": round(1 - float(ts[j]), 4),
                                    "0.15t*^-2": round(0.15 / float(ts[j]) ** 2, 4)}
            case.update(t_i=round(res["t_i"], 1), U_i=round(res["U_i"], 5), h_i=round(res["h_i"], 2),
                        Re=round(res["U_i"] * D / nu, 1),
                        We=round(S.RHO_L_CS06 * res["U_i"] ** 2 * D / S.SIGMA_CS06, 2), h_star=pts)
        out[f"Bo{bo:g}_theta{int(theta)}"] = case
        del lat
        torch.cuda.empty_cache()
    return out


def interface_series(G, torch, sc, precision, steps, every):
    """The drop's lower and upper interface on the vertical line through the cylinder centre
    (the mid-density crossings above the cylinder) every `every` steps, and the final mass
    change, for one precision."""
    from paper_2203_04508_gb300.film import FilmProbe
    lat = G.Lattice(sc.physics(), precision=precision)
    lat.init_droplets(sc.droplets())
    info = lat.eos_info()
    probe = FilmProbe(lat, sc.cx[0], sc.cy[0] + sc.r[0], info["rho_g"], info["rho_l"], 2 * sc.r0[0])
    for k in range(0, steps + 1, every):
        probe.sample(k)
        if k < steps:
            lat.step(every)
    M, M0, _ = lat.mass()
    del lat
    torch.cuda.empty_cache()
    return probe, M / M0 - 1


def run_precision_comparison(G, torch, sc, steps):
    """The impact workload in FP32 and in FP64 over `steps` steps: the drop's lower and upper
    interface on the centre line at five instants and the mass change of each."""
    every = steps // 4
    p32, m32 = interface_series(G, torch, sc, G.LBM_FP32, steps, every)
    p64, m64 = interface_series(G, torch, sc, G.LBM_FP64, steps, every)
    rows = {}
    for k, t in enumerate(p32.t):
        rows[f"t={int(t)}"] = {"bottom_fp32": round(p32.bottom[k], 3), "bottom_fp64": round(p64.bottom[k], 3),
                               "top_fp32": round(p32.top[k], 3), "top_fp64": round(p64.top[k], 3)}
    return {"steps": steps, "line": "x = cylinder centre, mid-density crossings above the cylinder",
            "interface": rows, "mass_change_fp32": m32, "mass_change_fp64": m64}


def run_c1_mass(G):
    """The 128 x 128 FP64 case (CS 0.7 Tc, BGK tau = 1, cylinder R = 20, drop r0 = 15, neutral
    wall), 2000 steps: the mass change with the present scheme and with IBC."""
    import scenarios as S
    out = {}
    for name, bc in (("present", S.BC_PRESENT), ("ibc", S.BC_IBC)):
        sc = S.c1_plain_fp64().with_(bc=bc)
        lat = G.Lattice(sc.physics(), precision=G.LBM_FP64)
        lat.init_droplets(sc.droplets())
        lat.step(sc.steps)
        M, M0, _ = lat.mass()
        out[name] = M / M0 - 1
    return {"steps": 2000, "mass_change": out}


def run_accuracy(G, torch):
    """FP32 and FP64 against the FP64 reference oracle on the full-size workloads, from the
    oracle's stored results (tests/golden/accuracy_refs.json, written by
    tests/golden/make_accuracy_refs.py from the oracle alone):
      c2: rho (pointwise) and v (relative to the largest speed) after 1000 FP32 steps at 1024
          seeded nodes, half of them in interfaces; at 5000 / 10000 / 20000 steps the drops'
          liquid densities, the gas density and the contact angles (largest relative
          differences) and the mass change (difference);
      c3: the drop's interfaces on the centre line every 100 steps up to 500 (largest
          difference, lu), the mass change, rho and v after 500 steps at 1024 seeded nodes;
      c5: J and dJ/d(dmu_w, dmu_w walls, cx, cy) after 4000 steps with checkpoints every 200,
          FP64 and FP32, against the oracle's complex-step and central-difference derivatives
          (largest relative difference over the four components)."""
    import numpy as np
    import scenarios as S
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from diagnostics import droplet_report, isoline_crossings_column, report_errors, sampled_errors
    path = os.path.join(ROOT, "tests", "golden", "accuracy_refs.json")
    if not os.path.exists(path):
        return None
    refs = json.load(open(path))
    g3 = lambda v: float(f"{v:.3g}")
    out = {"source": "FP64 oracle results in tests/golden/accuracy_refs.json"}
    if "c2" in refs:
        sc = S.c2_fp32_single()
        lat = G.Lattice(sc.physics(), precision=G.LBM_FP32)
        lat.init_droplets(sc.droplets())
        info = lat.eos_info()
        lat.step(1000)
        er, ev = sampled_errors(*lat.fields(), refs["c2"]["fields_1000"])
        c2 = {"fields_1000_steps": {"rho": g3(er), "v": g3(ev)}}
        done = 0 + 1000
        d = sc.droplets()
        for t in ("5000", "10000", "20000"):
            lat.step(int(t) - done)
            done = int(t)
            r, _, _ = lat.fields()
            rep = droplet_report(r.astype(np.float64), lat.kind() == 0, info["rho_g"], info["rho_l"],
                                 sc.cx, sc.cy, sc.r, d["x0"], d["y0"], d["r0"])
            M, M0, _ = lat.mass()
            rep["mass_change"] = M / M0 - 1
            e = report_errors(rep, refs["c2"]["reports"][t])
            c2[f"steady_{t}"] = {k: (g3(v) if isinstance(v, float) else v) for k, v in e.items()}
        out["c2_fp32"] = c2
        del lat
    if "c3" in refs:
        ref = refs["c3"]
        sc = S.c3_impact()
        lat = G.Lattice(sc.physics(), precision=G.LBM_FP32)
        lat.init_droplets(sc.droplets())
        info = lat.eos_info()
        mid = 0.5 * (info["rho_g"] + info["rho_l"])
        xc = ref["x_line"]
        dpos, dmass = 0.0, 0.0
        for k, st in enumerate(ref["steps"]):
            if k:
                lat.step(st - ref["steps"][k - 1])
            r, _, _ = lat.fields()
            ys = isoline_crossings_column(r[:, xc].astype(np.float64), lat.kind()[:, xc] == 0, mid,
                                          y_min=sc.cy[0] + sc.r[0] + 5.0)
            M, M0, _ = lat.mass()
            dpos = max(dpos, abs(ys[0] - ref["lower"][k]), abs(ys[-1] - ref["upper"][k]))
            dmass = max(dmass, abs((M / M0 - 1) - ref["mass_change"][k]))
        er, ev = sampled_errors(*lat.fields(), ref["fields_500"])
        out["c3_fp32_500_steps"] = {"interface_lu": g3(dpos), "mass_change": g3(dmass), "rho": g3(er), "v": g3(ev)}
        del lat
    if "c5" in refs:
        ref = refs["c5"]
        sc = S.c5_adjoint()
        cs = np.array([ref["complex_step"][k] for k in ref["order"]])
        cd = np.array([ref["central_differences"][k] for k in ref["order"]])
        c5 = {"steps": ref["steps"], "checkpoint_every": 200, "oracle_complex_vs_central": g3(np.max(np.abs(cd - cs) / np.abs(cs)))}
        for name, prec in (("fp64", G.LBM_FP64), ("fp32", G.LBM_FP32)):
            lat = G.Lattice(sc.physics(), precision=prec)
            lat.init_droplets(sc.droplets())
            lat.forward_checkpointed(ref["steps"], 200)
            J, seed = lat.objective(0, seed=True)
            g = np.asarray(lat.adjoint(drho=seed), dtype=np.float64)
            c5[name] = {"J": g3(abs(J - ref["J"]) / abs(ref["J"])),
                        "vs_complex_step": g3(np.max(np.abs(g - cs) / np.abs(cs))),
                        "vs_central_differences": g3(np.max(np.abs(g - cd) / np.abs(cd)))}
            del lat
        out["c5_gradients"] = c5
    torch.cuda.empty_cache()
    return out


def compact_paper_runs(pr):
    """The paper runs' mass changes reduced to their range per scheme and angle."""
    if pr is None:
        return None
    out = {"eos": pr["eos"], "flat_500x300": {"instances": pr["flat"]["instances"], "steps": pr["flat"]["steps"],
                                              "mlups_batched": pr["flat"]["mlups_batched"]}}
    for th in ("theta60", "theta120"):
        for sch in ("present", "ibc"):
            v = list(pr["flat"][th][sch].values())
            out["flat_500x300"][f"{th}_{sch}_mass_change"] = [float(f"{min(v):.3g}"), float(f"{max(v):.3g}")]
    out["curved_500x600"] = {f"{th}_{sch}_mass_change": float(f"{pr['curved'][th][sch]['mass_change']:.3g}")
                             for th in ("theta60", "theta120") for sch in ("present", "ibc")}
    film = pr.get("impact_film")
    if film:
        out["impact_film"] = {k: {kk: (v[kk] if kk != "h_star" else {t: h["h*"] for t, h in v[kk].items()})
                                  for kk in ("U_i", "Re", "We", "mass_change", "h_star") if kk in v}
                              for k, v in film.items()}
    return out


def compact_bc(bc):
    if bc is None:
        return None
    out = {"steps": bc["steps"]}
    for k, v in bc.items():
        if k == "steps":
            continue
        if "present" in v:
            out[k] = {sch: {"dM_late": float(f"{r['dM_late_mean_abs']:.3g}"), "max_speed": float(f"{r['max_speed']:.3g}")}
                      for sch, r in v.items()}
        else:
            out[k] = {"dM_late": float(f"{v['dM_late_mean_abs']:.3g}"), "max_speed": float(f"{v['max_speed']:.3g}")}
    return out


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


COLLIDE_REGION = (b"static_assert(CT_X * CT_Y == NODE_BLOCK", b"// Boundary links, then the deterministic")


def collide_source_hash():
    """Hash of the source the collide kernels are built from: their region of lbm_step.cu (the
    force terms, the plain and the TMA-pipelined kernel) and the device headers they include."""
    csrc = os.path.join(ROOT, "paper_2203_04508_gb300", "csrc")
    step = open(os.path.join(csrc, "lbm_step.cu"), "rb").read()
    a, b = step.find(COLLIDE_REGION[0]), step.find(COLLIDE_REGION[1])
    # the whole file where the region's markers have moved
    h = hashlib.sha256(step[a:b] if 0 <= a < b else step)
    for f in ("lbm_device.cuh", "lbm_phases.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload_name):
    """DRAM bytes per launch of the collide kernel from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", f"k_collide_{workload_name}_traffic.txt")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        if "=" in line and not line.startswith("#"):
            k, v = line.strip().split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_hash") != collide_source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def oracle_rate(sc, max_seconds, max_steps, threads=None):
    """MLUPS of the FP64 reference oracle on the host cores over a bounded number of steps."""
    import oracle as O
    O.build()
    if threads:
        O.set_threads(threads)
    o = O.Oracle(O.OracleConfig(**sc.physics()))
    d = sc.droplets()
    o.init_droplets(d["x0"], d["y0"], d["r0"], d["width"], d["ux0"], d["uy0"])
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter()
    per = t1 - t0
    n = max(1, min(max_steps, int(max_seconds / max(per, 1e-6))))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    return sc.nodes * n / dt / 1e6, n, O.get_threads()


def l2_note(workload_name):
    return ("flushed before every timed step" if workload_name == "c2"
            else "working set (0.68 GB) larger than L2, no flush")


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands on the host cores, on the same workload:
    `--warmup` untimed steps, then `--steps` timed ones (fewer if they would take more than 90 s;
    the line says how many ran).  Rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    sc, wname = workload(args.workload)
    O.build()
    o = O.Oracle(O.OracleConfig(**sc.physics()))
    d = sc.droplets()
    o.init_droplets(d["x0"], d["y0"], d["r0"], d["width"], d["ux0"], d["uy0"])
    t0 = time.perf_counter()
    o.step(1)
    per = time.perf_counter() - t0
    warm = max(0, min(args.warmup - 1, int(30.0 / max(per, 1e-6))))
    o.step(warm)
    n = max(1, min(args.steps, int(90.0 / max(per, 1e-6))))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    rate = sc.nodes * n / dt / 1e6
    cores = O.get_threads()
    sample = (f"{n} of the {args.steps} requested steps of the full {sc.nx}x{sc.ny} lattice after {warm + 1} "
              f"untimed ones, FP64, {cores} threads")
    line = {"metric": METRIC, "value": round(rate, 3), "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": n, "warmup": warm + 1, "ms_per_step": round(dt / n * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(sc, wname, l2_note(args.workload)),
            "cpu_baseline": {"value": round(rate, 3), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(rate, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c3", "c2", "c3pp"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=200,
                    help="steps of the batched-instances comparison (0: skip it)")
    ap.add_argument("--bc-steps", type=int, default=10000,
                    help="steps of the boundary-scheme comparison (0: skip it)")
    ap.add_argument("--precision-steps", type=int, default=10000,
                    help="steps of the FP32-versus-FP64 interface comparison on c3 (0: skip)")
    ap.add_argument("--pseudo-steps", type=int, default=1000,
                    help="steps of the pseudopotential-force variant of the impact lattice (0: skip)")
    ap.add_argument("--paper-runs", type=int, default=1,
                    help="1: run the paper's full-size PR drops (Sec. 4.1-4.2); 0: skip")
    ap.add_argument("--fp64-steps", type=int, default=200,
                    help="steps of the same workload in FP64 (0: skip it)")
    ap.add_argument("--adjoint-steps", type=int, default=4000,
                    help="steps of the gradient workload (0: skip it)")
    ap.add_argument("--adjoint-every", type=int, default=200)
    ap.add_argument("--layout", type=int, default=0, choices=[0, 1],
                    help="population layout of the headline lattice: 0 two lattices, 1 one lattice in AA order")
    ap.add_argument("--aa-steps", type=int, default=2000,
                    help="steps of the one-lattice (AA order) run of the headline lattice (0: skip it)")
    ap.add_argument("--accuracy", type=int, default=1,
                    help="1: FP32/FP64 against the oracle's stored full-size results (c2, c3, c5); 0: skip")
    ap.add_argument("--collide-kernel", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="collide kernel of the single lattice (-1: the library's choice; 2: the column "
                         "sweeps that also form the next density, for comparison)")
    ap.add_argument("--mode", default="full", choices=["full", "kernels", "adjoint", "batch"],
                    help="kernels: only warm-up and timed steps; adjoint: only the gradient "
                         "workload; batch: only the batched kernel on the first --batch-instances "
                         "lattices of the 256-lattice mix, one launch of --warmup steps and one of "
                         "--steps (all for profiler captures)")
    ap.add_argument("--batch-instances", type=int, default=256)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    args.warmup = max(args.warmup, 3)

    import torch
    import torch.distributed as dist
    import paper_2203_04508_gb300 as G
    from paper_2203_04508_gb300 import build as cuda_build

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        cuda_build.build()
    if world > 1:
        dist.barrier()
    G.load()
    if args.mode == "adjoint":
        print(json.dumps({"mode": "adjoint", **run_adjoint(G, torch, args.adjoint_steps, args.adjoint_every)}))
        return
    if args.mode == "batch":
        import scenarios as S
        scs = S.c4_batch()[:args.batch_instances]
        b = G.Batch([x.physics() for x in scs], precision=G.LBM_FP32)
        b.init([x.droplets() for x in scs])
        b.set_tile(5)
        b.set_schedule(1)   # 32 x 8 tiles in lockstep: the autotuner's choice on the 256-lattice mix
        b.step(args.warmup)
        b.synchronize()
        b.check()
        b.step(args.steps)
        b.synchronize()
        b.check()
        print(json.dumps({"mode": "batch", "instances": len(scs), "nodes": sum(x.nodes for x in scs),
                          "tile": "32x8", "schedule": "lockstep", "steps": args.steps, "warmup": args.warmup}))
        return

    sc, wname = workload(args.workload)
    # one lattice on one GPU, or its y-slabs on several (each rank its own rows plus halos
    # refreshed every SLAB_EXCHANGE_EVERY steps over NCCL)
    dslab = None
    if world > 1:
        from paper_2203_04508_gb300.slab import DistSlab
        dslab = DistSlab(sc.physics(), rank, world, halo=8 * SLAB_EXCHANGE_EVERY, precision=G.LBM_FP32,
                         steps_per_exchange=SLAB_EXCHANGE_EVERY)
        dslab.init_droplets(sc.droplets())
        lat = dslab.slab
        counts = {"fluid": None, "links": None}
        args.steps = max(SLAB_EXCHANGE_EVERY, args.steps // SLAB_EXCHANGE_EVERY * SLAB_EXCHANGE_EVERY)
        args.warmup = max(SLAB_EXCHANGE_EVERY, -(-args.warmup // SLAB_EXCHANGE_EVERY) * SLAB_EXCHANGE_EVERY)
        advance = dslab.step
    else:
        lat = G.Lattice(sc.physics(), precision=G.LBM_FP32, layout=args.layout)
        lat.init_droplets(sc.droplets())
        if args.collide_kernel >= 0:
            lat.set_collide_kernel(args.collide_kernel)
        counts = lat.counts()
        advance = lat.step
    if args.mode == "kernels":
        for _ in range(args.warmup + args.steps):
            lat.step(1)
        lat.synchronize()
        M, M0, _ = lat.mass()
        print(json.dumps({"mode": "kernels", "workload": wname, "steps": args.steps, "warmup": args.warmup,
                          "launches_per_step": lat.launches_per_step(), "mass_drift": M / M0 - 1}))
        return
    lps = lat.launches_per_step()
    collide_name = collide_kernel_name(lat.collide_kernel(), pseudo=False)
    flush = None
    if args.workload == "c2":
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    advance(args.warmup)
    if world == 1:
        # the graphs the timed lbm_step(K) launches, captured now, so that the clock does not run
        # while the host captures one (nothing is stepped)
        lat.prepare_steps(args.steps if flush is None else 1)
    lat.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    s = lat.stream
    if flush is None:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        advance(args.steps)
        e1.record(s)
        e1.synchronize()
        ms_total = e0.elapsed_time(e1)
    else:
        ms_total = 0.0
        for _ in range(args.steps):
            with torch.cuda.stream(s):
                flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            lat.step(1)
            e1.record(s)
            e1.synchronize()
            ms_total += e0.elapsed_time(e1)
    clk = clocks.stop()
    torch.cuda.synchronize()
    if world > 1:
        t = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
        dist.barrier()
    ms_step = ms_total / args.steps
    # the whole lattice's nodes: one lattice on one GPU, or shared out as slabs
    value = sc.nodes * args.steps / (ms_total / 1e3) / 1e6

    # dominant kernel: per-phase CUDA-event times on the library's stream (rank 0's lattice or slab)
    peak, peak_src = measured_peak()
    n_prof = max(10, min(200, args.steps // 10))
    if world == 1:
        phase_ms = lat.profile_steps(n_prof) / n_prof
        collide_ms = float(phase_ms[3])
        coll_bytes = COLLIDE_BYTES_PER_FLUID_NODE * counts["fluid"] + COLLIDE_BYTES_PER_NODE * sc.nodes
        achieved = coll_bytes / (collide_ms / 1e3) / 1e9
        traffic = recorded_traffic(args.workload)
        M, M0, _ = lat.mass()
    else:
        M, M0, _ = dslab.mass()
    step_eff = STEP_BYTES_PER_NODE * sc.nodes / (ms_step / 1e3) / 1e9
    del lat, dslab
    torch.cuda.empty_cache()

    # end to end through the public API with host buffers: set-up from host inputs, every step
    # one C-ABI call plus an 8-byte copy of its compensation sum into page-locked host memory
    # (queued, not waited for), fields back to the host at the end
    e2e = None
    if not args.no_e2e and world == 1:
        n_e2e = args.steps                # the workload the device-timed value measures
        # the caller's page-locked host buffers, made before the clock starts
        dm = torch.empty(n_e2e, dtype=torch.float64, pin_memory=True)
        host = [torch.empty((sc.ny, sc.nx), dtype=torch.float32, pin_memory=True) for _ in range(3)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat2 = G.Lattice(sc.physics(), precision=G.LBM_FP32)
        lat2.init_droplets(sc.droplets())
        for k in range(n_e2e):
            lat2.step(1)
            lat2.last_dM_async(dm, k)     # the step's result to page-locked host memory
        r, vx, vy = lat2.fields(out=host)  # synchronises; every step's result has arrived
        dt = time.perf_counter() - t0
        h2d = 8 * (4 * len(sc.r) + 5 * len(sc.r0)) + 4
        d2h_fields = 3 * sc.nodes * 4
        e2e = {"value": round(sc.nodes * n_e2e / dt / 1e6, 2), "unit": UNIT,
               "h2d_bytes_per_step": round(h2d / n_e2e, 2),
               "d2h_bytes_per_step": round(8 + d2h_fields / n_e2e, 2), "steps": n_e2e}
        del lat2

    single = world == 1 and rank == 0
    accuracy = run_accuracy(G, torch) if (single and args.accuracy) else None

    # the same workload with FP64 populations and arithmetic (the oracle's precision), for the
    # FP32-versus-FP64 throughput; GB300's FP64 rate is a small fraction of its FP32 rate
    fp64 = None
    if args.fp64_steps > 0 and single:
        lat64 = G.Lattice(sc.physics(), precision=G.LBM_FP64)
        lat64.init_droplets(sc.droplets())
        lat64.step(10)
        s64 = lat64.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s64)
        lat64.step(args.fp64_steps)
        e1.record(s64)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1) / args.fp64_steps
        fp64 = {"steps": args.fp64_steps, "ms_per_step": round(ms64, 4),
                "MLUPS": round(sc.nodes / ms64 / 1e3, 1), "fp32_over_fp64": round(ms64 / ms_step, 2)}
        del lat64
        torch.cuda.empty_cache()
        if args.precision_steps > 0 and args.workload == "c3":
            fp64["fp32_vs_fp64"] = run_precision_comparison(G, torch, sc, args.precision_steps)
        fp64["c1_128x128"] = run_c1_mass(G)

    batched = None
    if args.batch_steps > 0:
        batched = run_batched(G, torch, rank, world, args.batch_steps)
        # many small lattices, where one persistent launch replaces thousands of launches
        small = run_batched(G, torch, rank, world, args.batch_steps, small=True) if world == 1 else None
        if world > 1:
            t = torch.tensor([batched["ms_batched"], batched["ms_looped"]], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            nn = torch.tensor([batched["nodes"]], device="cuda", dtype=torch.float64)
            dist.all_reduce(nn)
            steps_b = args.batch_steps
            batched.update(ms_batched=float(t[0]), ms_looped=float(t[1]), nodes=int(nn.item()),
                           mlups_batched=round(float(nn.item()) * steps_b / float(t[0]) / 1e3, 1),
                           mlups_looped=round(float(nn.item()) * steps_b / float(t[1]) / 1e3, 1),
                           speedup=round(float(t[1]) / float(t[0]), 3), instances=256)
        if small is not None:
            batched["small_instances"] = {k: small[k] for k in ("instances", "nodes", "ms_batched", "mlups_batched",
                                                                 "ms_looped", "mlups_looped", "speedup", "tile",
                                                                 "schedule")}
            batched["small_instances"]["sizes"] = "64^2..128^2"

    adjoint = None
    if args.adjoint_steps > 0 and single:
        adjoint = run_adjoint(G, torch, args.adjoint_steps, args.adjoint_every)

    aa = None
    if args.aa_steps > 0 and single and args.workload in ("c3", "c2"):
        aa = run_aa(G, torch, sc, args.aa_steps, ms_step)

    pseudo = None
    if args.pseudo_steps > 0 and single:
        pseudo = run_pseudopotential(G, torch, args.pseudo_steps, ms_step)

    bc_comparison = None
    if args.bc_steps > 0 and single:
        bc_comparison = run_bc_comparison(G, max(1000, args.bc_steps // 1000 * 1000))

    paper_runs = None
    if args.paper_runs and single:
        paper_runs = run_paper_runs(G, torch)
        paper_runs["impact_film"] = run_film(G, torch)

    cpu = None
    if single and not args.no_cpu_baseline:
        rate, n, cores = oracle_rate(sc, max_seconds=20.0, max_steps=50)
        rate1, n1, _ = oracle_rate(sc, max_seconds=8.0, max_steps=50, threads=1)
        import oracle as O
        O.set_threads(cores)
        cpu = {"value": round(rate, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n} FP64 oracle steps of the full {sc.nx}x{sc.ny} lattice after one untimed step",
               "single_thread": {"value": round(rate1, 3), "cores": 1, "sample": f"{n1} steps"}}

    if rank == 0:
        l2 = l2_note(args.workload)
        if world == 1:
            roof = {"bound": "hbm", "kernel": collide_name,
                    "achieved": round(achieved, 1), "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": traffic,
                    "algorithmic_bytes_per_launch": coll_bytes, "launch_ms": round(collide_ms, 5),
                    "step_effective_GBs": round(step_eff, 1), "step_effective_frac": round(step_eff / peak, 4),
                    "phase_ms": {k: round(float(v), 5) for k, v in
                                 zip(("rho", "solid", "mu", "collide", "bc"), phase_ms)}}
        else:
            # several GPUs: the whole step's effective bandwidth over all of them
            roof = {"bound": "hbm", "kernel": "whole step (y-slabs)", "achieved": round(step_eff, 1),
                    "peak": round(peak * world, 1), "peak_source": peak_src, "unit": "GB/s",
                    "frac": round(step_eff / (peak * world), 4), "traffic": None}
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 5), "higher_is_better": True,
            "scaling": "weak" if world == 1 else "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(sc, wname, l2),
            "parallelism": "one lattice on one GPU" if world == 1 else
                           f"one lattice in {world} y-slabs (halo {8 * SLAB_EXCHANGE_EVERY} rows, exchanged every "
                           f"{SLAB_EXCHANGE_EVERY} steps over NCCL)",
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": lps * args.steps,
            "accuracy": accuracy,
            "batched": batched,
            "adjoint": adjoint,
            "aa_layout": aa,
            "fp64": fp64,
            "pseudopotential": None if pseudo is None else {k: pseudo[k] for k in ("ms_per_step", "mlups",
                                                                                    "step_time_vs_chemical_potential")}
                               | {"collide_frac": pseudo["roofline"]["frac"]},
            "bc_comparison": compact_bc(bc_comparison),
            "paper_runs": compact_paper_runs(paper_runs),
            "value_fluid_nodes": None if counts["fluid"] is None else round(value * counts["fluid"] / sc.nodes, 2),
            "mass_drift": M / M0 - 1,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
