"""Writes accuracy_refs.json: what the FP64 reference oracle gives on the full-size FP32
workloads, for the GPU accuracy report (tests/test_gpu_accuracy.py and bench.py's `accuracy`
entry).  Every value here comes from the oracle (oracle/) and from the post-processing in
tests/diagnostics.py; nothing from the CUDA path.

  c2 (1024 x 1024, 16 cylinders with resting drops, CS 0.6 Tc, MRT nu = 0.1):
     - after 1000 steps: rho and v = u + F/(2 rho) at 512 seeded fluid nodes and 512 seeded
       interface nodes (0.1 (rho_l - rho_g) < rho - rho_g < 0.9 (rho_l - rho_g)), and max |v|
       over the whole lattice (the normwise velocity error divides by it);
     - at 5000, 10000 and 20000 steps: the drops' liquid-core densities, the gas density, the
       contact angle of every drop on its cylinder (diagnostics.droplet_report), and the mass
       change (M - M0)/M0.
  c3 (2048 x 4096 drop impact): the drop's lower and upper interface on the vertical line
     through the cylinder centre and the mass change every 100 steps up to 500, and rho, v
     at 512 + 512 seeded nodes after 500 steps.
  c5 (512 x 512, drop r = 40 on a cylinder r = 80, 4000 steps): J = y_cm + L_wet and its
     derivatives with respect to the cylinder's and the walls' wall chemical-potential offset
     and the cylinder centre, by the complex step (h = 1e-20) and by central differences
     (h = 1e-4), checking first that the +-h geometries have the same node classes, link set
     and q branches.

Run:  python tests/golden/make_accuracy_refs.py [c2] [c3] [c5]    (all three: ~35 min on 8 cores)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.join(HERE, "..", "..")
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import oracle as O  # noqa: E402
import scenarios as S  # noqa: E402
from diagnostics import droplet_report, isoline_crossings_column  # noqa: E402
from harness import make_oracle, oracle_J  # noqa: E402

OUT = os.path.join(HERE, "accuracy_refs.json")
N_SAMPLE = 512


def sample_nodes(rho, fluid, rho_g, rho_l, seed):
    """512 fluid nodes and 512 interface nodes, seeded, as flat indices (y * nx + x)."""
    rng = np.random.default_rng(seed)
    flat = np.flatnonzero(fluid.reshape(-1))
    phi = (rho.reshape(-1) - rho_g) / (rho_l - rho_g)
    iface = np.flatnonzero(fluid.reshape(-1) & (phi > 0.1) & (phi < 0.9))
    a = rng.choice(flat, N_SAMPLE, replace=False)
    b = rng.choice(iface, min(N_SAMPLE, iface.size), replace=False)
    return np.sort(np.concatenate([a, b]))


def field_record(o, info, seed):
    r, vx, vy = o.fields()
    fluid = o.kind()[0] == 0
    idx = sample_nodes(r, fluid, info["rho_g"], info["rho_l"], seed)
    return {"nodes": idx.tolist(), "rho": r.reshape(-1)[idx].tolist(), "vx": vx.reshape(-1)[idx].tolist(),
            "vy": vy.reshape(-1)[idx].tolist(),
            "max_speed": float(np.hypot(vx, vy)[fluid].max())}


def run_c2():
    sc = S.c2_fp32_single()
    o = make_oracle(sc)
    info = o.eos_info()
    d = sc.droplets()
    out = {"scenario": sc.name, "rho_g": info["rho_g"], "rho_l": info["rho_l"], "reports": {}}
    done = 0
    for target in (1000, 5000, 10000, 20000):
        t = time.time()
        o.step(target - done)
        done = target
        print(f"c2: {done} steps ({time.time() - t:.0f} s)", flush=True)
        if done == 1000:
            out["fields_1000"] = field_record(o, info, 2203)
        else:
            r, _, _ = o.fields()
            fluid = o.kind()[0] == 0
            rep = droplet_report(r, fluid, info["rho_g"], info["rho_l"], sc.cx, sc.cy, sc.r, d["x0"], d["y0"], d["r0"])
            rep["mass_change"] = o.mass() / o.mass0() - 1
            out["reports"][str(done)] = rep
    return out


def run_c3():
    sc = S.c3_impact()
    o = make_oracle(sc)
    info = o.eos_info()
    xc = int(round(sc.cx[0]))
    out = {"scenario": sc.name, "x_line": xc, "steps": [], "lower": [], "upper": [], "mass_change": []}
    mid = 0.5 * (info["rho_g"] + info["rho_l"])
    for k in range(6):
        if k:
            o.step(100)
        r, _, _ = o.fields()
        fluid = o.kind()[0] == 0
        ys = isoline_crossings_column(r[:, xc], fluid[:, xc], mid, y_min=sc.cy[0] + sc.r[0] + 5.0)
        out["steps"].append(100 * k)
        out["lower"].append(ys[0])
        out["upper"].append(ys[-1])
        out["mass_change"].append(o.mass() / o.mass0() - 1)
        print(f"c3: {100 * k} steps, interface {ys[0]:.4f} .. {ys[-1]:.4f}", flush=True)
    out["fields_500"] = field_record(o, info, 4096)
    return out


def same_topology(sc, **over):
    a = make_oracle(sc, init=False)
    b = make_oracle(sc.with_(**over), init=False)
    la, lb = a.links(), b.links()
    qa, qb = la["q"], lb["q"]
    return (np.array_equal(a.kind()[0], b.kind()[0]) and np.array_equal(la["x1"], lb["x1"])
            and np.array_equal(la["dir"], lb["dir"]) and np.array_equal(qa < 0.5, qb < 0.5))


def run_c5():
    sc = S.c5_adjoint()
    steps = sc.steps
    t = time.time()
    J, _ = oracle_J(sc, steps)
    print(f"c5: J = {J!r} ({time.time() - t:.0f} s)", flush=True)
    hc = 1e-20
    cs = {"dmu_w": oracle_J(sc, steps, cs=(0, 0, hc))[1] / hc,
          "dmu_w_walls": oracle_J(sc, steps, cs=(0, -1, hc))[1] / hc,
          "cx": oracle_J(sc, steps, cs=(1, 0, hc))[1] / hc,
          "cy": oracle_J(sc, steps, cs=(2, 0, hc))[1] / hc}
    print(f"c5: complex step {cs}", flush=True)
    h = 1e-4
    pert = {"dmu_w": lambda s: dict(dmu_w=[sc.dmu_w[0] + s]),
            "dmu_w_walls": lambda s: dict(dmu_w_walls=sc.dmu_w_walls + s),
            "cx": lambda s: dict(cx=[sc.cx[0] + s]),
            "cy": lambda s: dict(cy=[sc.cy[0] + s])}
    cd = {}
    for name, p in pert.items():
        for s in (h, -h):
            assert same_topology(sc, **p(s)), name
        cd[name] = (oracle_J(sc, steps, **p(h))[0] - oracle_J(sc, steps, **p(-h))[0]) / (2 * h)
    print(f"c5: central differences {cd}", flush=True)
    return {"scenario": sc.name, "steps": steps, "J": J, "complex_step": cs, "central_differences": cd,
            "h_complex": hc, "h_central": h,
            "order": ["dmu_w", "dmu_w_walls", "cx", "cy"]}


def main():
    which = sys.argv[1:] or ["c2", "c3", "c5"]
    refs = json.load(open(OUT)) if os.path.exists(OUT) else {}
    refs["source"] = ("FP64 reference oracle (oracle/), written by tests/golden/make_accuracy_refs.py; "
                      "post-processing by tests/diagnostics.py")
    for w in which:
        refs[w] = {"c2": run_c2, "c3": run_c3, "c5": run_c5}[w]()
        with open(OUT, "w") as fh:
            json.dump(refs, fh, indent=0)


if __name__ == "__main__":
    main()
