"""Writes the contact angle versus wall chemical-potential offset tables.

The paper tunes the wettability through the chemical potential assigned to the solid nodes
(Sec. 2.3) but prints no mapping to the contact angle, so it is measured here with the
reference oracle only: a drop of radius 25 on a flat wall (wall at y = 1.5, q = 1/2) in a
160x80 box, MRT tau = 0.8, k = 0.25, 8000 steps; the angle is read by fitting a circle to
the mid-density isoline (tests/diagnostics.py).

  cs: Carnahan-Starling (a = 1, b = 4, R = 1) at T = 0.6 Tc, kappa^ = 0.05
      -> contact_angle_table.json
  pr: Peng-Robinson with the paper's constants (Eqs. 10-11: a = 2/49, b = 2/21, R = 1,
      omega = 0.344) at T = 0.7 Tc, kappa^ = 0.01 -> contact_angle_table_pr.json

Run:  python tests/golden/make_contact_angle_table.py [cs|pr]
"""
import json
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))
sys.path.insert(0, os.path.join(HERE, ".."))

TABLES = {
    "cs": dict(file="contact_angle_table.json",
               source="reference oracle, flat wall, CS T=0.6Tc, MRT tau=0.8, k=0.25, kappa=0.05",
               physics=dict(eos=1, T_over_Tc=0.6, kappa=0.05),
               offsets=[-0.12, -0.09, -0.06, -0.045, -0.03, -0.015, 0.0, 0.015, 0.03, 0.06, 0.09,
                        0.12, 0.16, 0.2]),
    "pr": dict(file="contact_angle_table_pr.json",
               source="reference oracle, flat wall, PR a=2/49 b=2/21 omega=0.344 T=0.7Tc, MRT tau=0.8, "
                      "k=0.25, kappa=0.01",
               physics=dict(eos=2, a=2 / 49, b=2 / 21, T_over_Tc=0.7, kappa=0.01),
               offsets=[-0.1, -0.08, -0.06, -0.05, -0.04, -0.03, -0.02, -0.01, 0.0, 0.01, 0.02, 0.03,
                        0.04, 0.05, 0.06, 0.08, 0.1]),
}


def measure(args, steps=8000, nx=160, ny=80):
    physics, dmu = args
    import oracle as O
    from diagnostics import contact_angle_flat
    O.set_threads(2)
    cfg = O.OracleConfig(nx=nx, ny=ny, walls=1, y_bottom=1.5, k=0.25, coll=O.COLL_MRT, tau=0.8,
                         dmu_w_walls=dmu, **physics)
    o = O.Oracle(cfg)
    info = o.eos_info()
    o.init_droplets([nx / 2], [1.5 + 10], [25.0], 5.0)
    o.step(steps)
    r, vx, vy = o.fields()
    kind, _ = o.kind()
    return contact_angle_flat(r, kind == 0, info["rho_g"], info["rho_l"], 1.5)


def main(which):
    t = TABLES[which]
    import oracle as O
    O.build()
    with mp.get_context("spawn").Pool(4) as pool:
        thetas = pool.map(measure, [(t["physics"], d) for d in t["offsets"]])
    out = {"source": t["source"], "dmu": t["offsets"], "theta_deg": [round(x, 3) for x in thetas]}
    with open(os.path.join(HERE, t["file"]), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "cs")
