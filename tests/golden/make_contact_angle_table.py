"""Writes contact_angle_table.json: contact angle versus wall chemical-potential offset.

The paper tunes the wettability through the chemical potential assigned to the solid nodes
(Sec. 2.3) but prints no mapping to the contact angle, so it is measured here with the
reference oracle only: a drop of radius 25 on a flat wall (wall at y = 1.5, q = 1/2) in a
160x80 box, CS EOS at T = 0.6 Tc, MRT tau = 0.8, k = 0.25, kappa^ = 0.05, 8000 steps; the
angle is read by fitting a circle to the mid-density isoline (tests/diagnostics.py).

Run:  python tests/golden/make_contact_angle_table.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))
sys.path.insert(0, os.path.join(HERE, ".."))

from oracle import Oracle, OracleConfig, EOS_CS, COLL_MRT  # noqa: E402
from diagnostics import contact_angle_flat  # noqa: E402

OFFSETS = [-0.12, -0.09, -0.06, -0.045, -0.03, -0.015, 0.0, 0.015, 0.03, 0.06, 0.09, 0.12, 0.16, 0.2]


def measure(dmu, steps=8000, nx=160, ny=80):
    cfg = OracleConfig(nx=nx, ny=ny, walls=1, y_bottom=1.5, eos=EOS_CS, T_over_Tc=0.6, k=0.25,
                       kappa=0.05, coll=COLL_MRT, tau=0.8, dmu_w_walls=dmu)
    o = Oracle(cfg)
    info = o.eos_info()
    o.init_droplets([nx / 2], [1.5 + 10], [25.0], 5.0)
    o.step(steps)
    r, vx, vy = o.fields()
    kind, _ = o.kind()
    return contact_angle_flat(r, kind == 0, info["rho_g"], info["rho_l"], 1.5)


def main():
    rows = [(d, measure(d)) for d in OFFSETS]
    out = {"source": "reference oracle, flat wall, CS T=0.6Tc, MRT tau=0.8, k=0.25, kappa=0.05",
           "dmu": [r[0] for r in rows], "theta_deg": [round(r[1], 3) for r in rows]}
    with open(os.path.join(HERE, "contact_angle_table.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
