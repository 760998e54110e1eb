"""Writes surface_tension.json: the surface tension of the chemical-potential model (CS,
T = 0.6 Tc, k = 0.25, kappa^ = 0.05), which sets the Bond number of the drop-impact runs
(Sec. 4.5, Bo = g (rho_l - rho_g) D^2 / sigma).  The paper gives no value for its own units, so
it is measured here with the reference oracle only, by the Laplace law of two static drops
(96 x 96 periodic, MRT tau = 0.8, 20000 steps): in 2D the pressure jump k^2 [p0(rho_in) -
p0(rho_out)] times the equimolar radius is sigma.  The Maxwell densities of the same EOS are
stored beside it (the Bond number uses rho_l - rho_g).

Run:  python tests/golden/make_surface_tension.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "..", ".."))

import oracle as O  # noqa: E402

PHYS = dict(eos=O.EOS_CS, T_over_Tc=0.6, k=0.25, kappa=0.05)


def laplace(R0, n=96, steps=20000):
    cfg = O.OracleConfig(nx=n, ny=n, walls=0, coll=O.COLL_MRT, tau=0.8, **PHYS)
    o = O.Oracle(cfg)
    o.init_droplets([n / 2], [n / 2], [R0], 5.0)
    o.step(steps)
    r = o.fields()[0]
    rin, rout = r[n // 2, n // 2], r[2, 2]
    p, _, _ = O.eos_eval(cfg, [rin, rout])
    dp = cfg.k ** 2 * (p[0] - p[1])
    req = float(np.sqrt((r.sum() - rout * n * n) / (np.pi * (rin - rout))))
    return float(dp), req


def main():
    rows = {R0: laplace(R0) for R0 in (16.0, 24.0)}
    sig = [dp * req for dp, req in rows.values()]
    _, _, info = O.eos_eval(O.OracleConfig(nx=8, ny=8, **PHYS), [1.0])
    out = {"source": "reference oracle, Laplace law of static drops, CS T=0.6Tc, k=0.25, kappa=0.05, MRT tau=0.8",
           "T_over_Tc": 0.6, "k": 0.25, "kappa": 0.05, "rho_g": info["rho_g"], "rho_l": info["rho_l"],
           "drops": [{"r0": R0, "dp": dp, "r_equimolar": req} for R0, (dp, req) in rows.items()],
           "sigma": float(np.mean(sig))}
    with open(os.path.join(HERE, "surface_tension.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
