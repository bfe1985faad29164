"""Write tests/golden/oracle_c0_ledger.json from the FP64 CPU oracle.

The stored values are the oracle's own (this paper prints no worked example
of the scheme): five steps of the 64x32 double Harris sheet, seed 0, with the
per-step energy ledger and field norms. They pin the oracle against silent
regressions. Run from the repository root:  python tests/golden/make_oracle_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from relsim_inputs import HarrisConfig, make_harris  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_c0_ledger.json")


def run(nsteps=5):
    hc = HarrisConfig()
    s = make_harris(hc)
    c = oracle.make_config(hc.nx, hc.ny, dt=hc.dt, theta=hc.theta, gmres_tol=1e-12,
                           gmres_restart=50)
    P = oracle.Particles(s["species"])
    E, B = s["E"], s["B"]
    rows = []
    for n in range(nsteps):
        E, B, led, _ = oracle.step(c, P, E, B)
        led = {k: v for k, v in led.items()}
        led["E_l2"] = float(np.sqrt((E * E).sum()))
        led["B_l2"] = float(np.sqrt((B * B).sum()))
        led["ux_sum"] = float(P.ux.sum())
        led["x_sum"] = float(P.x.sum())
        rows.append(led)
    return {"workload": "double Harris sheet 64x32, 16 ppc per species, seed 0, dt 0.5, theta 0.5",
            "source": "FP64 CPU oracle (oracle/relsim_oracle.c), gmres_tol 1e-12, restart 50",
            "steps": rows}


if __name__ == "__main__":
    with open(OUT, "w") as f:
        json.dump(run(), f, indent=1)
    print(OUT)
