"""Writes tests/golden/spinodal128_oracle.json: the FP64 oracle's domain size
L(t) (§4, squared structure factor) and interface area every 100 steps of
the 128^3 spinodal recipe (both components 0.7 +- 0.01, g = 0.1, tau = 1,
periodic, 2000 steps).  Calls only the oracle and the input generators.

    python tests/golden/make_spinodal_golden.py [--n 128] [--steps 2000] [--every 100]
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import analysis, lbref  # noqa: E402
from paper_1109_3277_gb300 import workloads as W  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--every", type=int, default=100)
    a = ap.parse_args()
    w = W.spinodal(n=a.n, steps=a.steps)
    lat = lbref.Lattice(w.shape, w.rho0, **w.params)
    out = {"workload": w.name, "recipe": "spinodal(seed=1111): both components 0.7 + U[-0.01, 0.01), "
           "g=0.1, tau=1, periodic", "every": a.every, "steps": [], "L": [], "Lxyz": [], "area": [],
           "mass": []}
    t0 = time.time()
    for s in range(a.every, a.steps + 1, a.every):
        lat.step(a.every)
        rho, _, _ = lat.read_fields()
        L, Lxyz = analysis.domain_size(rho)
        out["steps"].append(s)
        out["L"].append(L)
        out["Lxyz"].append(list(Lxyz))
        out["area"].append(analysis.interface_area(rho))
        out["mass"].append(list(lat.mass()))
        print(f"step {s}: L={L:.4f} area={out['area'][-1]} ({time.time() - t0:.0f} s)", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"spinodal{a.n}_oracle.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(path)


if __name__ == "__main__":
    main()
