"""Writes rt64_re4000_fronts.txt: bubble-front and spike-tip positions of the FP64
oracle for the Rayleigh-Taylor instability on the 64 x 64 x 256 box at Re = 4000
(At = 0.5, sqrt(gW) = 0.04, D = 4, sigma = 1e-4, Pe = 50; Sec. III C) at
t* = t sqrt(gW) / W = 1, 2, 3.

Calls only the oracle and the seeded input generators.  Fronts: along the column
x = y = 0 (where h of Eq. 42 is largest) the bubble front is the highest phi = 0
crossing; along x = y = W/2 the spike tip is the lowest one; linear interpolation
between nodes z_k = k + 1/2; reported as (z - 2W) / W.

Run: python tests/golden/make_rt_fronts.py   (about two hours on one CPU core)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import lbm_oracle as O  # noqa: E402
from paper_1507_07294_gb300 import inputs as I  # noqa: E402

W, RE = 64, 4000.0
STEPS = (1600, 3200, 4800)


def crossings(profile, z):
    k = np.flatnonzero(np.sign(profile[:-1]) * np.sign(profile[1:]) < 0)
    return z[k] - profile[k] * (z[k + 1] - z[k]) / (profile[k + 1] - profile[k])


def main(out=os.path.join(HERE, "rt64_re4000_fronts.txt")):
    w = I.rayleigh_taylor(W=W, Re=RE)
    o = O.Oracle(O.Params.from_workload(w))
    o.init(w.phi0)
    z = np.arange(w.nz) + 0.5
    rows = []
    for target in STEPS:
        o.step(target - o.t)
        phi = O.order_parameter(o.f)
        bubble = crossings(phi[:, 0, 0], z).max()
        spike = crossings(phi[:, W // 2, W // 2], z).min()
        tstar = target * 0.04 / W
        rows.append((target, tstar, (bubble - 2 * W) / W, (spike - 2 * W) / W))
        print(rows[-1], flush=True)
    with open(out, "w") as fh:
        fh.write("# FP64 oracle, Rayleigh-Taylor 64x64x256, Re = 4000, At = 0.5 (Sec. III C);\n")
        fh.write("# written by tests/golden/make_rt_fronts.py (oracle only).\n")
        fh.write("# columns: step, t*, bubble front (z - 2W)/W, spike tip (z - 2W)/W\n")
        for r in rows:
            fh.write(f"{r[0]} {r[1]:.6f} {r[2]:.8f} {r[3]:.8f}\n")


if __name__ == "__main__":
    main()
