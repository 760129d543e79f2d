"""Writes rt64_fronts.txt: bubble-front and spike-tip positions of the FP64 oracle for
the Rayleigh-Taylor instability (Sec. III C) on the 64 x 64 x 256 box: At = 0.5,
sqrt(gW) = 0.04, D = 4, sigma = 1e-4, Pe = 50, at t* = t sqrt(gW) / W = 0.5 and 1 for
Re = 256 and Re = 4000.  Later times are left out: with sigma = 1e-4 the order
parameter overshoots +-1 more and more as the interface is carried (the D3Q7 scheme
gives phi no numerical diffusion, and the Cahn-Hilliard restoring term is tiny at this
sigma): the Re = 4000 run diverges before t* = 2 in the oracle itself, and both
diverge before t* = 2 in the CUDA path.

Calls only the oracle and the seeded input generators.  Fronts: along the column
x = y = 0 (where h of Eq. 42 is largest) the bubble front is the highest phi = 0
crossing; along x = y = W/2 the spike tip is the lowest one; linear interpolation
between nodes z_k = k + 1/2; reported as (z - nz/2) / W.

Run: python tests/golden/make_rt_fronts.py   (about 45 minutes; the two Reynolds
numbers run in parallel processes)
"""
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))

W = 64
CASES = ((256.0, (800, 1600)), (4000.0, (800, 1600)))


def crossings(profile, z):
    k = np.flatnonzero(np.sign(profile[:-1]) * np.sign(profile[1:]) < 0)
    return z[k] - profile[k] * (z[k + 1] - z[k]) / (profile[k + 1] - profile[k])


def run_case(case):
    re, steps = case
    sys.path.insert(0, ROOT)
    from oracle import lbm_oracle as O
    from paper_1507_07294_gb300 import inputs as I
    w = I.rayleigh_taylor(W=W, Re=re)
    o = O.Oracle(O.Params.from_workload(w))
    o.init(w.phi0)
    z = np.arange(w.nz) + 0.5
    rows = []
    for target in steps:
        o.step(target - o.t)
        phi = O.order_parameter(o.f)
        bubble = crossings(phi[:, 0, 0], z).max()
        spike = crossings(phi[:, W // 2, W // 2], z).min()
        rows.append((re, target, target * 0.04 / W, (bubble - w.nz / 2) / W,
                     (spike - w.nz / 2) / W))
        print(rows[-1], flush=True)
    return rows


def main(out=os.path.join(HERE, "rt64_fronts.txt")):
    with mp.get_context("spawn").Pool(len(CASES)) as pool:
        results = pool.map(run_case, CASES)
    with open(out, "w") as fh:
        fh.write("# FP64 oracle, Rayleigh-Taylor 64x64x256, At = 0.5 (Sec. III C);\n")
        fh.write("# written by tests/golden/make_rt_fronts.py (oracle only).\n")
        fh.write("# columns: Re, step, t*, bubble front (z - nz/2)/W, spike tip (z - nz/2)/W\n")
        for rows in results:
            for r in rows:
                fh.write(f"{r[0]:g} {r[1]} {r[2]:.6f} {r[3]:.8f} {r[4]:.8f}\n")


if __name__ == "__main__":
    main()
