"""Oracle evaluation of one time step at sampled cells of a large grid.

The new populations of a cell after one step depend on the state within distance 3
of it (post-streaming value <- post-collision values at distance 1 <- lap mu at
distance 1 <- phi at distance 3).  So the oracle's step on a (2R+1)^3 patch around a
cell, R >= 3, gives that cell's exact FP64 result; only the patch rim is wrong.
Between z walls the patch is clipped to the domain and keeps the walls.
"""
from dataclasses import replace

import numpy as np

from oracle import lbm_oracle as O


def one_step_at(params: O.Params, f, g, phiu_prev, have_prev: bool, cells, R: int = 4,
                t: int = 1):
    """FP64 populations (f[7], g[15]) after one oracle step at each (z, y, x) in cells,
    starting from the given full state (arrays [q, z, y, x]) at step count t (which only
    matters for a time-dependent prescribed velocity)."""
    nz, ny, nx = f.shape[1:]
    if nx < 2 * R + 1 or ny < 2 * R + 1 or (not params.walls_z and nz < 2 * R + 1):
        raise ValueError("grid too small for the patch method")
    out_f, out_g = [], []
    for (z, y, x) in cells:
        xs = (x + np.arange(-R, R + 1)) % nx
        ys = (y + np.arange(-R, R + 1)) % ny
        if params.walls_z:
            zs = np.arange(max(0, z - R), min(nz, z + R + 1))
            zc = z - zs[0]
        else:
            zs = (z + np.arange(-R, R + 1)) % nz
            zc = R
        ix = np.ix_(zs, ys, xs)
        p = replace(params, nx=len(xs), ny=len(ys), nz=len(zs))
        o = O.Oracle(p, box=(nz, ny, nx), coords=(zs[:, None, None], ys[None, :, None],
                                                  xs[None, None, :]))
        o.f = np.stack([a[ix] for a in f]).astype(np.float64)
        o.g = np.stack([a[ix] for a in g]).astype(np.float64)
        o.phiu_prev = np.stack([a[ix] for a in phiu_prev]).astype(np.float64) if have_prev else None
        o.t = t
        o.step(1)
        out_f.append(o.f[:, zc, R, R])
        out_g.append(o.g[:, zc, R, R])
    return np.array(out_f), np.array(out_g)


def sample_cells(shape, n: int, seed: int = 0, include_edges: bool = True):
    """n seeded cells (z, y, x), plus the corners of the box when include_edges."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    cells = [tuple(int(v) for v in (rng.integers(nz), rng.integers(ny), rng.integers(nx)))
             for _ in range(n)]
    if include_edges:
        for z in (0, nz - 1):
            for y in (0, ny - 1):
                for x in (0, nx - 1):
                    cells.append((z, y, x))
    return cells
