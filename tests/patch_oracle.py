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


def patch_axes(params: O.Params, shape, cell, R: int = 4):
    """Grid coordinates (zs, ys, xs) of the patch around cell (z, y, x), periodic images
    folded in, clipped at z walls, and the cell's z position zc within it."""
    nz, ny, nx = shape
    if nx < 2 * R + 1 or ny < 2 * R + 1 or (not params.walls_z and nz < 2 * R + 1):
        raise ValueError("grid too small for the patch method")
    z, y, x = cell
    xs = (x + np.arange(-R, R + 1)) % nx
    ys = (y + np.arange(-R, R + 1)) % ny
    if params.walls_z:
        zs = np.arange(max(0, z - R), min(nz, z + R + 1))
        zc = z - zs[0]
    else:
        zs = (z + np.arange(-R, R + 1)) % nz
        zc = R
    return zs, ys, xs, zc


def one_step_on_patch(params: O.Params, zs, ys, xs, zc, f, g, phiu_prev, R: int = 4,
                      t: int = 1):
    """FP64 (f[7], g[15]) after one oracle step at the centre cell of a patch whose
    state (arrays [q, len(zs), len(ys), len(xs)]; phiu_prev None when there is no
    previous step) is given."""
    p = replace(params, nx=len(xs), ny=len(ys), nz=len(zs))
    o = O.Oracle(p, box=(params.nz, params.ny, params.nx),
                 coords=(zs[:, None, None], ys[None, :, None], xs[None, None, :]))
    o.f = np.asarray(f, dtype=np.float64)
    o.g = np.asarray(g, dtype=np.float64)
    o.phiu_prev = None if phiu_prev is None else np.asarray(phiu_prev, dtype=np.float64)
    o.t = t
    o.step(1)
    return o.f[:, zc, R, R], o.g[:, zc, R, R]


def one_step_at(params: O.Params, f, g, phiu_prev, have_prev: bool, cells, R: int = 4,
                t: int = 1):
    """FP64 populations (f[7], g[15]) after one oracle step at each (z, y, x) in cells,
    starting from the given full state (arrays [q, z, y, x]) at step count t (which only
    matters for a time-dependent prescribed velocity)."""
    out_f, out_g = [], []
    for cell in cells:
        zs, ys, xs, zc = patch_axes(params, f.shape[1:], cell, R)
        ix = np.ix_(zs, ys, xs)
        of, og = one_step_on_patch(
            params, zs, ys, xs, zc, np.stack([a[ix] for a in f]), np.stack([a[ix] for a in g]),
            np.stack([a[ix] for a in phiu_prev]) if have_prev else None, R, t)
        out_f.append(of)
        out_g.append(og)
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
