"""Grid-size limits on the GPU (needs a GPU): the largest grid the C ABI admits, and
grids longer than a launch grid's y and z extents allow per dimension.

lbm_create admits grids of fewer than 2^31 - 64 cells.  The largest with whole pairs of
tiles in every row (nx a multiple of 64, the two-cells-per-thread stream-collide) is
2^31 - 128 = 128 x 1365 x 12291 cells, where every per-cell index is within 128 of
INT_MAX and the state's byte offsets run past 100 GB; with 16-bit populations in place
(LBM_PATTERN_AA, 93 B per cell) its context takes 200 GB.

The initial condition is periodic with periods (17, 15, 64) in (z, y, x), which divide
the grid, and the grid is periodic in every direction, so each cell of the big grid
computes exactly what the matching cell of a 17 x 15 x 64 grid computes, step after
step (the per-cell arithmetic does not depend on where the cell sits).  So the big
grid's state at cells sampled over its whole index range, the first and last cells
among them, must equal the small grid's bit for bit, after steps of both parities and
graph replays; its FP64 sums must be the small grid's times the number of periods; and
the small grid itself is compared with the FP64 oracle.

Skipped when the GPU has less than the context plus the 17 GB FP64 upload buffer free,
or the host less than about 30 GB of memory available.
"""
import gc
from dataclasses import replace

import numpy as np
import pytest

from oracle import lbm_oracle as O
from paper_1507_07294_gb300 import inputs as I

pytestmark = pytest.mark.gpu

NX, NY, NZ = 128, 1365, 12291          # 2^31 - 128 cells
PX, PY, PZ = 64, 15, 17                # periods of the initial condition
STEPS = 5


def _host_available_bytes() -> int:
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


@pytest.fixture(scope="module")
def L():
    from paper_1507_07294_gb300 import lbm
    lbm.load_library()
    return lbm


def _small_workload():
    w = I.droplet(n=PY, R=5.0, D=4.0, nx=PX, ny=PY, nz=PZ)
    return I.perturbed(w, seed=31, phi_amp=0.05)


def test_largest_admitted_grid_equals_its_period(L):
    import torch
    n = NX * NY * NZ
    assert n == 2 ** 31 - 128

    small = _small_workload()
    big = replace(small, name="periodic_max", nx=NX, ny=NY, nz=NZ, phi0=None)
    grid, params = L.params_from_workload(big, pattern="aa", storage="fp16")
    need = L.lbm_memory_bytes(grid, params) + 8 * n + (2 << 30)
    free, _ = torch.cuda.mem_get_info()
    if free < need:
        pytest.skip(f"needs {need / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")
    if _host_available_bytes() < 8 * n + (12 << 30):
        pytest.skip("needs about 30 GB of available host memory")

    # the small grid: state after STEPS steps, sums, and the oracle's phi
    with L.Solver(small, pattern="aa", storage="fp16") as s:
        s.step(STEPS)
        f_s, g_s, p_s, t_s = s.state()
        mass_s, mom_s = s.reduce()
        phi_s = s.fields(L.LBM_FIELD_PHI)["phi"]
    o = O.Oracle(O.Params.from_workload(small))
    o.init(small.phi0)
    o.step(STEPS)
    # 16-bit populations against FP64 after a few steps (the tolerance of the 16-bit
    # precision tests after 100 steps)
    assert np.abs(phi_s - o.fields()["phi"]).max() <= 5e-4

    # the big grid: the same initial condition repeated (one 17 GB host array)
    reps = (NZ // PZ, NY // PY, NX // PX)
    phi_big = np.broadcast_to(small.phi0[None, :, None, :, None, :],
                              (reps[0], PZ, reps[1], PY, reps[2], PX)).reshape(NZ, NY, NX)
    big = replace(big, phi0=phi_big)
    del phi_big
    rng = np.random.default_rng(32)
    lin = np.concatenate([rng.integers(0, n, 4000), np.arange(64), n - 1 - np.arange(64),
                          [n // 2, 2 ** 30, 2 ** 31 - 256]]).astype(np.int64)
    try:
        with L.Solver(big, pattern="aa", storage="fp16") as b:
            big.phi0 = None
            gc.collect()
            b.step(STEPS)
            f_b, g_b, p_b, t_b = b.state_at(lin)
            mass_b, mom_b = b.reduce()
    finally:
        big = None
        gc.collect()
        torch.cuda.empty_cache()
    assert t_b == t_s == STEPS
    z, r = np.divmod(lin, NX * NY)
    y, x = np.divmod(r, NX)
    zs, ys, xs = z % PZ, y % PY, x % PX
    for name, got, ref in (("f", f_b, f_s), ("g", g_b, g_s), ("phi u", p_b, p_s)):
        want = ref[:, zs, ys, xs]
        assert np.array_equal(got, want), f"{name}: {int((got != want).sum())} values differ"
    copies = reps[0] * reps[1] * reps[2]
    # the same FP32 phi values summed in FP64 in another order
    assert abs(mass_b - copies * mass_s) <= 1e-3
    np.testing.assert_allclose(mom_b, copies * np.asarray(mom_s), rtol=1e-6,
                               atol=1e-9 * n)


@pytest.mark.parametrize("shape,period", [((1100 * 1000, 1, 1), (1100, 1, 1)),
                                          ((2, 600 * 1000, 1), (2, 600, 1))])
def test_long_thin_grids_equal_their_period(L, shape, period):
    """Grids longer than 65535 bricks of the chemical-potential pass in z (nz > 1048560)
    or in y (ny > 524280): a column of 1.1M cells and a strip of 0.6M rows, periodic,
    with an initial condition of period 1100 (600) along their long axis, step exactly
    as the one-period grid does, bit for bit, at every cell."""
    nz, ny, nx = shape
    pz, py, px = period
    rng = np.random.default_rng(33)
    m = max(pz, py)  # the long axis' period
    prof = np.clip(np.tanh(4.0 * np.sin(np.linspace(0.0, 2.0 * np.pi, m, endpoint=False)))
                   + 0.02 * rng.uniform(-1, 1, m), -1.0, 1.0)
    if pz > py:
        phi_small = prof.reshape(pz, 1, 1)
    else:
        phi_small = np.broadcast_to(prof[None, :, None], (pz, py, px)).copy()
    base = I.droplet(n=4, R=1.0)
    small = replace(base, name="period", nx=px, ny=py, nz=pz, phi0=phi_small)
    big = replace(base, name="long", nx=nx, ny=ny, nz=nz,
                  phi0=np.tile(phi_small, (nz // pz, ny // py, nx // px)))
    with L.Solver(small) as s, L.Solver(big) as b:
        s.step(4)
        b.step(4)
        fs, gs, ps, _ = s.state()
        fb, gb, pb, _ = b.state()
    reps = (nz // pz, ny // py, nx // px)
    for name, got, ref in (("f", fb, fs), ("g", gb, gs), ("phi u", pb, ps)):
        want = np.tile(ref, (1,) + reps)
        assert np.array_equal(got, want), f"{name}: {int((got != want).sum())} values differ"
