"""Every configuration bench.py times, at its full size and in the launch configuration
the bench uses, against the FP64 oracle (needs a GPU).

The main line (256 x 256 x 1024 Rayleigh-Taylor, FP32, two arrays) is covered in
test_gpu_parity.py; here are the bench's other lines on the same grid -- 16-bit
populations (FP16, BF16), the in-place pattern (FP32 and FP16), the single-pass step,
the SRT flow lattice, the D3Q7-weighted stencils -- and interface tracking on its
256^3 deformation box.  Each runs a few steps on the GPU (graph replays of step pairs
included), then one more; at 100 seeded cells (plus the box corners) the oracle takes
the same step from the state of a 9^3 patch around the cell, read from the GPU with
lbm_read_state_at, so no whole state leaves the device.

Tolerances: FP32 storage, a few FP32 ulps of the population magnitudes (2e-6 of the
largest); 16-bit storage, the rounding of the stored result, half an ulp relative
(2^-11 for FP16, 2^-8 for BF16) plus the FP32 allowance, and for FP16, whose values
below 2^-14 are subnormal with a fixed spacing of 2^-24, half that spacing absolute.
"""
import numpy as np
import pytest

from oracle import lbm_oracle as O
from paper_1507_07294_gb300 import inputs as I
from tests.patch_oracle import one_step_on_patch, patch_axes, sample_cells

pytestmark = pytest.mark.gpu

REL = {"fp32": 0.0, "fp16": 2.0 ** -11, "bf16": 2.0 ** -8}
ABS = {"fp32": 0.0, "fp16": 2.0 ** -25, "bf16": 0.0}


@pytest.fixture(scope="module")
def L():
    from paper_1507_07294_gb300 import lbm
    lbm.load_library()
    return lbm


def _rt256(**kw):
    from dataclasses import replace
    w = I.rayleigh_taylor(W=256, Re=4000.0)
    return replace(w, **kw) if kw else w


LINES = {
    "fp16": dict(storage="fp16"),
    "bf16": dict(storage="bf16"),
    "aa": dict(pattern="aa"),
    "aa_fp16": dict(pattern="aa", storage="fp16"),
    "single_pass": dict(fused=True),
    "srt_flow": dict(variant=dict(srt_flow=True)),
    "d3q7_stencil": dict(variant=dict(stencil="d3q7")),
    "interface_tracking": dict(tracking=True),
}


@pytest.mark.parametrize("line", list(LINES))
def test_bench_line_at_full_size_one_step(L, line):
    cfg = LINES[line]
    storage = cfg.get("storage", "fp32")
    w = I.deformation(n=256) if cfg.get("tracking") else _rt256(**cfg.get("variant", {}))
    warm = 9
    p = O.Params.from_workload(w)
    cells = sample_cells(w.shape, 100, seed=41)
    with L.Solver(w, pattern=cfg.get("pattern", "ab"), storage=storage) as s:
        if cfg.get("fused"):
            L.lbm_set_tuning(s.ctx, L.LBM_TUNE_FUSED, 1)
            assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_FUSED) == 1
        s.step(warm)
        patches = []
        for cell in cells:
            zs, ys, xs, zc = patch_axes(p, w.shape, cell)
            lin = ((zs[:, None, None] * w.ny + ys[None, :, None]) * w.nx
                   + xs[None, None, :]).reshape(-1)
            f, g, phiu, t = s.state_at(lin)
            shape = (len(zs), len(ys), len(xs))
            patches.append((zs, ys, xs, zc, f.reshape((7,) + shape), g.reshape((15,) + shape),
                            phiu.reshape((3,) + shape)))
        assert t == warm
        s.step(1)
        f1, g1, _, _ = s.state_at(np.array(cells))
    of, og = [], []
    for zs, ys, xs, zc, f, g, phiu in patches:
        a, b = one_step_on_patch(p, zs, ys, xs, zc, f, g, phiu, t=warm)
        of.append(a)
        og.append(b)
    of, og = np.array(of).T, np.array(og).T
    rel, floor = REL[storage], ABS[storage]
    tol_f = rel * np.abs(of) + floor + 2e-6 * max(1.0, np.abs(of).max())
    assert np.all(np.abs(f1 - of) <= tol_f), f"max |df| = {np.abs(f1 - of).max():.3e}"
    if not cfg.get("tracking"):
        tol_g = rel * np.abs(og) + floor + 2e-6 * np.abs(og).max() + 1e-9
        assert np.all(np.abs(g1 - og) <= tol_g), f"max |dg| = {np.abs(g1 - og).max():.3e}"
