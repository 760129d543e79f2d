"""The stream-collide pass with two cells per thread (LBM_TUNE_CELL_PAIRS) against the
one-cell pass (needs a GPU).

Both run the same per-cell arithmetic, written with explicit rounding: the paired
kernel does each step for two cells at once in the two lanes of a paired FP32
instruction, which rounds each lane like the scalar instruction.  So the states agree
bit for bit: walled and periodic grids, all storage types, the model variants, the
fused step sums and the graph replays.
"""
import numpy as np
import pytest

from paper_1507_07294_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1507_07294_gb300 import lbm
    lbm.load_library()
    return lbm


def _workload(case, seed):
    if case == "walls":
        w = I.perturbed(I.rayleigh_taylor(W=64, nz=24, Re=300.0), seed=seed, phi_amp=0.03,
                        u_amp=0.01, p_amp=1e-3)
        w.ny = 12
        w.phi0 = np.ascontiguousarray(w.phi0[:, :12, :])
        w.u0 = np.ascontiguousarray(w.u0[:, :, :12, :])
        w.p0 = np.ascontiguousarray(w.p0[:, :12, :])
        return w
    return I.perturbed(I.droplet(n=64, R=6.0, nx=128, ny=10, nz=12), seed=seed, phi_amp=0.02,
                       u_amp=0.01, p_amp=1e-3)


def _same(a, b):
    for x, y, name in zip(a.state()[:3], b.state()[:3], ("f", "g", "phiu")):
        assert np.array_equal(x, y), f"{name}: {int((x != y).sum())} values differ"


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("case", ["walls", "periodic"])
def test_pairs_equal_single_cells(L, storage, case):
    w = _workload(case, seed=21)
    st = L.STORAGES[storage]
    with L.Solver(w, storage=st) as a, L.Solver(w, storage=st) as b:
        assert L.lbm_get_tuning(a.ctx, L.LBM_TUNE_CELL_PAIRS) == 1
        L.lbm_set_tuning(b.ctx, L.LBM_TUNE_CELL_PAIRS, 0)
        assert L.lbm_get_tuning(b.ctx, L.LBM_TUNE_CELL_PAIRS) == 0
        for n in (1, 2, 5):
            a.step(n)
            b.step(n)
            _same(a, b)
        for n in (1, 3):
            ra = L.lbm_step_reduce(a.ctx, n)
            rb = L.lbm_step_reduce(b.ctx, n)
            assert ra[0] == rb[0] and np.array_equal(ra[1], rb[1])
        _same(a, b)


@pytest.mark.parametrize("variant", ["srt_flow", "d3q7_stencil"])
def test_pairs_equal_single_cells_for_the_variants(L, variant):
    w = _workload("walls", seed=22)
    setattr(w, variant if variant == "srt_flow" else "stencil",
            True if variant == "srt_flow" else "d3q7")
    with L.Solver(w) as a, L.Solver(w) as b:
        L.lbm_set_tuning(b.ctx, L.LBM_TUNE_CELL_PAIRS, 0)
        a.step(4)
        b.step(4)
        _same(a, b)


def test_pairs_only_where_they_apply(L):
    w = I.droplet(n=32, R=6.0)  # nx = 32: not a pair of tiles per row
    with L.Solver(w) as s:
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_CELL_PAIRS) == 0
    w = _workload("walls", seed=23)
    with L.Solver(w, pattern=L.LBM_PATTERN_AA) as s:
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_CELL_PAIRS) == 1
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_STENCIL_STAGE) == 1  # FP32 default
        with pytest.raises(L.LbmError):
            L.lbm_set_tuning(s.ctx, L.LBM_TUNE_CELL_PAIRS, 2)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("case", ["walls", "periodic"])
def test_staged_stencils_equal_loaded_stencils(L, storage, case):
    """LBM_TUNE_STENCIL_STAGE: the two-cell pass fetching its blocks' phi and mu rows
    into shared memory by TMA bulk copies reads the same values as the per-cell stencil
    loads (nx = 64 walled, 128 periodic: 4 and 2 rows per block)."""
    w = _workload(case, seed=24)
    st = L.STORAGES[storage]
    with L.Solver(w, storage=st) as a, L.Solver(w, storage=st) as b, L.Solver(w, storage=st) as c:
        # on by default with FP32 populations only
        assert L.lbm_get_tuning(a.ctx, L.LBM_TUNE_STENCIL_STAGE) == (storage == "fp32")
        L.lbm_set_tuning(a.ctx, L.LBM_TUNE_STENCIL_STAGE, 1)
        assert L.lbm_get_tuning(a.ctx, L.LBM_TUNE_STENCIL_STAGE) == 1
        L.lbm_set_tuning(b.ctx, L.LBM_TUNE_STENCIL_STAGE, 0)
        assert L.lbm_get_tuning(b.ctx, L.LBM_TUNE_STENCIL_STAGE) == 0
        L.lbm_set_tuning(c.ctx, L.LBM_TUNE_CELL_PAIRS, 0)
        assert L.lbm_get_tuning(c.ctx, L.LBM_TUNE_STENCIL_STAGE) == 0
        for n in (1, 2, 4):
            for s in (a, b, c):
                s.step(n)
            _same(a, b)
            _same(a, c)


def test_staged_stencils_for_the_variants_and_grid_shapes(L):
    for variant in ("srt_flow", "d3q7_stencil"):
        w = _workload("walls", seed=25)
        setattr(w, variant if variant == "srt_flow" else "stencil",
                True if variant == "srt_flow" else "d3q7")
        with L.Solver(w) as a, L.Solver(w) as b:
            L.lbm_set_tuning(b.ctx, L.LBM_TUNE_STENCIL_STAGE, 0)
            a.step(3)
            b.step(3)
            _same(a, b)
    # a block's 256 cells straddle two planes (64 x 10 planes of 640 cells) and the last
    # block is half full (n = 64 x 10 x 3 = 1920 = 7.5 blocks)
    w = I.perturbed(I.droplet(n=64, R=4.0, nx=64, ny=10, nz=3), seed=26, phi_amp=0.02,
                    u_amp=0.01, p_amp=1e-3)
    with L.Solver(w) as a, L.Solver(w) as b:
        assert L.lbm_get_tuning(a.ctx, L.LBM_TUNE_STENCIL_STAGE) == 1
        L.lbm_set_tuning(b.ctx, L.LBM_TUNE_CELL_PAIRS, 0)
        a.step(3)
        b.step(3)
        _same(a, b)
    # nx = 192: pairs, but rows of 192 cells do not tile a block of 256: no staging
    w = I.droplet(n=32, R=6.0, nx=192, ny=4, nz=4)
    with L.Solver(w) as s:
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_CELL_PAIRS) == 1
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_STENCIL_STAGE) == 0


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("case", ["walls", "periodic"])
def test_in_place_pattern_pairs(L, storage, case):
    """The in-place pattern with two cells per thread (both of its steps, in place)
    equals it with one cell per thread and equals the two-array pattern, across odd and
    even step counts, graph replays and the fused step sums."""
    w = _workload(case, seed=28)
    st = L.STORAGES[storage]
    with L.Solver(w, storage=st, pattern=L.LBM_PATTERN_AA) as a, \
            L.Solver(w, storage=st, pattern=L.LBM_PATTERN_AA) as b, \
            L.Solver(w, storage=st, pattern=L.LBM_PATTERN_AA) as d, \
            L.Solver(w, storage=st) as c:
        assert L.lbm_get_tuning(a.ctx, L.LBM_TUNE_CELL_PAIRS) == 1
        L.lbm_set_tuning(a.ctx, L.LBM_TUNE_STENCIL_STAGE, 0)
        L.lbm_set_tuning(d.ctx, L.LBM_TUNE_STENCIL_STAGE, 1)  # staged stencils, in place
        assert L.lbm_get_tuning(d.ctx, L.LBM_TUNE_STENCIL_STAGE) == 1
        L.lbm_set_tuning(b.ctx, L.LBM_TUNE_CELL_PAIRS, 0)
        L.lbm_set_tuning(b.ctx, L.LBM_TUNE_GRAPHS, 0)
        for n in (1, 2, 3, 4):
            for s in (a, b, c, d):
                s.step(n)
            _same(a, b)
            _same(a, c)
            _same(a, d)
        ra = L.lbm_step_reduce(a.ctx, 3)
        rb = L.lbm_step_reduce(b.ctx, 3)
        rc = L.lbm_step_reduce(c.ctx, 3)
        rd = L.lbm_step_reduce(d.ctx, 3)
        assert ra[0] == rb[0] == rc[0] == rd[0]
        for r in (rb, rc, rd):
            assert np.array_equal(ra[1], r[1])
        _same(a, c)
        _same(a, d)
