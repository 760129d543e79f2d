"""The single-pass step kernel (LBM_TUNE_FUSED) against the three-kernel step (needs a
GPU).

Both compute every value with the same per-cell code in the same order, so their states
agree bit for bit: on walled and periodic grids, for every storage type, for any segment
length (including ones that leave a short last segment and segments of one plane), any
prefetch distance, with the fused step sums, with CUDA-graph replays, and when batched
(three-kernel) steps are interleaved with single-pass ones.  It also meets the FP64
oracle at the coupled tolerances after 100 steps on its own.
"""
import numpy as np
import pytest

from oracle import lbm_oracle as O
from paper_1507_07294_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1507_07294_gb300 import lbm
    lbm.load_library()
    return lbm


def _rt(W, ny, nz, seed=3):
    w = I.perturbed(I.rayleigh_taylor(W=W, nz=nz, Re=300.0), seed=seed, phi_amp=0.03,
                    u_amp=0.01, p_amp=1e-3)
    if ny != W:
        w.ny = ny
        w.phi0 = np.ascontiguousarray(w.phi0[:, :ny, :])
        w.u0 = np.ascontiguousarray(w.u0[:, :, :ny, :])
        w.p0 = np.ascontiguousarray(w.p0[:, :ny, :])
    return w


def _periodic(nx, ny, nz, seed=4):
    w = I.perturbed(I.droplet(n=max(nx, ny, nz), R=5.0, nx=nx, ny=ny, nz=nz), seed=seed,
                    phi_amp=0.02, u_amp=0.01, p_amp=1e-3)
    return w


def _same_state(a, b):
    sa, sb = a.state(), b.state()
    for x, y, name in zip(sa[:3], sb[:3], ("f", "g", "phiu")):
        assert np.array_equal(x, y), f"{name} differs: max {np.abs(x - y).max()}"
    assert sa[3] == sb[3]


def _pair(L, w, storage="fp32", seg=0, pf=None):
    st = L.STORAGES[storage]
    a = L.Solver(w, storage=st)
    b = L.Solver(w, storage=st)
    L.lbm_set_tuning(a.ctx, L.LBM_TUNE_FUSED, 1)
    L.lbm_set_tuning(b.ctx, L.LBM_TUNE_FUSED, 0)
    if seg:
        L.lbm_set_tuning(a.ctx, L.LBM_TUNE_FUSED_SEGMENT, seg)
    if pf is not None:
        L.lbm_set_tuning(a.ctx, L.LBM_TUNE_FUSED_PREFETCH, pf)
    assert L.lbm_get_tuning(a.ctx, L.LBM_TUNE_FUSED) == 1
    assert L.lbm_get_tuning(b.ctx, L.LBM_TUNE_FUSED) == 0
    return a, b


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("case", ["walls", "periodic"])
def test_single_pass_equals_three_kernels(L, storage, case):
    w = _rt(32, 16, 44) if case == "walls" else _periodic(64, 24, 20)
    a, b = _pair(L, w, storage, seg=5)
    try:
        for n in (1, 1, 3, 6):
            a.step(n)
            b.step(n)
            _same_state(a, b)
        fa, fb = a.fields(), b.fields()
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), k
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("seg", [1, 2, 3, 7, 16, 40])
def test_any_segment_length(L, seg):
    """Segments of 1..40 planes on 40 walled planes (40 = one segment, 7 leaves a
    short last one)."""
    w = _rt(32, 8, 40, seed=5)
    a, b = _pair(L, w, "fp32", seg=seg)
    try:
        a.step(4)
        b.step(4)
        _same_state(a, b)
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("shape", [(32, 8, 1), (32, 8, 2), (32, 8, 3), (64, 8, 5)])
def test_thin_periodic_grids(L, shape):
    """z periodic with 1 to 5 planes: the halo planes are images of the own ones."""
    nx, ny, nz = shape
    w = _periodic(nx, ny, nz, seed=6)
    a, b = _pair(L, w, "fp32", seg=2)
    try:
        a.step(3)
        b.step(3)
        _same_state(a, b)
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("nz", [1, 2, 3])
def test_thin_walled_grids(L, nz):
    w = _rt(32, 8, 8, seed=7)
    w.nz = nz
    w.phi0 = np.ascontiguousarray(w.phi0[:nz])
    w.u0 = np.ascontiguousarray(w.u0[:, :nz])
    w.p0 = np.ascontiguousarray(w.p0[:nz])
    a, b = _pair(L, w, "fp32")
    try:
        a.step(3)
        b.step(3)
        _same_state(a, b)
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("pf", [0, 1, 5])
def test_prefetch_distance_does_not_change_results(L, pf):
    w = _rt(64, 16, 24, seed=8)
    a, b = _pair(L, w, "fp16", seg=8, pf=pf)
    try:
        a.step(3)
        b.step(3)
        _same_state(a, b)
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_step_sums_are_identical(L, storage):
    w = _rt(32, 16, 30, seed=9)
    a, b = _pair(L, w, storage, seg=4)
    try:
        for n in (1, 2, 3):
            ra = L.lbm_step_reduce(a.ctx, n)
            rb = L.lbm_step_reduce(b.ctx, n)
            assert ra[0] == rb[0]
            assert np.array_equal(ra[1], rb[1])
        _same_state(a, b)
    finally:
        a.close()
        b.close()


def test_graph_replays_equal_plain_launches(L):
    w = _rt(32, 16, 36, seed=10)
    st = L.STORAGES["fp16"]
    with L.Solver(w, storage=st) as a, L.Solver(w, storage=st) as b:
        for s in (a, b):
            L.lbm_set_tuning(s.ctx, L.LBM_TUNE_FUSED, 1)
        L.lbm_set_tuning(b.ctx, L.LBM_TUNE_GRAPHS, 0)
        for n in (1, 4, 3, 6):  # odd counts change which phi array is current
            a.step(n)
            b.step(n)
        _same_state(a, b)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_batched_steps_between_single_pass_steps(L, storage):
    """Single-pass steps, batched (three-kernel) steps, single-pass again: the same
    state as three-kernel steps throughout (with 16-bit storage the current phi array
    alternates under the single-pass steps only)."""
    w = _rt(32, 16, 28, seed=11)
    a, b = _pair(L, w, storage, seg=6)
    try:
        with L.Batch() as batch:
            a.step(3)
            b.step(3)
            batch.step([a.ctx], 2)
            batch.step([b.ctx], 2)
            a.step(5)
            b.step(5)
            batch.step([a.ctx], 1)
            batch.step([b.ctx], 1)
            a.step(2)
            b.step(2)
        _same_state(a, b)
    finally:
        a.close()
        b.close()


def test_tuning_reports_where_it_applies(L):
    with L.Solver(I.droplet(n=16, R=5.0)) as s:  # nx not a multiple of 32
        L.lbm_set_tuning(s.ctx, L.LBM_TUNE_FUSED, 1)
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_FUSED) == 0
    w = _rt(32, 8, 16)
    with L.Solver(w, pattern=L.LBM_PATTERN_AA) as s:
        L.lbm_set_tuning(s.ctx, L.LBM_TUNE_FUSED, 1)
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_FUSED) == 0
    with L.Solver(w) as s:
        L.lbm_set_tuning(s.ctx, L.LBM_TUNE_FUSED, 1)
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_FUSED) == 1
        assert 1 <= L.lbm_get_tuning(s.ctx, L.LBM_TUNE_FUSED_SEGMENT) <= 16
        L.lbm_set_tuning(s.ctx, L.LBM_TUNE_ROWS, 0)
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_FUSED) == 0
        with pytest.raises(L.LbmError):
            L.lbm_set_tuning(s.ctx, L.LBM_TUNE_FUSED, 2)
        with pytest.raises(L.LbmError):
            L.lbm_set_tuning(s.ctx, L.LBM_TUNE_FUSED_PREFETCH, 65)


@pytest.mark.parametrize("case", ["droplet", "rt"])
def test_single_pass_against_the_oracle(L, case):
    """100 single-pass steps against the FP64 oracle: max|dphi| <= 1e-5 and
    max|du|/U <= 1e-4 (the 32^3 droplet of the parity tests; a walled Rayleigh-Taylor
    crop with short segments)."""
    if case == "droplet":
        w = I.perturbed(I.droplet(n=32, R=8.0), seed=0, u_amp=0.005, p_amp=1e-4)
    else:
        w = _rt(32, 16, 40, seed=12)
    with L.Solver(w) as s:
        L.lbm_set_tuning(s.ctx, L.LBM_TUNE_FUSED, 1)
        L.lbm_set_tuning(s.ctx, L.LBM_TUNE_FUSED_SEGMENT, 8)
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_FUSED) == 1
        s.step(100)
        gf = s.fields()
    o = O.Oracle(O.Params.from_workload(w))
    o.init(w.phi0, w.u0, w.p0)
    o.step(100)
    of = o.fields()
    assert np.abs(gf["phi"] - of["phi"]).max() <= 1e-5
    assert np.abs(gf["u"] - of["u"]).max() / w.U <= 1e-4
