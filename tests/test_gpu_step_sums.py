"""lbm_step_reduce: the sums of the new state computed inside the last step (needs a GPU).

The fused sums add up the post-collision values the step stores, with the momentum of
populations that bounce off a wall negated; they must agree with lbm_reduce's separate
pass over the new state (up to the FP32 rounding of the 32-cell warp sums) and with the
FP64 oracle's totals, and the step itself must store exactly what lbm_step stores.
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


def _walled():
    return I.perturbed(I.rayleigh_taylor(W=24, nz=40, Re=300.0), seed=21, u_amp=0.02, p_amp=1e-3)


def _periodic():
    return I.perturbed(I.droplet(n=16, R=5.0, nx=19, ny=17, nz=15), seed=22, u_amp=0.02, p_amp=1e-3)


def _tol(w):
    # a warp sum of 32 FP32 values of magnitude <= 1 rounds by at most ~5 x 2^-24 x 32
    return 1e-5 * (w.cells / 32 + 1)


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("case", ["walled", "periodic"])
def test_fused_sums_match_the_separate_reduction(L, case, pattern, storage):
    w = _walled() if case == "walled" else _periodic()
    with L.Solver(w, pattern=pattern, storage=storage) as s:
        s.step(2)
        for n in (1, 3):
            sp, mom = L.lbm_step_reduce(s.ctx, n)
            rp, rmom = s.reduce()
            assert abs(sp - rp) <= _tol(w), (sp, rp)
            np.testing.assert_allclose(mom, rmom, rtol=0, atol=_tol(w))


def test_fused_sums_match_the_oracle(L):
    w = _walled()
    o = O.Oracle(O.Params.from_workload(w))
    o.init(w.phi0, w.u0, w.p0)
    o.step(5)
    osp, omom = o.totals()
    with L.Solver(w) as s:
        s.step(4)
        sp, mom = L.lbm_step_reduce(s.ctx, 1)
    assert abs(sp - osp) <= 1e-4 * np.abs(w.phi0).sum() / w.cells * 10 + _tol(w)
    np.testing.assert_allclose(mom, omom, atol=1e-6 * w.cells * 1e-2 + _tol(w))


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_fused_step_stores_what_lbm_step_stores(L, pattern, storage):
    w = _walled()
    with L.Solver(w, pattern=pattern, storage=storage) as a, \
            L.Solver(w, pattern=pattern, storage=storage) as b:
        a.step(5)
        b.step(1)
        L.lbm_step_reduce(b.ctx, 2)
        L.lbm_step_reduce(b.ctx, 2)
        for x, y in zip(a.state()[:3], b.state()[:3]):
            assert np.array_equal(x, y)
        assert a.t == b.t == 5


def test_fallback_for_variants_and_tracking(L):
    wv = _periodic()
    wv.srt_flow = True
    with L.Solver(wv) as s:
        s.step(2)
        sp, mom = L.lbm_step_reduce(s.ctx, 2)
        rp, rmom = s.reduce()
    assert sp == rp and np.array_equal(mom, rmom)  # separate pass: identical
    wt = I.deformation(n=16, period=200.0)
    with L.Solver(wt) as s:
        sp, mom = L.lbm_step_reduce(s.ctx, 3)
        rp, rmom = s.reduce()
    assert sp == rp and np.array_equal(mom, rmom)


def test_async_matches_sync_and_nan_is_reported(L):
    import torch
    w = _periodic()
    with L.Solver(w) as a, L.Solver(w) as b:
        a.step(1)
        b.step(1)
        sp, mom = L.lbm_step_reduce(a.ctx, 2)
        buf = torch.zeros(5, dtype=torch.float64, device="cuda")
        L.lbm_step_reduce_async(b.ctx, 2, buf.data_ptr())
        torch.cuda.synchronize()
        got = buf.cpu().numpy()
        assert got[0] == sp and np.array_equal(got[1:4], mom) and got[4] == 0
        with pytest.raises(L.LbmError):
            L.lbm_step_reduce(a.ctx, 0)
    wn = I.droplet(n=8, R=2.5)
    wn.phi0 = wn.phi0.copy()
    wn.phi0[3, 4, 5] = np.nan
    with L.Solver(wn) as s:
        s.step(1)
        _, _, st = L.lbm_step_reduce(s.ctx, 1, check=False)
    assert st == L.LBM_EUNSTABLE


def test_sums_prefetch_distance_changes_speed_not_results(L):
    """LBM_TUNE_PREFETCH_COLLIDE_SUMS starts at the plain steps' distance and, set to
    another value (0: no prefetch), leaves the sums and the stored state bit for bit as
    they were."""
    w = _walled()
    with L.Solver(w) as a, L.Solver(w) as b:
        assert (L.lbm_get_tuning(a.ctx, L.LBM_TUNE_PREFETCH_COLLIDE_SUMS)
                == L.lbm_get_tuning(a.ctx, L.LBM_TUNE_PREFETCH_COLLIDE) > 0)
        L.lbm_set_tuning(b.ctx, L.LBM_TUNE_PREFETCH_COLLIDE_SUMS, 0)
        assert L.lbm_get_tuning(b.ctx, L.LBM_TUNE_PREFETCH_COLLIDE_SUMS) == 0
        for _ in range(3):
            ma, ja = L.lbm_step_reduce(a.ctx, 2)
            mb, jb = L.lbm_step_reduce(b.ctx, 2)
            assert ma == mb and np.array_equal(ja, jb)
        for x, y in zip(a.state()[:3], b.state()[:3]):
            assert np.array_equal(x, y)
