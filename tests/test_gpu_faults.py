"""Failures injected on the host (needs a GPU for the real allocations).

An allocator that refuses chosen requests stands in for running out of device memory:
every entry point that allocates must return LBM_ENOMEM, release what it had taken, and
leave an existing context usable.  Nothing here faults or stalls the GPU.
"""
import ctypes

import numpy as np
import pytest

from paper_1507_07294_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1507_07294_gb300 import lbm
    lbm.load_library()
    return lbm


class FlakyAllocator:
    """PyTorch's caching allocator behind a switch: refuses the request number
    `fail_at` (0-based) and, with `refuse_all`, every request; counts what is live."""

    def __init__(self, L, fail_at=None):
        import torch
        self.fail_at = fail_at
        self.refuse_all = False
        self.calls = 0
        self.live = set()

        def _alloc(nbytes, user):
            k = self.calls
            self.calls += 1
            if self.refuse_all or k == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes))
            self.live.add(p)
            return p

        def _free(ptr, user):
            self.live.discard(ptr)
            torch.cuda.caching_allocator_delete(ptr)

        self._a = L.ALLOC_FN(_alloc)
        self._f = L.FREE_FN(_free)
        self.struct = L.LbmAllocator(self._a, self._f, None)


def _create(L, w, alloc):
    grid, params = L.params_from_workload(w)
    out = ctypes.c_void_p()
    st = L.load_library().lbm_create(ctypes.byref(grid), ctypes.byref(params),
                                     ctypes.byref(alloc.struct), None, ctypes.byref(out))
    return st, out


def test_create_releases_everything_when_an_allocation_fails(L):
    w = I.droplet(n=12, R=3.0)
    probe = FlakyAllocator(L)
    st, h = _create(L, w, probe)
    assert st == L.LBM_OK
    total = probe.calls
    L.load_library().lbm_destroy(h)
    assert not probe.live
    for k in range(total):
        a = FlakyAllocator(L, fail_at=k)
        st, h = _create(L, w, a)
        assert st == L.LBM_ENOMEM and h.value is None, k
        assert not a.live, f"allocation {k}: {len(a.live)} buffers not released"
        assert "allocation" in L.lbm_last_error()


def test_refused_staging_leaves_the_context_usable(L):
    lib = L.load_library()
    w = I.perturbed(I.droplet(n=12, R=3.0), seed=31, u_amp=0.01)
    a = FlakyAllocator(L)
    st, h = _create(L, w, a)
    assert st == L.LBM_OK
    ctx = L.Context(h, w.cells, w.shape, a)
    live = len(a.live)
    a.refuse_all = True
    with pytest.raises(L.LbmError) as e:
        L.lbm_init_phi(ctx, w.phi0, w.u0)  # needs a staging buffer
    assert e.value.status == L.LBM_ENOMEM and len(a.live) == live
    a.refuse_all = False
    L.lbm_init_phi(ctx, w.phi0, w.u0)
    L.lbm_step(ctx, 3)
    a.refuse_all = True
    with pytest.raises(L.LbmError) as e:
        L.lbm_read_fields(ctx, L.LBM_FIELD_PHI)  # needs the widening buffer
    assert e.value.status == L.LBM_ENOMEM and len(a.live) == live
    sp, _ = L.lbm_reduce(ctx)  # allocates nothing
    a.refuse_all = False
    phi = L.lbm_read_fields(ctx, L.LBM_FIELD_PHI)["phi"]
    assert np.isfinite(phi).all() and abs(phi.sum() - sp) < 1e-3
    assert lib.lbm_destroy(h) == L.LBM_OK
    assert not a.live


def test_batch_create_reports_a_refused_table(L):
    lib = L.load_library()
    a = FlakyAllocator(L)
    a.refuse_all = True
    out = ctypes.c_void_p()
    assert lib.lbm_batch_create(ctypes.byref(a.struct), None, ctypes.byref(out)) == L.LBM_ENOMEM
    assert out.value is None and "batch table" in L.lbm_last_error()


def test_tma_wait_budget_runs_out_cleanly(L):
    """The TMA chemical-potential pass bounds its wait for each copy.  A budget of 0
    polls makes every block give up at once (it still lets its copy land before
    exiting): the next reduction reports LBM_ETIMEOUT, the report clears the flag, and
    the context keeps working."""
    w = I.perturbed(I.droplet(n=16, R=5.0, nx=64, ny=16, nz=24), seed=51, u_amp=0.01)
    with L.Solver(w) as s:
        L.lbm_set_tuning(s.ctx, L.LBM_TUNE_FUSED, 0)  # the three-kernel step uses the TMA pass
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_MU_TMA) == 1
        default = L.lbm_get_tuning(s.ctx, L.LBM_TUNE_TMA_WAIT_POLLS)
        assert default > 1000
        s.step(2)
        s.reduce()
        L.lbm_set_tuning(s.ctx, L.LBM_TUNE_TMA_WAIT_POLLS, 0)
        s.step(1)
        with pytest.raises(L.LbmError) as e:
            s.reduce()
        assert e.value.status == L.LBM_ETIMEOUT and "TMA" in str(e.value)
        s.reduce()  # reported once, then cleared
        s.step(1)
        with pytest.raises(L.LbmError) as e:
            L.lbm_step_reduce(s.ctx, 1)
        assert e.value.status == L.LBM_ETIMEOUT
        s.step(1)
        with pytest.raises(L.LbmError) as e:
            s.fields(L.LBM_FIELD_PHI)
        assert e.value.status == L.LBM_ETIMEOUT
        L.lbm_set_tuning(s.ctx, L.LBM_TUNE_TMA_WAIT_POLLS, default)
        s.step(3)
        sp, _ = s.reduce()
        assert np.isfinite(sp)
