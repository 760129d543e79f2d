"""CUDA path vs FP64 oracle, through the C ABI (needs a GPU).

Tolerances (FP32 arithmetic and storage against FP64): after 100 steps
max|phi_gpu - phi_oracle| <= 1e-5 and max|u_gpu - u_oracle| / U <= 1e-4, U the
problem's velocity scale; one step from a common state agrees to a few FP32 ulps of
the population magnitudes.
"""
import numpy as np
import pytest

from oracle import lbm_oracle as O
from paper_1507_07294_gb300 import inputs as I
from tests.patch_oracle import one_step_at, sample_cells

pytestmark = pytest.mark.gpu

PHI_TOL = 1e-5
U_TOL_REL = 1e-4


@pytest.fixture(scope="module")
def L():
    from paper_1507_07294_gb300 import lbm
    lbm.load_library()
    return lbm


def _oracle(w):
    o = O.Oracle(O.Params.from_workload(w))
    o.init(w.phi0, w.u0, w.p0)
    return o


def _compare_fields(gf, of, U, phi_tol=PHI_TOL, u_tol=U_TOL_REL, p_tol=None):
    dphi = np.abs(gf["phi"] - of["phi"]).max()
    du = np.abs(gf["u"] - of["u"]).max() / U
    assert dphi <= phi_tol, f"max|dphi| = {dphi:.3e}"
    assert du <= u_tol, f"max|du|/U = {du:.3e}"
    if p_tol is not None:
        dp = np.abs(gf["p"] - of["p"]).max()
        assert dp <= p_tol, f"max|dp| = {dp:.3e}"
    np.testing.assert_allclose(gf["rho"], of["rho"], atol=1e-5)
    return dphi, du


def test_initial_fields(L):
    w = I.perturbed(I.droplet(n=16, R=5.0, nx=20, ny=18, nz=16), seed=1, u_amp=0.01, p_amp=1e-3)
    with L.Solver(w) as s:
        gf = s.fields()
    of = _oracle(w).fields()
    _compare_fields(gf, of, w.U, phi_tol=1e-6, u_tol=1e-5, p_tol=1e-7)
    np.testing.assert_allclose(gf["mu"], of["mu"], atol=1e-7)


@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_droplet_100_steps(L, pattern):
    """The static droplet (32^3, R = 8, D = 4, sigma = 0.01, rho 3:1, nu = 0.1,
    Mob = 0.1), seeded velocity and pressure noise so every term acts."""
    w = I.perturbed(I.droplet(n=32, R=8.0), seed=0, u_amp=0.005, p_amp=1e-4)
    with L.Solver(w, pattern=pattern) as s:
        s.step(100)
        gf = s.fields()
        assert s.t == 100
    o = _oracle(w)
    o.step(100)
    _compare_fields(gf, o.fields(), w.U, p_tol=1e-6)


@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_rayleigh_taylor_ragged_100_steps(L, pattern):
    """Walls in z, gravity, ragged sizes in all three directions (not multiples of a
    block or a warp)."""
    w = I.rayleigh_taylor(W=37, nz=70, Re=256.0)
    w.ny = 29
    w.phi0 = np.ascontiguousarray(w.phi0[:, :29, :])
    w = I.perturbed(w, seed=2, u_amp=0.01, p_amp=1e-4)
    with L.Solver(w, pattern=pattern) as s:
        s.step(100)
        gf = s.fields()
    o = _oracle(w)
    o.step(100)
    _compare_fields(gf, o.fields(), w.U, p_tol=1e-6)


def test_every_term_and_option(L):
    """Unequal relaxation rates in both lattices, unequal viscosities, gravity along
    all axes in the buoyancy form, A != 1/4: 40 steps."""
    w = I.perturbed(I.droplet(n=14, R=4.0, nx=17, ny=14, nz=13, nu=0.05), seed=3,
                    phi_amp=0.05, u_amp=0.01, p_amp=1e-3)
    w.nu_g = 0.2
    w.g = (2e-5, -1e-5, 3e-5)
    w.buoyancy = True
    w.A = 0.2
    w.sf = (1.1, 1.4, 1.4, 1.4, 1.3, 0.8, 1.6)
    w.sg = (1.0, 1.2, 0.9, 1.1, 1.3, 1.1, 1.3, 1.1, 1.3, 1.0, 1.0, 1.0, 1.0, 1.0, 1.5)
    with L.Solver(w) as s:
        s.step(40)
        gf = s.fields()
    o = _oracle(w)
    o.step(40)
    _compare_fields(gf, o.fields(), 0.01, p_tol=1e-6)


@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("shape,walls", [((1, 1, 1), False), ((1, 5, 7), False), ((3, 1, 4), True),
                                         ((1, 2, 3), True), ((5, 3, 2), False), ((9, 33, 1), True)])
def test_degenerate_grids(L, shape, walls, pattern):
    """Grids one cell thick in some direction, a single cell, walls one cell apart."""
    nz, ny, nx = shape
    w = I.droplet(n=4, R=1.5, nx=nx, ny=ny, nz=nz)
    w.walls_z = walls
    w = I.perturbed(w, seed=4, phi_amp=0.3, u_amp=0.01, p_amp=1e-3)
    w.g = (1e-5, 0.0, -2e-5)
    with L.Solver(w, pattern=pattern) as s:
        s.step(20)
        gf = s.fields()
    o = _oracle(w)
    o.step(20)
    _compare_fields(gf, o.fields(), 0.01)


@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("walls", [False, True])
def test_state_after_one_and_two_steps(L, walls, pattern):
    """Raw populations against the oracle after one (odd layout) and two (even layout)
    steps: within a few FP32 ulps of the population magnitudes."""
    if walls:
        w = I.perturbed(I.rayleigh_taylor(W=12, nz=20, Re=100.0), seed=5, u_amp=0.02, p_amp=1e-3)
    else:
        w = I.perturbed(I.droplet(n=12, R=4.0, nx=13, ny=12, nz=11), seed=5, u_amp=0.02, p_amp=1e-3)
    o = _oracle(w)
    with L.Solver(w, pattern=pattern) as s:
        for k in (1, 2):
            s.step(1)
            o.step(1)
            f, g, phiu, t = s.state()
            assert t == k
            np.testing.assert_allclose(f, o.f, atol=2e-6 * np.abs(o.f).max())
            np.testing.assert_allclose(g, o.g, atol=2e-6 * np.abs(o.g).max())
            np.testing.assert_allclose(phiu, o.phiu_prev, atol=1e-7)


def _sampled_one_step(L, w, warm_steps, n_samples, seed, pattern="ab"):
    """Run warm_steps on the GPU, take its state, advance one more step on the GPU and,
    at sampled cells, with the oracle from the same state."""
    p = O.Params.from_workload(w)
    with L.Solver(w, pattern=pattern) as s:
        s.step(warm_steps)
        f, g, phiu, _ = s.state()
        s.step(1)
        f1, g1, _, _ = s.state()
    cells = sample_cells(w.shape, n_samples, seed=seed)
    of, og = one_step_at(p, f, g, phiu, warm_steps > 0, cells)
    idx = tuple(np.array(cells).T)
    gf = np.moveaxis(f1[(slice(None),) + idx], 0, 1)
    gg = np.moveaxis(g1[(slice(None),) + idx], 0, 1)
    np.testing.assert_allclose(gf, of, atol=2e-6 * max(1.0, np.abs(of).max()))
    np.testing.assert_allclose(gg, og, atol=2e-6 * np.abs(og).max() + 1e-9)


@pytest.mark.parametrize("pattern", ["ab", "aa"])
def test_full_size_rayleigh_taylor_64(L, pattern):
    """Coupled Rayleigh-Taylor at its full size (64 x 64 x 256, Re = 256, At = 0.5):
    one step at 200 sampled cells (plus the box corners) after 99 GPU steps."""
    w = I.rayleigh_taylor(W=64, Re=256.0)
    _sampled_one_step(L, w, 99, 200, seed=7, pattern=pattern)


def test_full_size_rayleigh_taylor_256(L):
    """Rayleigh-Taylor at Re = 4000 on 256 x 256 x 1024 (67M cells), the benchmarked
    configuration: one step at 100 sampled cells after 9 GPU steps."""
    w = I.rayleigh_taylor(W=256, Re=4000.0)
    _sampled_one_step(L, w, 9, 100, seed=8)


def test_mass_conservation(L):
    """sum phi (FP64 device reduction) drifts only by FP32 rounding over 500 steps."""
    w = I.perturbed(I.rayleigh_taylor(W=32, nz=96, Re=256.0), seed=9, u_amp=0.01)
    with L.Solver(w) as s:
        s0, _ = s.reduce()
        s.step(500)
        s1, _ = s.reduce()
    assert abs(s1 - s0) <= 1e-6 * np.abs(w.phi0).sum()


def test_reduce_matches_oracle(L):
    w = I.perturbed(I.droplet(n=16, R=5.0, nx=19, ny=16, nz=15), seed=10, u_amp=0.01, p_amp=1e-3)
    o = _oracle(w)
    with L.Solver(w) as s:
        s.step(7)
        sp, mom = s.reduce()
    o.step(7)
    osp, omom = o.totals()
    assert abs(sp - osp) <= 1e-5 * np.abs(w.phi0).sum() / w.cells * 10 + 1e-4
    np.testing.assert_allclose(mom, omom, atol=1e-6 * w.cells * 1e-2)


@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("k", [3, 4])
def test_resume_is_bit_exact(L, k, pattern):
    """Read the state after k steps (odd and even step counts), continue 5 steps; a
    fresh context resumed from that state gives the same populations bit for bit, also
    when it resumes with the other storage pattern."""
    w = I.perturbed(I.rayleigh_taylor(W=16, nz=24, Re=100.0), seed=11, u_amp=0.01, p_amp=1e-3)
    with L.Solver(w, pattern=pattern) as a:
        a.step(k)
        st = a.state()
        a.step(5)
        ref = a.state()
    other = "aa" if pattern == "ab" else "ab"
    with L.Solver(w, init=False, pattern=other) as b:
        b.set_state(st[0], st[1], st[2], st[3])
        assert b.t == k
        b.step(5)
        got = b.state()
    for x, y in zip(ref[:3], got[:3]):
        assert np.array_equal(x, y)
    assert ref[3] == got[3] == k + 5


def test_zero_steps_changes_nothing(L):
    w = I.droplet(n=8, R=2.5)
    with L.Solver(w) as s:
        before = s.state()
        s.step(0)
        after = s.state()
    for x, y in zip(before[:3], after[:3]):
        assert np.array_equal(x, y)


def test_non_finite_state_is_reported(L):
    """A NaN in the initial condition surfaces as LBM_EUNSTABLE from lbm_reduce."""
    w = I.droplet(n=8, R=2.5)
    w.phi0 = w.phi0.copy()
    w.phi0[3, 4, 5] = np.nan
    with L.Solver(w) as s:
        s.step(2)
        _, _, st = L.lbm_reduce(s.ctx, check=False)
    assert st == L.LBM_EUNSTABLE


def test_step_before_init_is_rejected(L):
    w = I.droplet(n=8, R=2.5)
    with L.Solver(w, init=False) as s:
        with pytest.raises(L.LbmError) as e:
            s.step(1)
        assert e.value.status == L.LBM_EINVAL


def test_profile_counts_launches(L):
    w = I.droplet(n=16, R=5.0)
    with L.Solver(w) as s:
        L.lbm_profile(s.ctx, True)
        s.step(6)
        for k in range(3):
            ms, n = L.lbm_profile_read(s.ctx, k)
            assert n == 6 and ms > 0
        L.lbm_profile(s.ctx, False)


def test_patterns_agree_bit_for_bit(L):
    """The two-array and the in-place storage patterns run the same arithmetic: after
    any number of steps their states are identical."""
    w = I.perturbed(I.rayleigh_taylor(W=20, nz=36, Re=200.0), seed=12, phi_amp=0.02,
                    u_amp=0.01, p_amp=1e-3)
    with L.Solver(w, pattern="ab") as a, L.Solver(w, pattern="aa") as b:
        for n in (1, 2, 5):
            a.step(n)
            b.step(n)
            sa, sb = a.state(), b.state()
            for x, y in zip(sa[:3], sb[:3]):
                assert np.array_equal(x, y)


@pytest.mark.parametrize("variant", ["srt_flow", "d3q7_stencil", "both"])
def test_comparison_variants_100_steps(L, variant):
    """The paper's comparison variants as flags: SRT flow lattice, D3Q7-weighted
    difference schemes; walls and gravity on, 100 steps."""
    w = I.perturbed(I.rayleigh_taylor(W=20, nz=40, Re=150.0), seed=17, u_amp=0.01, p_amp=1e-4)
    w.srt_flow = variant in ("srt_flow", "both")
    w.stencil = "d3q7" if variant in ("d3q7_stencil", "both") else "d3q15"
    with L.Solver(w) as s:
        s.step(100)
        gf = s.fields()
    o = _oracle(w)
    o.step(100)
    _compare_fields(gf, o.fields(), w.U, p_tol=1e-6)


def test_autotune_changes_speed_not_results(L):
    """Autotuning sets only prefetch distances: a tuned run and an untuned run advanced
    by the same number of steps hold identical states."""
    from paper_1507_07294_gb300 import tune
    w = I.perturbed(I.rayleigh_taylor(W=32, nz=64, Re=200.0), seed=18, u_amp=0.01)
    with L.Solver(w) as a:
        chosen = tune.autotune(a.ctx, steps=2, warm=1)
        n = a.t
        sa = a.state()
    assert n == tune.tuning_steps(steps=2, warm=1)
    for name, d in chosen.items():
        assert d["value"] in [int(k) for k in d["ms"]]
    with L.Solver(w) as b:
        b.step(n)
        sb = b.state()
    for x, y in zip(sa[:3], sb[:3]):
        assert np.array_equal(x, y)


def test_read_fields_into_given_buffers(L):
    """Preallocated (here page-locked) output arrays receive the same values."""
    import torch
    w = I.perturbed(I.droplet(n=12, R=4.0, nx=13), seed=23, u_amp=0.01, p_amp=1e-3)
    with L.Solver(w) as s:
        s.step(3)
        ref = s.fields()
        bufs = {"phi": torch.empty(w.cells, dtype=torch.float64, pin_memory=True).numpy(),
                "u": np.empty((3,) + w.shape)}
        got = L.lbm_read_fields(s.ctx, L.LBM_FIELD_PHI | L.LBM_FIELD_U | L.LBM_FIELD_MU, out=bufs)
        with pytest.raises(ValueError):
            L.lbm_read_fields(s.ctx, L.LBM_FIELD_PHI, out={"phi": np.empty(3)})
    assert np.shares_memory(got["phi"], bufs["phi"]) and np.shares_memory(got["u"], bufs["u"])
    for k in ("phi", "u", "mu"):
        assert np.array_equal(got[k], ref[k])


def test_page_locked_host_buffers_give_the_same_values(L):
    """Page-locked host buffers are read (initial phi, u, p) and written (every field)
    by the library's kernels directly; pageable ones go through device staging and
    copies.  Both give the same state and the same fields, also when page-locked and
    pageable buffers are mixed in one call."""
    import torch
    w = I.perturbed(I.droplet(n=12, R=4.0, nx=13), seed=24, u_amp=0.01, p_amp=1e-3)

    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True).numpy()
        t[...] = a
        return t

    mask = L.LBM_FIELD_ALL
    with L.Solver(w) as a, L.Solver(w, init=False) as b, L.Solver(w, init=False) as c:
        L.lbm_init_phi(b.ctx, pinned(w.phi0), pinned(w.u0), pinned(w.p0))
        L.lbm_init_phi(c.ctx, pinned(w.phi0), w.u0, pinned(w.p0))
        for s in (a, b, c):
            s.step(3)
        sa, sb, sc = a.state(), b.state(), c.state()
        for x, y, z in zip(sa[:3], sb[:3], sc[:3]):
            assert np.array_equal(x, y) and np.array_equal(x, z)
        ref = a.fields(mask)
        out = {k: pinned(np.zeros_like(v)) for k, v in ref.items()}
        got = L.lbm_read_fields(b.ctx, mask, out=out)
        mixed = {"phi": pinned(np.zeros_like(ref["phi"])), "u": np.zeros_like(ref["u"])}
        got2 = L.lbm_read_fields(c.ctx, L.LBM_FIELD_PHI | L.LBM_FIELD_U, out=mixed)
    for k in ref:
        assert np.shares_memory(got[k], out[k])
        assert np.array_equal(got[k], ref[k]), k
    for k in ("phi", "u"):
        assert np.array_equal(got2[k], ref[k]), k
    # the state read into page-locked arrays
    import ctypes
    with L.Solver(w) as d:
        d.step(3)
        want = d.state()
        bufs = [torch.zeros((q,) + w.shape, dtype=torch.float32, pin_memory=True).numpy()
                for q in (7, 15, 3)]
        step = ctypes.c_longlong()
        lib = L.load_library()
        assert lib.lbm_read_state(d.ctx.handle, *(b.ctypes.data_as(ctypes.c_void_p) for b in bufs),
                                  ctypes.byref(step)) == L.LBM_OK
    assert step.value == want[3] == 3
    for x, y in zip(bufs, want[:3]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("shape, walls", [((64, 16, 24), False), ((64, 16, 18), True),
                                          ((96, 24, 40), True), ((64, 64, 64), False)])
def test_tma_halo_path_matches_plain_loads(L, shape, walls):
    """The chemical-potential pass with TMA-fetched halo bricks (grids whose x and y are
    whole bricks) gives bit-identical states to the plain-load pass, on periodic and
    walled grids and with a partial last brick in z."""
    nx, ny, nz = shape
    if walls:
        w = I.rayleigh_taylor(W=nx, nz=nz, Re=300.0)
        w.ny = ny
        w.phi0 = np.ascontiguousarray(w.phi0[:, :ny, :])
    else:
        w = I.droplet(n=nx, R=min(nx, ny, nz) / 3, nx=nx, ny=ny, nz=nz)
    w = I.perturbed(w, seed=41, u_amp=0.01, p_amp=1e-3)
    with L.Solver(w) as a, L.Solver(w) as b:
        for s in (a, b):  # the three-kernel step (the single-pass one has no mu pass)
            L.lbm_set_tuning(s.ctx, L.LBM_TUNE_FUSED, 0)
        assert L.lbm_get_tuning(a.ctx, L.LBM_TUNE_MU_TMA) == 1
        L.lbm_set_tuning(b.ctx, L.LBM_TUNE_MU_TMA, 0)
        assert L.lbm_get_tuning(b.ctx, L.LBM_TUNE_MU_TMA) == 0
        a.step(7)
        b.step(7)
        for x, y in zip(a.state()[:3], b.state()[:3]):
            assert np.array_equal(x, y)
        fa, fb = a.fields(L.LBM_FIELD_MU), b.fields(L.LBM_FIELD_MU)
        assert np.array_equal(fa["mu"], fb["mu"])


def test_tma_halo_path_100_steps_against_the_oracle(L):
    w = I.perturbed(I.rayleigh_taylor(W=64, nz=40, Re=256.0), seed=42, u_amp=0.01, p_amp=1e-4)
    w.ny = 16
    w.phi0 = np.ascontiguousarray(w.phi0[:, :16, :])
    w.u0 = np.ascontiguousarray(w.u0[:, :, :16, :])
    w.p0 = np.ascontiguousarray(w.p0[:, :16, :])
    with L.Solver(w) as s:
        L.lbm_set_tuning(s.ctx, L.LBM_TUNE_FUSED, 0)
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_MU_TMA) == 1
        s.step(100)
        gf = s.fields()
    o = _oracle(w)
    o.step(100)
    _compare_fields(gf, o.fields(), w.U, p_tol=1e-6)


def test_tma_halo_path_only_where_it_applies(L):
    for shape in ((37, 16, 24), (64, 12, 24), (32, 16, 24), (64, 16, 17)):
        w = I.droplet(n=16, R=4.0, nx=shape[0], ny=shape[1], nz=shape[2])
        with L.Solver(w) as s:
            assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_MU_TMA) == 0, shape
    with L.Solver(I.droplet(n=16, R=4.0, nx=64, ny=16, nz=18)) as s:
        with pytest.raises(L.LbmError):
            L.lbm_set_tuning(s.ctx, L.LBM_TUNE_MU_TMA, 2)


@pytest.mark.parametrize("pattern, storage", [("ab", "fp32"), ("aa", "fp32"), ("ab", "fp16"),
                                              ("aa", "bf16")])
def test_graph_replay_matches_plain_launches(L, pattern, storage):
    """lbm_step replays pairs of steps from captured CUDA graphs; the populations must
    be those of plain launches bit for bit, across odd step counts, a tuning change
    (which drops the graphs), a checkpoint restore and lbm_step_reduce."""
    w = I.perturbed(I.rayleigh_taylor(W=64, nz=40, Re=300.0), seed=43, u_amp=0.01, p_amp=1e-3)
    with L.Solver(w, pattern=pattern, storage=storage) as a, \
            L.Solver(w, pattern=pattern, storage=storage) as b:
        L.lbm_set_tuning(b.ctx, L.LBM_TUNE_GRAPHS, 0)
        assert L.lbm_get_tuning(a.ctx, L.LBM_TUNE_GRAPHS) == 1
        assert L.lbm_get_tuning(b.ctx, L.LBM_TUNE_GRAPHS) == 0
        for s in (a, b):
            s.step(5)
            s.step(4)
        L.lbm_set_tuning(a.ctx, L.LBM_TUNE_PREFETCH_COLLIDE, 100)
        L.lbm_set_tuning(b.ctx, L.LBM_TUNE_PREFETCH_COLLIDE, 100)
        for s in (a, b):
            s.step(3)
            L.lbm_step_reduce(s.ctx, 4)
        assert a.t == b.t == 16
        sa, sb = a.state(), b.state()
        for x, y in zip(sa[:3], sb[:3]):
            assert np.array_equal(x, y)
        a.set_state(*sa)  # resume from the checkpoint, then replay again
        b.set_state(*sb)
        a.step(6)
        b.step(6)
        for x, y in zip(a.state()[:3], b.state()[:3]):
            assert np.array_equal(x, y)


ROW_GRIDS = [  # (nx, ny, nz, walls): one and several tiles per row, planes not a multiple
    (32, 1, 1, False),  # of the order-parameter pass's column, walls on both sides of
    (32, 3, 5, True),   # a single plane's neighbours, ny = 1 and ny odd
    (64, 1, 2, True),
    (64, 8, 9, False),
    (96, 5, 7, True),
    (64, 16, 24, False),
]


@pytest.mark.parametrize("pattern, storage", [("ab", "fp32"), ("ab", "fp16"), ("ab", "bf16"),
                                              ("aa", "fp32"), ("aa", "fp16")])
@pytest.mark.parametrize("grid", ROW_GRIDS, ids=lambda g: "x".join(map(str, g[:3])) + ("w" if g[3] else "p"))
def test_row_addressing_matches_per_cell(L, grid, pattern, storage):
    """The whole-row addressing (order-parameter column kernel and row-delta loads of
    the two-array pattern; row-delta loads and stores of the odd in-place steps) must
    give the per-cell addressing's state bit for bit."""
    import dataclasses
    nx, ny, nz, walls = grid
    w = I.droplet(n=16, R=min(nx, ny, nz) / 3 + 0.5, nx=nx, ny=ny, nz=nz)
    if walls:
        w = dataclasses.replace(w, walls_z=True, g=(0.0, 0.0, -1e-5))
    w = I.perturbed(w, seed=61, u_amp=0.01, p_amp=1e-3)
    with L.Solver(w, pattern=pattern, storage=storage) as a, \
            L.Solver(w, pattern=pattern, storage=storage) as b:
        assert L.lbm_get_tuning(a.ctx, L.LBM_TUNE_ROWS) == 1
        L.lbm_set_tuning(b.ctx, L.LBM_TUNE_ROWS, 0)
        assert L.lbm_get_tuning(b.ctx, L.LBM_TUNE_ROWS) == 0
        for s in (a, b):
            s.step(7)
            L.lbm_step_reduce(s.ctx, 2)
        for x, y in zip(a.state()[:3], b.state()[:3]):
            assert np.array_equal(x, y)
        fa, fb = a.fields(), b.fields()
        assert np.array_equal(fa["phi"], fb["phi"])


def test_row_addressing_applicability(L):
    w = I.droplet(n=16, R=4.0, nx=48, ny=8, nz=8)
    with L.Solver(w) as s:
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_ROWS) == 0  # rows are not whole tiles
    w = I.droplet(n=16, R=4.0, nx=32, ny=8, nz=8)
    with L.Solver(w, pattern="aa") as s:
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_ROWS) == 1  # the odd in-place steps
    with L.Solver(w) as s:
        assert L.lbm_get_tuning(s.ctx, L.LBM_TUNE_ROWS) == 1
        with pytest.raises(L.LbmError):
            L.lbm_set_tuning(s.ctx, L.LBM_TUNE_ROWS, 2)


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("walls", [True, False])
def test_state_at_listed_cells_matches_the_full_read(L, storage, pattern, walls):
    """lbm_read_state_at returns, at listed cells (repeats, corners, wall planes, both
    index forms), exactly what lbm_read_state returns there: before the first step
    (phi u all zero), after an odd and after an even number of steps, for either
    pattern and every storage type; cells outside the grid are refused."""
    from dataclasses import replace
    w = I.perturbed(replace(I.droplet(n=10, R=3.5, nx=64, ny=10, nz=9), walls_z=walls),
                    seed=4, u_amp=0.01, p_amp=1e-3)
    rng = np.random.default_rng(5)
    n = w.cells
    lin = np.concatenate([rng.integers(0, n, 300), [0, n - 1, n - 1, 63, 64, n - 64],
                          rng.integers(0, n, 5)]).astype(np.int64)
    zyx = np.array(sample_cells(w.shape, 40, seed=6))
    with L.Solver(w, storage=storage, pattern=pattern) as s:
        for steps in (0, 3, 2):
            s.step(steps)
            f, g, phiu, t = s.state()
            for cells in (lin, zyx):
                fa, ga, pa, ta = s.state_at(cells)
                if cells.ndim == 2:
                    z, y, x = cells.T
                else:
                    z, r = np.divmod(cells, w.nx * w.ny)
                    y, x = np.divmod(r, w.nx)
                assert ta == t
                assert np.array_equal(fa, f[:, z, y, x])
                assert np.array_equal(ga, g[:, z, y, x])
                assert np.array_equal(pa, phiu[:, z, y, x])
            if steps == 0:
                assert not phiu.any()
        fa, ga, pa, _ = s.state_at(np.zeros(0, np.int64))
        assert fa.shape == (7, 0) and ga.shape == (15, 0) and pa.shape == (3, 0)
        for bad in ([n], [-1], [0, n + 5]):
            with pytest.raises(L.LbmError) as e:
                s.state_at(np.array(bad, np.int64))
            assert e.value.status == L.LBM_EINVAL
