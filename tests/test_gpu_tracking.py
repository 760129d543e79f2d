"""Interface-tracking mode on the GPU vs the FP64 oracle (needs a GPU).

Only the D3Q7 lattice evolves and the velocity is prescribed (Sec. III A, B: the
rotation of Eq. 37, the deformation flow of Eq. 41, and a uniform velocity).
Tolerance after 100 steps: max|phi_gpu - phi_oracle| <= 1e-5.
"""
import numpy as np
import pytest

from oracle import lbm_oracle as O
from paper_1507_07294_gb300 import diagnostics as Dg
from paper_1507_07294_gb300 import inputs as I
from tests.patch_oracle import one_step_at, sample_cells

pytestmark = pytest.mark.gpu

PHI_TOL = 1e-5


@pytest.fixture(scope="module")
def L():
    from paper_1507_07294_gb300 import lbm
    lbm.load_library()
    return lbm


def _oracle(w):
    o = O.Oracle(O.Params.from_workload(w))
    o.init(w.phi0, w.u0, w.p0)
    return o


def _tracking_cases():
    zal = I.zalesak(n=30)
    dfm = I.deformation(n=32, period=150.0)
    dfm.nx, dfm.ny, dfm.nz = 32, 30, 34  # ragged box (L = nx)
    x, y, z = I.node_coords(32, 30, 34, False)
    r = np.sqrt((x - 11.2) ** 2 + (y - 10.5) ** 2 + (z - 11.9) ** 2)
    dfm.phi0 = np.broadcast_to(np.tanh(2.0 * (4.8 - r) / 2.0), (34, 30, 32)).copy()
    slab = I.translating_slab(n=40)
    return {"rotation": zal, "deformation": dfm, "uniform": slab}


@pytest.mark.parametrize("pattern", ["ab", "aa"])
@pytest.mark.parametrize("case", ["rotation", "deformation", "uniform"])
def test_tracking_100_steps(L, case, pattern):
    w = _tracking_cases()[case]
    with L.Solver(w, pattern=pattern) as s:
        s.step(100)
        gf = s.fields()
        mass, mom = s.reduce()
    o = _oracle(w)
    o.step(100)
    of = o.fields()
    dphi = np.abs(gf["phi"] - of["phi"]).max()
    assert dphi <= PHI_TOL, f"max|dphi| = {dphi:.3e}"
    # the reported velocity is the prescribed field at the current step
    np.testing.assert_allclose(gf["u"], of["u"], atol=2e-8)
    assert np.all(gf["p"] == 0.0)
    assert np.all(mom == 0.0)
    assert abs(mass - w.phi0.sum()) <= 1e-6 * np.abs(w.phi0).sum()


def test_full_size_deformation_128_one_step(L):
    """The 128^3 deformation flow (R = 19.2 at 44.8, U = 0.02, T = 3000 steps,
    Pe = 400): one step at 200 sampled cells after 749 GPU steps (time factor
    cos(pi 749 / 3000))."""
    w = I.deformation(n=128, period=3000.0)
    p = O.Params.from_workload(w)
    with L.Solver(w) as s:
        s.step(749)
        f, g, phiu, t = s.state()
        s.step(1)
        f1, _, _, _ = s.state()
    cells = sample_cells(w.shape, 200, seed=21)
    of, _ = one_step_at(p, f, g, phiu, True, cells, t=t)
    idx = tuple(np.array(cells).T)
    gf = np.moveaxis(f1[(slice(None),) + idx], 0, 1)
    np.testing.assert_allclose(gf, of, atol=2e-6)


def test_deformation_128_returns_at_T(L):
    """Over one period of the time-reversed deformation flow the sphere deforms and
    comes back: the Err of Eq. 40 at T is far below its value at T/2, and mass is
    conserved."""
    w = I.deformation(n=128, period=3000.0)
    with L.Solver(w) as s:
        s.step(1500)
        err_half = Dg.relative_error(s.fields(L.LBM_FIELD_PHI)["phi"], w.phi0)
        s.step(1500)
        phi_T = s.fields(L.LBM_FIELD_PHI)["phi"]
        mass, _ = s.reduce()
    err_T = Dg.relative_error(phi_T, w.phi0)
    print(f"deformation 128^3: Err(T/2) = {err_half:.4e}, Err(T) = {err_T:.4e}")
    assert err_half > 0.02
    assert err_T < err_half / 20
    assert abs(mass - w.phi0.sum()) <= 1e-5 * np.abs(w.phi0).sum()


def test_set_velocity_rejects_bad_arguments(L):
    w = I.droplet(n=8, R=2.5)
    with L.Solver(w, init=False) as s:
        for kind, U, T in ((7, 0.02, 1.0), (L.LBM_VELOCITY_DEFORMATION, 0.02, 0.0)):
            with pytest.raises(L.LbmError) as e:
                L.lbm_set_velocity(s.ctx, kind, U, T)
            assert e.value.status == L.LBM_EINVAL
