"""The sampled-cell oracle step agrees with the full-grid oracle step (CPU)."""
import numpy as np
import pytest

from oracle import lbm_oracle as O
from paper_1507_07294_gb300 import inputs as I
from tests.patch_oracle import one_step_at, sample_cells


@pytest.mark.parametrize("walls", [False, True])
def test_patch_step_equals_full_step(walls):
    if walls:
        w = I.perturbed(I.rayleigh_taylor(W=11, nz=14, Re=100.0), seed=5, u_amp=0.02, p_amp=1e-3)
        w.nx = 12
        w.phi0 = np.concatenate([w.phi0, w.phi0[:, :, :1]], axis=2)
        w.u0 = np.concatenate([w.u0, w.u0[..., :1]], axis=3)
        w.p0 = np.concatenate([w.p0, w.p0[..., :1]], axis=2)
    else:
        w = I.perturbed(I.droplet(n=10, R=3.0, nx=12, ny=11, nz=10), seed=6, u_amp=0.02, p_amp=1e-3)
    p = O.Params.from_workload(w)
    o = O.Oracle(p)
    o.init(w.phi0, w.u0, w.p0)
    o.step(3)
    f, g, phiu = o.f.copy(), o.g.copy(), o.phiu_prev.copy()
    cells = sample_cells(w.shape, 12, seed=1)
    pf, pg = one_step_at(p, f, g, phiu, True, cells, R=4)
    o.step(1)
    for k, (z, y, x) in enumerate(cells):
        np.testing.assert_allclose(pf[k], o.f[:, z, y, x], atol=1e-14)
        np.testing.assert_allclose(pg[k], o.g[:, z, y, x], atol=1e-14)


def test_patch_step_equals_full_step_in_tracking_mode():
    """The prescribed velocity is evaluated at the patch's global coordinates and time."""
    w = I.deformation(n=14, period=40.0)
    p = O.Params.from_workload(w)
    o = O.Oracle(p)
    o.init(w.phi0)
    o.step(7)
    f, g, phiu = o.f.copy(), o.g.copy(), o.phiu_prev.copy()
    cells = sample_cells(w.shape, 10, seed=2)
    pf, _ = one_step_at(p, f, g, phiu, True, cells, R=4, t=o.t)
    o.step(1)
    for k, (z, y, x) in enumerate(cells):
        np.testing.assert_allclose(pf[k], o.f[:, z, y, x], atol=1e-14)
