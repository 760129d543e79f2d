"""Host diagnostics: Err of Eq. 40, interface crossings, Rayleigh-Taylor fronts."""
import numpy as np
import pytest

from paper_1507_07294_gb300 import diagnostics as Dg
from paper_1507_07294_gb300 import inputs as I


def test_relative_error_definition():
    phi0 = np.array([1.0, -1.0, 0.5, -0.5])
    assert Dg.relative_error(phi0, phi0) == 0.0
    assert Dg.relative_error(phi0 + 0.3, phi0) == pytest.approx(4 * 0.3 / 3.0)


def test_crossings_interpolate_linearly():
    z = np.arange(5) + 0.5
    prof = np.array([-1.0, -0.5, 0.5, 1.0, -1.0])
    np.testing.assert_allclose(Dg.interface_crossings(prof, z), [2.0, 4.0])
    # an off-centre crossing: -1 at z = 0.5, +3 at z = 1.5 -> zero at 0.75
    np.testing.assert_allclose(Dg.interface_crossings([-1.0, 3.0], [0.5, 1.5]), [0.75])


@pytest.mark.parametrize("W, nz", [(64, 256), (32, 128), (16, 40)])
def test_rt_fronts_of_the_initial_interface(W, nz):
    """Eq. 42-43: the interface sits at nz/2 + h, h(0, 0) = 0.1 W, h(W/2, W/2) = -0.1 W;
    linear interpolation of the tanh profile between nodes errs by far less than 1e-3 W."""
    w = I.rayleigh_taylor(W=W, Re=256.0, nz=nz)
    bubble, spike = Dg.rt_fronts(w.phi0, W)
    assert bubble == pytest.approx(0.1, abs=1e-3)
    assert spike == pytest.approx(-0.1, abs=1e-3)
