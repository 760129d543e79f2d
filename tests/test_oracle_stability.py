"""Linear stability of the interface lattice under a uniform flow, and the oracle's
agreement with it.

About a uniform phase (phi = 1) the D3Q7 scheme of Eqs. 4-19 is linear in the
perturbation: mu = 8 beta dphi - kappa lap dphi (Eq. 2 linearised, lap of Eq. 36), the
equilibrium moments of Eq. 17 and the source of Eq. 18 with the backward difference of
Eq. 34 are linear in phi, and propagation (Eq. 16) is a shift.  For one Fourier mode
exp(i k . x) a step is then an 8 x 8 matrix acting on the seven populations and the
previous step's phi.  This file builds that matrix from the printed M (Eq. 9) and the
formulas themselves -- no oracle code -- and checks two things:

* the oracle, run with a prescribed uniform velocity on a periodic box that holds the
  mode, grows or decays at the rate of the matrix's largest eigenvalue;
* the paper's coupled relaxation rates (Eq. 45, s_1 = 1.25) at the Rayleigh-Taylor
  parameters (sigma = 1e-4, D = 4, Mob = sqrt(gW) W / Pe = 0.0512 for W = 64) make this
  mode grow once |u| is a few hundredths, while equal rates of 1 keep it bounded, and a
  mobility two orders larger damps it.  This is the instability behind the divergence of
  the Rayleigh-Taylor runs documented with the readings of the paper.
"""
import numpy as np
import pytest

from oracle import lbm_oracle as O
from tests.golden_io import load

C7 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
              dtype=float)
C15 = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                [1, 1, 1], [-1, -1, -1], [1, 1, -1], [-1, -1, 1], [1, -1, 1], [-1, 1, -1],
                [1, -1, -1], [-1, 1, 1]], dtype=float)
W15 = np.array([1 / 9] * 6 + [1 / 72] * 8)
SF_COUPLED = (1.0, 1.25, 1.25, 1.25, 1.2, 1.0, 1.0)   # Eq. 45
SF_UNIT = (1.0,) * 7


def lap15_symbol(k):
    """Eq. 36 on the D3Q15 stencil for exp(i k.x): (2/c_s^2) sum w_i (cos k.c_i - 1)."""
    return 2.0 * 3.0 * float(np.sum(W15 * (np.cos(C15 @ k) - 1.0)))


def amplification(k, u, sf, mob, sigma, D, A=0.25):
    """One step of the linearised D3Q7 scheme for the mode exp(i k.x); state
    (f_0..f_6, phi of the previous step)."""
    M = load("d3q7_M.txt")
    Mi = np.linalg.inv(M)
    S = np.diag(sf)
    beta, kappa = 3 * sigma / (4 * D), 3 * D * sigma / 8
    eta = mob / (A * (1.0 / sf[1] - 0.5))
    dmu = 8 * beta - kappa * lap15_symbol(k)   # d mu / d phi about phi = 1
    G = np.zeros((8, 8), complex)
    for j in range(8):
        e = np.zeros(8, complex)
        e[j] = 1.0
        f, phi_prev = e[:7], e[7]
        phi = f.sum()
        mu = dmu * phi
        meq = np.array([phi, phi * u[0], phi * u[1], phi * u[2], 6 * phi - 21 * A * eta * mu, 0, 0])
        dt = u * (phi - phi_prev)
        mR = np.array([0, dt[0], dt[1], dt[2], 0, 0, 0])
        m = M @ f
        fp = Mi @ (m - S @ (m - meq) + (np.eye(7) - S / 2) @ mR)
        G[:7, j] = np.exp(-1j * (C7 @ k)) * fp
        G[7, j] = phi
    return G


def growth_per_step(k, u, sf, mob, sigma=1e-4, D=4.0):
    return float(np.abs(np.linalg.eigvals(amplification(np.asarray(k, float),
                                                        np.asarray(u, float), sf, mob,
                                                        sigma, D))).max())


def oracle_growth(n, U, sf, mob, steps0, steps1, sigma=1e-4, D=4.0, eps=1e-7):
    """Per-step growth of the k = 2 pi / n mode of phi along x in the oracle with the
    prescribed velocity (U, 0, 0) on an n x 1 x 1 periodic box, between two step counts."""
    p = O.Params(nx=n, ny=1, nz=1, walls_z=False, rho_l=3.0, rho_g=1.0, nu_l=0.1, nu_g=0.1,
                 mobility=mob, D=D, sigma=sigma, g=(0.0, 0.0, 0.0), sf=sf,
                 velocity=("uniform", U))
    o = O.Oracle(p)
    x = np.arange(n)
    o.init((1.0 + eps * np.cos(2 * np.pi * x / n)).reshape(1, 1, n))

    def amp():
        phi = O.order_parameter(o.f).reshape(n)
        return abs(np.sum((phi - 1.0) * np.exp(-2j * np.pi * x / n)))

    o.step(steps0)
    a0 = amp()
    o.step(steps1 - steps0)
    return (amp() / a0) ** (1.0 / (steps1 - steps0))


@pytest.mark.parametrize("sf, mob, U", [(SF_COUPLED, 0.0512, 0.04), (SF_UNIT, 0.0512, 0.04),
                                        (SF_COUPLED, 5.0, 0.04)])
def test_oracle_follows_the_linear_analysis(sf, mob, U):
    g = growth_per_step((2 * np.pi / 3, 0, 0), (U, 0, 0), sf, mob)
    # steps 100..600: past the start-up transient (the other eigenvalues are <= 0.25), and
    # the decaying case stays well above round-off (1e-7 x 0.987^600 ~ 4e-11)
    measured = oracle_growth(3, U, sf, mob, 100, 600)
    assert measured == pytest.approx(g, abs=1e-6)


def test_paper_rates_are_unstable_under_advection_at_the_rt_mobility():
    k = (2 * np.pi / 3, 0, 0)
    # coupled rates of Eq. 45 at the Rayleigh-Taylor mobility: grows, faster with |u|
    g2 = growth_per_step(k, (0.02, 0, 0), SF_COUPLED, 0.0512)
    g4 = growth_per_step(k, (0.04, 0, 0), SF_COUPLED, 0.0512)
    assert 1.0 < g2 < g4
    assert g4 - 1.0 > 5e-4  # e-folds within about 1000 steps (a t* = 1 at W = 64 is 1600)
    # at rest, or with all rates 1, or with a mobility 100 times larger: no growth
    assert growth_per_step(k, (0.0, 0, 0), SF_COUPLED, 0.0512) <= 1.0 + 1e-12
    assert growth_per_step(k, (0.04, 0, 0), SF_UNIT, 0.0512) <= 1.0 + 1e-6
    assert growth_per_step(k, (0.04, 0, 0), SF_COUPLED, 5.0) <= 1.0 + 1e-12
