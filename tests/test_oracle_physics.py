"""Physics pins of the full oracle time step.

Each test runs the coupled scheme on a small seeded or analytic case and checks a
result the paper or the continuum equations fix independently of the code: exact
invariants (mass, momentum budget), analytic equilibria (flat interface, hydrostatic
column, Laplace's law) and the two transport coefficients the Chapman-Enskog analyses
give (nu of Eq. 33 from a decaying shear wave, Mob of Eq. 19 from a decaying
order-parameter wave).
"""
import numpy as np
import pytest

from oracle import lbm_oracle as O
from paper_1507_07294_gb300 import inputs as I


def _oracle(w):
    o = O.Oracle(O.Params.from_workload(w))
    o.init(w.phi0, w.u0, w.p0)
    return o


def test_init_reproduces_the_initial_fields():
    """With uniform phi (no force), the equilibrium populations give back phi0, u0, p0."""
    w = I.perturbed(I.flat_interface(nz=6, nxy=5), seed=3, u_amp=0.02, p_amp=1e-3)
    w.phi0 = np.full(w.shape, 0.3)
    o = _oracle(w)
    fl = o.fields()
    np.testing.assert_allclose(fl["phi"], 0.3, atol=1e-15)
    np.testing.assert_allclose(fl["u"], w.u0, atol=1e-15)
    np.testing.assert_allclose(fl["p"], w.p0, atol=1e-15)


@pytest.mark.parametrize("walls", [False, True])
def test_mass_is_conserved_to_round_off(walls):
    """sum phi is invariant: m_0 is conserved by the collision (Eqs. 17-18) and
    propagation, with or without bounce-back walls, permutes populations."""
    if walls:
        w = I.perturbed(I.rayleigh_taylor(W=8, nz=24, Re=50.0), seed=1, u_amp=0.01, p_amp=1e-3)
    else:
        w = I.perturbed(I.droplet(n=12, R=3.5), seed=1, u_amp=0.01, p_amp=1e-3)
    o = _oracle(w)
    s0, _ = o.totals()
    o.step(150)
    s1, _ = o.totals()
    assert abs(s1 - s0) <= 1e-12 * np.abs(w.phi0).sum()


def test_momentum_budget():
    """Periodic box: sum_x j(t+1) - sum_x j(t) = sum_x F(t) for any relaxation rates,
    because the first-order rows give m+_3 = j_x + F_x (Eqs. 29, 31, 32)."""
    w = I.perturbed(I.droplet(n=10, R=3.0), seed=2, u_amp=0.02, p_amp=1e-3)
    w.g = (1e-4, -2e-4, 3e-4)
    w.sg = (0.9, 1.1, 1.3, 1.0, 1.2, 1.0, 0.7, 1.0, 1.5, 1.0, 1.0, 1.0, 1.0, 1.0, 1.4)
    o = _oracle(w)
    o.step(2)
    for _ in range(3):
        F = o.macroscopic()["F"].reshape(3, -1).sum(axis=1)
        _, j0 = o.totals()
        o.step(1)
        _, j1 = o.totals()
        np.testing.assert_allclose(j1 - j0, F, atol=1e-14)
        assert np.abs(F).max() > 1e-6  # the check is not vacuous


def test_flat_interface_is_steady():
    """phi = tanh(2z/D) is the mu = 0 profile of Eq. 2 with kappa = 3 D sigma/8 and
    beta = 3 sigma/(4D); on the lattice it relaxes only by the discretisation error of
    the stencil (< 2% of the jump), stays centred, and the flow dies out."""
    w = I.flat_interface(nz=32, nxy=1, steps=3000)
    o = _oracle(w)
    o.step(3000)
    fl = o.fields()
    dphi = fl["phi"] - w.phi0
    assert np.abs(dphi).max() < 0.015
    assert np.abs(fl["u"]).max() < 1e-6
    assert np.abs(fl["mu"]).max() < 5e-5
    # the interface (phi = 0 crossing, linear interpolation) stays at the mid-plane
    prof = fl["phi"][:, 0, 0]
    zc = np.arange(w.nz) + 0.5
    k = int(np.flatnonzero((prof[:-1] < 0) & (prof[1:] >= 0))[0])
    z0 = zc[k] - prof[k] * (zc[k + 1] - zc[k]) / (prof[k + 1] - prof[k])
    assert abs(z0 - w.nz / 2) < 1e-3


def test_hydrostatic_column():
    """Single fluid between walls under G = rho g: the steady state has u = 0 and
    dp/dz = -rho g (gravity along -z)."""
    w = I.flat_interface(nz=12, nxy=1)
    w.phi0 = np.ones(w.shape)
    gacc = 1e-4
    w.g = (0.0, 0.0, -gacc)
    o = _oracle(w)
    o.step(3000)
    fl = o.fields()
    p = fl["p"][:, 0, 0]
    dpdz = np.diff(p)[2:-2]
    np.testing.assert_allclose(dpdz, -w.rho_l * gacc, rtol=1e-3)
    assert np.abs(fl["u"]).max() < 1e-6


@pytest.mark.parametrize("phi_fill", [1.0, -1.0])
def test_hydrostatic_column_buoyancy_form(phi_fill):
    """Single fluid between walls under the buoyancy form G = (rho - (rho_l + rho_g)/2) g:
    the steady state has u = 0 and dp/dz = -(rho - rho_mean) g.  With rho_l = 3,
    rho_g = 1 the liquid column (phi = 1) feels +1 x g and the gas column (phi = -1)
    -1 x g, so the pressure gradient has the gas column's sign reversed; the plain
    weight would give -3 g and -1 g."""
    w = I.flat_interface(nz=12, nxy=1)
    w.phi0 = np.full(w.shape, phi_fill)
    w.buoyancy = True
    gacc = 1e-4
    w.g = (0.0, 0.0, -gacc)
    o = _oracle(w)
    o.step(3000)
    fl = o.fields()
    rho = w.rho_l if phi_fill > 0 else w.rho_g
    p = fl["p"][:, 0, 0]
    dpdz = np.diff(p)[2:-2]
    np.testing.assert_allclose(dpdz, -(rho - 0.5 * (w.rho_l + w.rho_g)) * gacc, rtol=1e-3)
    assert np.abs(fl["u"]).max() < 1e-6


def test_shear_wave_decay_gives_eq33_viscosity():
    """u_x = U sin(2 pi z / N) in one fluid decays like exp(-nu k^2 t) with
    nu = c_s^2 (tau_g - 1/2) (Eq. 33)."""
    n = 64
    w = I.flat_interface(nz=n, nxy=1)
    w.walls_z = False
    w.phi0 = np.ones(w.shape)
    z = np.arange(n)
    u0 = np.zeros((3,) + w.shape)
    u0[0, :, 0, 0] = 1e-3 * np.sin(2 * np.pi * z / n)
    w.u0 = u0
    o = _oracle(w)
    o.step(100)

    def amp():
        return 2 / n * np.sum(o.fields()["u"][0, :, 0, 0] * np.sin(2 * np.pi * z / n))

    a0 = amp()
    o.step(400)
    a1 = amp()
    rate = -np.log(a1 / a0) / 400
    np.testing.assert_allclose(rate, w.nu_l * (2 * np.pi / n) ** 2, rtol=2e-3)


def test_order_parameter_wave_decay_gives_eq19_mobility():
    """Linearised Cahn-Hilliard about phi = 1: a perturbation eps cos(kx) decays at
    Mob k^2 (8 beta + kappa k^2), with Mob = eta c_s^2 (tau_f - 1/2) (Eq. 19)."""
    n = 32
    w = I.flat_interface(nz=1, nxy=1)
    w.nx, w.ny, w.nz, w.walls_z = n, 1, 1, False
    w.sigma, w.D, w.mobility = 0.1, 2.0, 0.1
    x = np.arange(n)
    w.phi0 = (1 + 1e-4 * np.cos(2 * np.pi * x / n)).reshape(1, 1, n)
    o = _oracle(w)
    o.step(100)

    def amp():
        return 2 / n * np.sum((o.fields()["phi"][0, 0] - 1) * np.cos(2 * np.pi * x / n))

    a0 = amp()
    o.step(300)
    a1 = amp()
    rate = -np.log(a1 / a0) / 300
    p = o.p
    k = 2 * np.pi / n
    np.testing.assert_allclose(rate, p.mobility * k * k * (8 * p.beta + p.kappa * k * k), rtol=1e-2)


def test_laplace_law_static_droplet():
    """3D Laplace law: the pressure jump across a static droplet is 2 sigma / R
    (32^3 box, R = 8, D = 4, sigma = 0.01, rho_l/rho_g = 3, nu = 0.1, Mob = 0.1)."""
    w = I.droplet(n=32, R=8.0)
    o = _oracle(w)
    o.step(600)
    fl = o.fields()
    n = w.nx
    x = np.arange(n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt((X - n / 2) ** 2 + (Y - n / 2) ** 2 + (Z - n / 2) ** 2)
    dp = fl["p"][r < w.D].mean() - fl["p"][r > 8.0 + w.D].mean()
    np.testing.assert_allclose(dp, 2 * w.sigma / 8.0, rtol=0.05)
    # spurious currents are small against the capillary velocity scale sigma/(rho nu)
    assert np.abs(fl["u"]).max() < 1e-3 * w.U


def test_time_derivative_is_the_backward_difference(monkeypatch):
    """The CHE source receives d_t(phi u) = phi u(t) - phi u(t - 1) (Eq. 34), from the
    macroscopic fields of consecutive steps, and zero on the first step after
    initialisation (no earlier value exists)."""
    w = I.perturbed(I.droplet(n=10, R=3.0), seed=4, u_amp=0.02, p_amp=1e-3)
    o = _oracle(w)
    seen = []
    orig = O.d3q7_mR

    def spy(d):
        seen.append(np.array(d, copy=True))
        return orig(d)

    monkeypatch.setattr(O, "d3q7_mR", spy)
    fl0 = o.fields()
    o.step(1)
    fl1 = o.fields()
    o.step(1)
    assert len(seen) == 2
    assert np.all(seen[0] == 0)
    expected = fl1["phi"][None] * fl1["u"] - fl0["phi"][None] * fl0["u"]
    np.testing.assert_allclose(seen[1], expected, atol=1e-16)
    assert np.abs(expected).max() > 1e-5


def test_srt_flow_with_unit_rates_equals_mrt_with_unit_rates():
    """The SRT flow lattice sets every lambda_k to the viscous rate; with nu = 1/6 that
    rate is 1, the same as an MRT run whose rates are all 1."""
    w = I.perturbed(I.droplet(n=10, R=3.0, nu=1.0 / 6.0), seed=15, u_amp=0.01, p_amp=1e-3)
    a = _oracle(w)
    a.step(5)
    w.srt_flow = True
    b = _oracle(w)
    b.step(5)
    np.testing.assert_allclose(a.g, b.g, atol=1e-16)
    np.testing.assert_allclose(a.f, b.f, atol=1e-16)


def test_srt_flow_relaxes_all_moments_at_the_viscous_rate(monkeypatch):
    """With srt_flow every D3Q15 moment relaxes at 1/(nu/c_s^2 + 1/2) (text after Eq. 10
    for the SRT special case, Eq. 33 for the rate)."""
    w = I.perturbed(I.droplet(n=8, R=2.5, nu=0.05), seed=16, u_amp=0.01, p_amp=1e-3)
    w.srt_flow = True
    o = _oracle(w)
    seen = []
    orig = O.collide_moments

    def spy(m, meq, rates, msrc):
        seen.append(np.array(rates, copy=True))
        return orig(m, meq, rates, msrc)

    monkeypatch.setattr(O, "collide_moments", spy)
    o.step(1)
    rates_g = seen[0]
    assert rates_g.shape[0] == 15
    np.testing.assert_allclose(rates_g, 1.0 / (3 * 0.05 + 0.5))
