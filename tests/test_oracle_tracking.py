"""Pins of the oracle's interface-tracking mode (Sec. III A, B): only the D3Q7 lattice
evolves (Eq. 4) and the velocity is prescribed (Eqs. 37, 41).

Checks: a slab carried by a uniform velocity moves by U t; a blob in the rigid
rotation of Eq. 37 turns by the angle Omega t; in the time-reversed deformation flow of
Eq. 41 the interface deforms at T/2 and comes back at T (the Err of Eq. 40 falls by two
orders); mass is conserved; the velocity fields are divergence-free and match their
formulas at hand-picked points.
"""
import numpy as np
import pytest

from oracle import lbm_oracle as O
from paper_1507_07294_gb300 import diagnostics as Dg
from paper_1507_07294_gb300 import inputs as I


def _oracle(w):
    o = O.Oracle(O.Params.from_workload(w))
    o.init(w.phi0, w.u0, w.p0)
    return o


def test_velocity_fields_at_points():
    box = (100, 100, 100)
    # Eq. 37 at (x, y, z) = (3, 70, 20): v = (U pi/100)(50 - z), w = (U pi/100)(y - 50)
    u = O.prescribed_velocity("rotation", 0.02, 1.0, box, 0, coords=([20], [70], [3]))
    np.testing.assert_allclose(u[:, 0], [0.0, 0.02 * np.pi / 100 * 30, 0.02 * np.pi / 100 * 20])
    # Eq. 41 at x = 25, y = z = 12.5, L = 100, t/T = 1/4: sin^2(pi/4) = 1/2,
    # sin(pi/2) = 1, sin^2(pi/8) = (1 - 1/sqrt(2))/2, sin(pi/4) = 1/sqrt(2), cos(pi/4) = 1/sqrt(2)
    u = O.prescribed_velocity("deformation", 0.02, 200.0, box, 50.0, coords=([12.5], [12.5], [25]))
    r2 = 1 / np.sqrt(2)
    s2q = (1 - r2) / 2
    U = 0.02
    np.testing.assert_allclose(u[:, 0], [2 * U * 0.5 * r2 * r2 * r2, -U * 1.0 * s2q * r2 * r2,
                                         -U * 1.0 * r2 * s2q * r2], rtol=1e-12)


@pytest.mark.parametrize("kind", ["rotation", "deformation"])
def test_velocity_fields_are_divergence_free(kind):
    """Central differences of the fields sum to zero up to O(h^2) (rotation: exactly)."""
    n = 64
    u = O.prescribed_velocity(kind, 0.02, 100.0, (n, n, n), 10.0)
    div = ((np.roll(u[0], -1, 2) - np.roll(u[0], 1, 2)) + (np.roll(u[1], -1, 1) - np.roll(u[1], 1, 1))
           + (np.roll(u[2], -1, 0) - np.roll(u[2], 1, 0))) / 2.0
    inner = div[2:-2, 2:-2, 2:-2]
    assert np.abs(inner).max() < (1e-15 if kind == "rotation" else 2e-5)


def test_uniform_velocity_translates_the_interface():
    w = I.translating_slab(n=64, U=0.02)
    o = _oracle(w)
    o.step(800)
    cross = Dg.interface_crossings(o.fields()["phi"][0, 0], np.arange(64))
    # the left interface started at x = 16 and moved by U t = 16 cells
    assert abs(cross[0] - 32.0) < 0.25
    o.step(2400)  # one full period n / U
    assert Dg.relative_error(o.fields()["phi"], w.phi0) < 0.03


def test_rotation_turns_a_blob_by_omega_t():
    n = 24
    w = I.zalesak(n=n)
    x, y, z = I.node_coords(n, n, n, False)
    r = np.sqrt((x - n / 2) ** 2 + (y - n / 2) ** 2 + (z - n / 2 + 6) ** 2)
    w.phi0 = np.broadcast_to(np.tanh(2 * (4 - r) / 2.0), (n, n, n)).copy()
    o = _oracle(w)
    o.step(int(2 * n / 0.02 / 4))  # a quarter turn: Omega t = pi / 2
    ph = (o.fields()["phi"] + 1) / 2
    Z, Y, X = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    com = [(ph * A).sum() / ph.sum() for A in (X, Y, Z)]
    # started at (y, z) = (n/2, n/2 - 6); a quarter turn takes it to (n/2 + 6, n/2)
    np.testing.assert_allclose(com, [n / 2, n / 2 + 6, n / 2], atol=0.1)


def test_deformation_flow_returns_the_sphere():
    w = I.deformation(n=32, period=750.0)
    o = _oracle(w)
    o.step(375)
    err_half = Dg.relative_error(o.fields()["phi"], w.phi0)
    o.step(375)
    phi_T = o.fields()["phi"]
    err_T = Dg.relative_error(phi_T, w.phi0)
    assert err_half > 0.02          # strongly deformed at T/2
    assert err_T < err_half / 20    # back at T
    assert abs(phi_T.sum() - w.phi0.sum()) < 1e-9 * np.abs(w.phi0).sum()


def test_carried_interface_overshoot_at_small_sigma():
    """A limit of the scheme, not a pin of a printed value: the D3Q7 equilibrium puts all
    of phi on the rest population (f_i^eq, i != 0, holds only omega_i eta mu and the flux
    c_i . phi u / 2), so advection adds no numerical diffusion of phi and is slightly
    anti-diffusive; only the Cahn-Hilliard term M lap(mu) holds the profile.  At the
    Rayleigh-Taylor setting (sigma = 1e-4, D = 4, S^f of Eq. 45) a carried interface
    overshoots +-1 more and more; with the tracking runs' sigma and S^f (Eq. 38) it stays
    close to +-1."""
    def overshoot(sigma, D, mob, sf, steps):
        w = I.translating_slab(n=64, U=0.02, D=D, sigma=sigma, mobility=mob)
        w.sf = sf
        o = _oracle(w)
        o.step(steps)
        return float(np.abs(O.order_parameter(o.f)).max())
    small_sigma = overshoot(1e-4, 4.0, 0.05, I.SF_COUPLED, 1600)
    assert small_sigma > 1.1
    assert overshoot(0.04, 2.0, 0.02, I.SF_TRACKING, 1600) < 1.01
    assert overshoot(1e-4, 4.0, 0.05, I.SF_TRACKING, 1600) < small_sigma - 0.08
