"""Pins of the oracle's lattices, moment matrices, equilibria and source terms.

Each check ties the oracle to something other than itself: the matrices the paper
prints (golden fixtures), the weight conditions of Eq. 7, or a second transcription
of the same quantity from another equation of the paper (population space vs moment
space).
"""
import itertools

import numpy as np
import pytest

from oracle import lbm_oracle as O
from tests.golden_io import load


# ---------------------------------------------------------------- lattices -------

def test_d3q15_velocity_order_matches_eq23():
    C = load("d3q15_velocities.txt").T
    np.testing.assert_array_equal(C, O.D3Q15_C)


def test_d3q7_matrix_matches_printed_eq9():
    np.testing.assert_array_equal(O.d3q7_moment_matrix(), load("d3q7_M.txt"))


def test_d3q15_matrix_matches_printed_eq25():
    """Read each printed column's velocity from rows 3, 5, 7 (c_x, c_y, c_z), evaluate
    the oracle's row polynomials on those velocities and compare all 15 rows."""
    G = load("d3q15_Gamma.txt")
    C_printed = G[[3, 5, 7]].T.astype(np.int64)
    # the printed columns are a permutation of the Eq. 23 velocity set
    assert sorted(map(tuple, C_printed)) == sorted(map(tuple, O.D3Q15_C))
    np.testing.assert_array_equal(O.d3q15_moment_matrix(C_printed), G)


def test_d3q15_corner_order_differs_from_eq23():
    """The printed corner columns are NOT in Eq. 23's order: evaluating the polynomial
    rows in Eq. 23's order must differ from the printed matrix (why Gamma is defined by
    its polynomials)."""
    G = load("d3q15_Gamma.txt")
    assert not np.array_equal(O.d3q15_moment_matrix(O.D3Q15_C), G)


@pytest.mark.parametrize("A", [0.1, 0.25, 0.3])
def test_d3q7_weight_conditions_eq7(A):
    w = O.d3q7_weights(A)
    C = O.D3Q7_C.astype(float)
    assert abs(w.sum() - 1) < 1e-15
    np.testing.assert_allclose(w @ C, 0, atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, C, C), A * np.eye(3), atol=1e-15)


def test_d3q15_weight_conditions():
    """Eq. 7's conditions with c_s^2 = 1/3, plus the fourth-order isotropy the flow
    lattice needs."""
    w, C = O.D3Q15_W, O.D3Q15_C.astype(float)
    cs2 = O.D3Q15_CS2
    assert abs(w.sum() - 1) < 1e-15
    np.testing.assert_allclose(w @ C, 0, atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, C, C), cs2 * np.eye(3), atol=1e-15)
    four = np.einsum("i,ia,ib,ic,id->abcd", w, C, C, C, C)
    d = np.eye(3)
    iso = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                      + np.einsum("ad,bc->abcd", d, d))
    np.testing.assert_allclose(four, iso, atol=1e-15)


def test_rows_orthogonal_with_known_norms():
    for T, norms in ((O.M7, [7, 2, 2, 2, 42, 12, 4]),
                     (O.GAMMA, [15, 18, 360, 10, 40, 10, 40, 10, 40, 12, 4, 8, 8, 8, 8])):
        np.testing.assert_array_equal(T @ T.T, np.diag(norms))
        np.testing.assert_allclose(T @ np.linalg.inv(T), np.eye(len(norms)), atol=1e-13)


def test_opposites():
    for C, opp in ((O.D3Q7_C, O.OPP7), (O.D3Q15_C, O.OPP15)):
        np.testing.assert_array_equal(C[opp], -C)


# ------------------------------------------------------------- equilibria --------

def _rand_state(rng, n=50):
    phi = rng.uniform(-1.2, 1.2, n)
    mu = rng.uniform(-0.1, 0.1, n)
    u = rng.uniform(-0.1, 0.1, (3, n))
    p = rng.uniform(-0.05, 0.05, n)
    rho = rng.uniform(0.5, 3.0, n)
    return phi, mu, u, p, rho


@pytest.mark.parametrize("A", [0.1, 0.25, 0.3])
def test_d3q7_equilibrium_moments_eq5_vs_eq17(A):
    rng = np.random.default_rng(1)
    phi, mu, u, _, _ = _rand_state(rng)
    eta = 0.7
    feq = O.d3q7_feq(phi, mu, u, eta, A)
    np.testing.assert_allclose(O.M7 @ feq, O.d3q7_mfeq(phi, mu, u, eta, A), atol=1e-14)
    # the order parameter is the zeroth moment of the equilibrium (Eq. 13)
    np.testing.assert_allclose(feq.sum(axis=0), phi, atol=1e-14)


@pytest.mark.parametrize("A", [0.1, 0.25])
def test_d3q7_source_moments_eq12_vs_eq18(A):
    rng = np.random.default_rng(2)
    d = rng.uniform(-1e-3, 1e-3, (3, 40))
    np.testing.assert_allclose(O.M7 @ O.d3q7_R(d, A), O.d3q7_mR(d), atol=1e-17)


def test_d3q15_equilibrium_moments_eq21_vs_eq31():
    rng = np.random.default_rng(3)
    _, _, u, p, rho = _rand_state(rng)
    geq = O.d3q15_geq(p, rho, u)
    np.testing.assert_allclose(O.GAMMA @ geq, O.d3q15_mgeq(p, rho, u), atol=1e-14)
    # zeroth and first moments: sum g^eq = 0 and sum c_i g^eq = rho u
    np.testing.assert_allclose(geq.sum(axis=0), 0, atol=1e-15)
    np.testing.assert_allclose(O.D3Q15_C.T.astype(float) @ geq, rho * u, atol=1e-15)


def test_d3q15_s_moments():
    """sum_i s_i = 0, sum_i c_i s_i = u (Eq. 22 with the weight conditions)."""
    u = np.array([0.03, -0.02, 0.05])
    s = O.d3q15_s(u)
    assert abs(s.sum()) < 1e-16
    np.testing.assert_allclose(O.D3Q15_C.T.astype(float) @ s, u, atol=1e-16)


def test_d3q15_source_eq28_vs_eq32_exact_rows_and_quadratic_rest():
    """Eq. 32 is Gamma T of Eq. 28 up to O(u^2): rows 0, 3, 5, 7 (mass flux and forces)
    agree exactly; all other differences vanish with u like u^2."""
    rng = np.random.default_rng(4)
    grad_rho = rng.uniform(-0.1, 0.1, 3)
    F = rng.uniform(-1e-3, 1e-3, 3)
    direction = rng.uniform(-1, 1, 3)
    diffs = []
    for scale in (1e-2, 5e-3, 2.5e-3):
        u = scale * direction
        d = O.GAMMA @ O.d3q15_T(u, grad_rho, F) - O.d3q15_mT(u, grad_rho, F)
        np.testing.assert_allclose(d[[0, 3, 5, 7]], 0, atol=1e-18)
        diffs.append(np.abs(d).max())
    # quadratic: halving u divides the difference by 4
    assert diffs[0] > 0
    np.testing.assert_allclose(diffs[0] / diffs[1], 4.0, rtol=1e-6)
    np.testing.assert_allclose(diffs[1] / diffs[2], 4.0, rtol=1e-6)


def test_d3q15_source_at_rest_is_exact():
    """With u = 0 every row of Eq. 32 equals Gamma T exactly (only the force rows and
    their energy-flux companions are non-zero)."""
    grad_rho = np.array([0.05, -0.02, 0.01])
    F = np.array([1e-3, 2e-3, -3e-3])
    u = np.zeros(3)
    np.testing.assert_allclose(O.GAMMA @ O.d3q15_T(u, grad_rho, F),
                               O.d3q15_mT(u, grad_rho, F), atol=1e-18)


# -------------------------------------------------- macroscopic recovery ---------

def test_velocity_and_pressure_recover_equilibrium_state():
    """For g = g^eq(p, rho, u) with no force and uniform density, Eqs. 29-30 return
    u and p exactly."""
    rng = np.random.default_rng(5)
    n = 30
    u = rng.uniform(-0.1, 0.1, (3, n))
    p = rng.uniform(-0.05, 0.05, n)
    rho = rng.uniform(1, 3, n)
    g = O.d3q15_geq(p, rho, u)
    z3 = np.zeros((3, n))
    uu = O.velocity(g, rho, z3, z3, np.zeros(n), 3.0, 1.0, 0.1)
    np.testing.assert_allclose(uu, u, atol=1e-15)
    np.testing.assert_allclose(O.pressure(g, uu, z3, rho), p, atol=1e-15)


def test_velocity_is_the_half_force_momentum_balance():
    """Eq. 29 rearranged: rho u = sum c_i g_i + (F_s + F_a + G)/2 with
    F_a = (rho_l - rho_g) Mob lap(mu) u / 2."""
    rng = np.random.default_rng(6)
    n = 25
    g = rng.uniform(-0.01, 0.01, (15, n))
    rho = rng.uniform(1, 3, n)
    Fs = rng.uniform(-1e-3, 1e-3, (3, n))
    G = rng.uniform(-1e-3, 1e-3, (3, n))
    lap_mu = rng.uniform(-0.1, 0.1, n)
    rl, rg, mob = 3.0, 1.0, 0.2
    u = O.velocity(g, rho, Fs, G, lap_mu, rl, rg, mob)
    Fa = 0.5 * (rl - rg) * mob * lap_mu * u
    j = O.D3Q15_C.T.astype(float) @ g
    np.testing.assert_allclose(rho * u, j + 0.5 * (Fs + Fa + G), atol=1e-16)


def test_pressure_density_gradient_term():
    """With g = g^eq(p, rho, u) and a density gradient, Eq. 30 adds
    c_s^2/(1-omega_0) * u.grad(rho)/2 to p."""
    u = np.array([[0.02], [0.01], [-0.03]])
    p = np.array([0.01])
    rho = np.array([2.0])
    gr = np.array([[0.1], [0.2], [-0.1]])
    g = O.d3q15_geq(p, rho, u)
    extra = (1 / 3) / (1 - 2 / 9) * 0.5 * float(np.sum(u * gr))
    np.testing.assert_allclose(O.pressure(g, u, gr, rho), p + extra, atol=1e-16)


# ------------------------------------------------------------ collision ---------

def test_srt_reduction_d3q7():
    """All rates equal to s: the moment-space collision equals the textbook BGK
    collision with forcing F_i = (1 - s/2) R_i in population space (text after Eq. 10)."""
    rng = np.random.default_rng(7)
    n, A, eta, s = 20, 0.25, 0.9, 1.37
    f = rng.uniform(-0.2, 1.0, (7, n))
    phi, mu, u = f.sum(0), rng.uniform(-0.05, 0.05, n), rng.uniform(-0.05, 0.05, (3, n))
    d = rng.uniform(-1e-3, 1e-3, (3, n))
    mpost = O.collide_moments(O.M7 @ f, O.d3q7_mfeq(phi, mu, u, eta, A),
                              np.full((7, 1), s), O.d3q7_mR(d))
    bgk = f - s * (f - O.d3q7_feq(phi, mu, u, eta, A)) + (1 - s / 2) * O.d3q7_R(d, A)
    np.testing.assert_allclose(O.M7_INV @ mpost, bgk, atol=1e-14)


def test_srt_reduction_d3q15():
    rng = np.random.default_rng(8)
    n, s = 20, 1.6
    g = rng.uniform(-0.01, 0.01, (15, n))
    u = rng.uniform(-0.05, 0.05, (3, n))
    p, rho = rng.uniform(-0.01, 0.01, n), rng.uniform(1, 3, n)
    gr, F = rng.uniform(-0.1, 0.1, (3, n)), rng.uniform(-1e-3, 1e-3, (3, n))
    mT = O.d3q15_mT(u, gr, F)
    mpost = O.collide_moments(O.GAMMA @ g, O.d3q15_mgeq(p, rho, u), np.full((15, 1), s), mT)
    bgk = g - s * (g - O.d3q15_geq(p, rho, u)) + (1 - s / 2) * (O.GAMMA_INV @ mT)
    np.testing.assert_allclose(O.GAMMA_INV @ mpost, bgk, atol=1e-15)


def test_collision_conserves_phi_for_any_rates():
    rng = np.random.default_rng(9)
    n = 16
    f = rng.uniform(-0.2, 1.0, (7, n))
    phi = f.sum(0)
    rates = rng.uniform(0.1, 1.9, (7, 1))
    mpost = O.collide_moments(O.M7 @ f,
                              O.d3q7_mfeq(phi, rng.uniform(-.1, .1, n), rng.uniform(-.1, .1, (3, n)), 0.5, 0.25),
                              rates, O.d3q7_mR(rng.uniform(-1e-3, 1e-3, (3, n))))
    np.testing.assert_allclose((O.M7_INV @ mpost).sum(0), phi, atol=1e-15)


def test_parameter_relations():
    p = O.Params(nx=4, ny=4, nz=4, walls_z=False, rho_l=3, rho_g=1, nu_l=0.1, nu_g=0.01,
                 mobility=0.1, D=4.0, sigma=0.01, g=(0, 0, 0))
    assert abs(p.kappa - 3 * 4 * 0.01 / 8) < 1e-18
    assert abs(p.beta - 3 * 0.01 / 16) < 1e-18
    # Eq. 19 with tau_f = 1/1.25 = 0.8 and c_s^2 = A = 0.25
    assert abs(p.eta * 0.25 * (0.8 - 0.5) - 0.1) < 1e-15
    # Eq. 33: nu = c_s^2 (tau_g - 1/2) at both pure phases
    for phi, nu in ((1.0, 0.1), (-1.0, 0.01)):
        tau = 1.0 / p.viscous_rate(np.array(phi))
        assert abs((tau - 0.5) / 3.0 - nu) < 1e-15
