"""Pins of the oracle's difference schemes (Eqs. 35-36) and propagation (Eq. 16).

The stencils are checked against closed-form symbols of plane waves on a periodic
grid (derived by hand from the D3Q15 weights, independent of the oracle's loop), exact
results on low-order polynomials, and the global conservation property the paper
states for them.  Propagation is checked by moving single populations.
"""
import numpy as np
import pytest

from oracle import lbm_oracle as O


def _plane_wave(shape, m):
    nz, ny, nx = shape
    k = 2 * np.pi * np.array([m[0] / nx, m[1] / ny, m[2] / nz])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return k, k[0] * x + k[1] * y + k[2] * z


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 0), (0, 0, 3), (1, 2, 3), (3, 1, 2), (4, 5, 5)])
def test_laplacian_plane_wave_symbol(m):
    """lap cos(k.x) = L(k) cos(k.x) with
    L(k) = 4/3 sum_a (cos k_a - 1) + 2/3 (cos k_x cos k_y cos k_z - 1)."""
    shape = (12, 10, 8)
    k, arg = _plane_wave(shape, m)
    c = np.cos(k)
    L = 4 / 3 * np.sum(c - 1) + 2 / 3 * (np.prod(c) - 1)
    np.testing.assert_allclose(O.lap_iso(np.cos(arg), False), L * np.cos(arg), atol=1e-13)


@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 0), (0, 0, 3), (1, 2, 3), (3, 4, 5)])
def test_gradient_plane_wave_symbol(m):
    """grad_a cos(k.x) = -G_a(k) sin(k.x) with
    G_a = 2/3 sin k_a + 1/3 sin k_a prod_{b != a} cos k_b."""
    shape = (12, 10, 8)
    k, arg = _plane_wave(shape, m)
    s, c = np.sin(k), np.cos(k)
    G = np.array([2 / 3 * s[0] + 1 / 3 * s[0] * c[1] * c[2],
                  2 / 3 * s[1] + 1 / 3 * s[1] * c[0] * c[2],
                  2 / 3 * s[2] + 1 / 3 * s[2] * c[0] * c[1]])
    got = O.grad_iso(np.cos(arg), False)
    for a in range(3):
        np.testing.assert_allclose(got[a], -G[a] * np.sin(arg), atol=1e-13)


def test_second_order_in_space():
    """The Laplacian symbol tends to -|k|^2 with an error that falls like |k|^2
    (second order, text after Eq. 36): halving k quarters the relative error."""
    errs = []
    for n in (32, 64):
        k, arg = _plane_wave((n, n, n), (1, 1, 1))
        lap = O.lap_iso(np.cos(arg), False)[0, 0, 0]
        errs.append(abs(lap / (-np.dot(k, k)) - 1))
    assert 3.9 < errs[0] / errs[1] < 4.1


def test_exact_on_polynomials_between_walls():
    """Between walls (z = k + 1/2) a linear and a quadratic profile in z have exact
    gradient and Laplacian away from the wall rows; the wall rows see the ghost copy of
    the adjacent node."""
    nz = 10
    z = (np.arange(nz) + 0.5)[:, None, None] * np.ones((nz, 3, 4))
    g = O.grad_iso(z, True)
    np.testing.assert_allclose(g[2][1:-1], 1.0, atol=1e-14)
    np.testing.assert_allclose(g[0], 0, atol=1e-14)
    np.testing.assert_allclose(g[1], 0, atol=1e-14)
    # bottom row: ghost z(-1) = z(0), so the central difference is (z1 - z0)/2
    np.testing.assert_allclose(g[2][0], 0.5, atol=1e-14)
    q = z ** 2
    lap = O.lap_iso(q, True)
    np.testing.assert_allclose(lap[1:-1], 2.0, atol=1e-12)
    np.testing.assert_allclose(lap[0], q[1] - q[0], atol=1e-12)
    np.testing.assert_allclose(lap[-1], q[-2] - q[-1], atol=1e-12)


@pytest.mark.parametrize("walls", [False, True])
def test_laplacian_sums_to_zero(walls):
    """Global conservation property of the isotropic Laplacian (text after Eq. 36)."""
    chi = np.random.default_rng(0).uniform(-1, 1, (9, 7, 6))
    assert abs(O.lap_iso(chi, walls).sum()) < 1e-12


def test_neighbour_periodic_and_ghost():
    chi = np.arange(4 * 3 * 5, dtype=float).reshape(4, 3, 5)
    nb = O.neighbour(chi, (1, -1, 1), False)
    assert nb[0, 0, 0] == chi[1, 2, 1]
    assert nb[3, 2, 4] == chi[0, 1, 0]
    nbw = O.neighbour(chi, (1, 0, 1), True)
    assert nbw[3, 1, 2] == chi[3, 1, 3]  # top ghost = top node
    nbw = O.neighbour(chi, (0, 1, -1), True)
    assert nbw[0, 1, 2] == chi[0, 2, 2]  # bottom ghost = bottom node


# --------------------------------------------------------------- propagation ----

@pytest.mark.parametrize("lattice", ["d3q7", "d3q15"])
def test_stream_moves_each_population_along_its_velocity(lattice):
    C, opp = (O.D3Q7_C, O.OPP7) if lattice == "d3q7" else (O.D3Q15_C, O.OPP15)
    shape = (5, 6, 7)
    x0 = np.array([2, 3, 4])  # (z, y, x)
    for i, c in enumerate(C):
        post = np.zeros((len(C),) + shape)
        post[i][tuple(x0)] = 1.0
        out = O.stream(post, C, opp, walls_z=False)
        dest = (x0 + np.array([c[2], c[1], c[0]])) % np.array(shape)
        assert out[i][tuple(dest)] == 1.0
        assert out.sum() == 1.0


def test_stream_periodic_wrap_and_bounce_back():
    C, opp = O.D3Q15_C, O.OPP15
    shape = (4, 3, 3)
    for i, c in enumerate(C):
        if c[2] == 0:
            continue
        post = np.zeros((15,) + shape)
        zsrc = 3 if c[2] > 0 else 0  # population leaving through the wall
        post[i][zsrc, 1, 1] = 1.0
        out = O.stream(post, C, opp, walls_z=True)
        # comes back to the same node, reversed
        assert out[opp[i]][zsrc, 1, 1] == 1.0
        assert out.sum() == 1.0
        # periodic in z instead: wraps to the other side
        out = O.stream(post, C, opp, walls_z=False)
        assert out[i][(zsrc + c[2]) % 4, (1 + c[1]) % 3, (1 + c[0]) % 3] == 1.0


@pytest.mark.parametrize("walls", [False, True])
def test_stream_is_a_permutation(walls):
    rng = np.random.default_rng(3)
    post = rng.uniform(size=(15, 6, 5, 4))
    out = O.stream(post, O.D3Q15_C, O.OPP15, walls)
    np.testing.assert_array_equal(np.sort(out.ravel()), np.sort(post.ravel()))


@pytest.mark.parametrize("m", [(1, 0, 0), (1, 2, 3), (3, 4, 5)])
def test_d3q7_weighted_schemes_are_central_differences(m):
    """With the D3Q7 weights (omega_i / c_s^2 = 1/2) Eqs. 35-36 become the 7-point
    central differences: lap symbol 2 sum_a (cos k_a - 1), grad symbol sin k_a."""
    shape = (12, 10, 8)
    k, arg = _plane_wave(shape, m)
    L7 = 2 * np.sum(np.cos(k) - 1)
    np.testing.assert_allclose(O.lap_iso(np.cos(arg), False, "d3q7"), L7 * np.cos(arg), atol=1e-13)
    got = O.grad_iso(np.cos(arg), False, "d3q7")
    for a in range(3):
        np.testing.assert_allclose(got[a], -np.sin(k[a]) * np.sin(arg), atol=1e-13)
