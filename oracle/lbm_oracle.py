"""FP64 CPU oracle for the three-dimensional MRT lattice Boltzmann multiphase model of
Liang, Shi and Chai, "An efficient three-dimensional multiple-relaxation-time lattice
Boltzmann model for multiphase flows" (arXiv:1507.07294).

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct statement
of what one time step of the method computes.  Only the test-suite, the package's
smoke check and the benchmark's CPU-baseline leg may import it; the product path never
does.  It shares no code with the CUDA path.

Equation numbers are those of the paper, counted in order of appearance (Eq. 1 is the
Cahn-Hilliard equation, Eq. 4 the D3Q7 lattice Boltzmann equation, Eq. 20 the D3Q15
one, Eqs. 35-36 the isotropic difference schemes).

How it is written
-----------------
* Everything is float64 numpy, vectorised over the whole grid.  Arrays are indexed
  [z, y, x] (x fastest); population sets as [q, z, y, x]; vectors as [3, z, y, x].
* The moment matrices M (Eq. 9) and Gamma (Eq. 25) are built by evaluating their row
  polynomials on the discrete velocities in the paper's order (Eqs. 6 and 23); their
  inverses come from numerical inversion.  The transforms are dense matrix products.
* Collisions run in moment space with the paper's closed-form equilibria and sources
  (Eqs. 17-18 and 31-32).  The population-space equilibria and sources (Eqs. 5, 12,
  21, 22, 28) are also written out: the tests check each pair against the other.
* Streaming is a pull: f_i(x, t+1) = f_i^+(x - c_i, t) (Eq. 16).

Readings of points the paper leaves open (both this oracle and the CUDA path follow
them)
-----------------------------------------------------------------------------------
* Gamma's columns 7..14 are printed in d'Humieres' corner order, not the order of
  Eq. 23; Gamma is therefore defined by its row polynomials, evaluated on whatever
  velocity order the code uses.
* The difference schemes Eqs. 35-36 use the D3Q15 weights and c_s^2 = 1/3 (the flow
  lattice), giving a 15-point stencil.  The Laplacian has no factor c_i (a misprint).
* The first step after initialisation takes d_t(phi u) = 0 (no earlier value).
* The kinematic viscosity is interpolated linearly in phi between nu_g and nu_l; the
  five viscous rates are lambda_9..13 = 1 / (nu(phi)/c_s^2 + 1/2) (Eq. 33).
* rho_A, rho_B in F_a and Eq. 29 are rho_l, rho_g.
* No-slip walls (Sec. III C) are halfway bounce-back of both f and g at z = 0 and
  z = nz; the stencils see a ghost layer equal to the adjacent fluid node (zero normal
  gradient).
* The external force is the weight G = rho g (vector g); optionally the buoyancy form
  G = (rho - (rho_l + rho_g)/2) g.
* eta follows from the mobility by Eq. 19 with tau_f = 1/s_1 (s_1 = s_2 = s_3).

Pins: the tests in tests/test_oracle_*.py tie each function to something other than
itself (printed matrices, closed-form symbols, exact invariants, special cases).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

# ----------------------------------------------------------------------------------
# Lattices
# ----------------------------------------------------------------------------------

#: D3Q7 discrete velocities in the order of Eq. 6 (c = 1).
D3Q7_C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0],
                   [0, 0, 1], [0, 0, -1]], dtype=np.int64)

#: D3Q15 discrete velocities in the order of Eq. 23 (c = 1).
D3Q15_C = np.array([[0, 0, 0],
                    [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                    [1, 1, 1], [-1, -1, -1], [1, 1, -1], [-1, -1, 1],
                    [1, -1, 1], [-1, 1, -1], [1, -1, -1], [-1, 1, 1]], dtype=np.int64)

#: D3Q15 weights, Eq. 24.
D3Q15_W = np.array([2.0 / 9.0] + [1.0 / 9.0] * 6 + [1.0 / 72.0] * 8)

#: D3Q15 sound speed squared: c = sqrt(3) c_s with c = 1 (text after Eq. 23).
D3Q15_CS2 = 1.0 / 3.0


def d3q7_weights(A: float) -> np.ndarray:
    """omega_0 = 1 - 3A, omega_1..6 = A/2 (Eq. 8); c_s^2 = A (text after Eq. 8)."""
    return np.array([1.0 - 3.0 * A] + [A / 2.0] * 6)


def opposite(C: np.ndarray) -> np.ndarray:
    """Index of -c_i for every i."""
    return np.array([int(np.flatnonzero((C == -c).all(axis=1))[0]) for c in C])


def d3q7_moment_matrix(C: np.ndarray = D3Q7_C) -> np.ndarray:
    """M of Eq. 9, row by row from the velocity polynomials
    1, c_x, c_y, c_z, 6 - 7|c|^2, 3c_x^2 - |c|^2, c_y^2 - c_z^2."""
    cx, cy, cz = (C[:, a].astype(np.float64) for a in range(3))
    c2 = cx ** 2 + cy ** 2 + cz ** 2
    rows = [np.ones_like(cx), cx, cy, cz, 6.0 - 7.0 * c2, 3.0 * cx ** 2 - c2,
            cy ** 2 - cz ** 2]
    return np.array(rows)


def d3q15_moment_matrix(C: np.ndarray = D3Q15_C) -> np.ndarray:
    """Gamma of Eq. 25 from its row polynomials (d'Humieres' basis):
    1, c^2 - 2, (15c^4 - 55c^2 + 32)/2, c_x, (5c^2 - 13)c_x/2, c_y, (5c^2 - 13)c_y/2,
    c_z, (5c^2 - 13)c_z/2, 3c_x^2 - c^2, c_y^2 - c_z^2, c_x c_y, c_y c_z, c_x c_z,
    c_x c_y c_z."""
    cx, cy, cz = (C[:, a].astype(np.float64) for a in range(3))
    c2 = cx ** 2 + cy ** 2 + cz ** 2
    q = (5.0 * c2 - 13.0) / 2.0
    rows = [np.ones_like(cx), c2 - 2.0, (15.0 * c2 ** 2 - 55.0 * c2 + 32.0) / 2.0,
            cx, q * cx, cy, q * cy, cz, q * cz,
            3.0 * cx ** 2 - c2, cy ** 2 - cz ** 2,
            cx * cy, cy * cz, cx * cz, cx * cy * cz]
    return np.array(rows)


M7 = d3q7_moment_matrix()
M7_INV = np.linalg.inv(M7)
GAMMA = d3q15_moment_matrix()
GAMMA_INV = np.linalg.inv(GAMMA)
OPP7 = opposite(D3Q7_C)
OPP15 = opposite(D3Q15_C)


def to_moments(T: np.ndarray, pops: np.ndarray) -> np.ndarray:
    """Dense product T @ pops over the leading (population) axis."""
    return np.tensordot(T, pops, axes=(1, 0))


# ----------------------------------------------------------------------------------
# Equilibria and source terms
# ----------------------------------------------------------------------------------

def _dot_c(C: np.ndarray, v: np.ndarray) -> np.ndarray:
    """c_i . v for every i: shape (q, ...)."""
    return np.tensordot(C.astype(np.float64), v, axes=(1, 0))


def d3q7_feq(phi, mu, u, eta, A):
    """f_i^eq of Eq. 5: phi + (omega_0 - 1) eta mu for i = 0,
    omega_i eta mu + omega_i c_i . (phi u) / c_s^2 otherwise (c_s^2 = A)."""
    w = d3q7_weights(A)
    w_ = w.reshape((-1,) + (1,) * np.ndim(phi))
    feq = w_ * eta * mu + w_ * _dot_c(D3Q7_C, phi * u) / A
    feq[0] = phi + (w[0] - 1.0) * eta * mu
    return feq


def d3q7_mfeq(phi, mu, u, eta, A):
    """Moment-space equilibrium of Eq. 17 (c = 1):
    (phi, phi u_x, phi u_y, phi u_z, 6 phi - 21 A eta mu, 0, 0)."""
    z = np.zeros_like(phi)
    return np.array([phi, phi * u[0], phi * u[1], phi * u[2],
                     6.0 * phi - 21.0 * A * eta * mu, z, z])


def d3q7_R(dt_phiu, A):
    """R_i = omega_i c_i . d_t(phi u) / c_s^2 (Eq. 12)."""
    w = d3q7_weights(A).reshape((-1,) + (1,) * (np.ndim(dt_phiu) - 1))
    return w * _dot_c(D3Q7_C, dt_phiu) / A


def d3q7_mR(dt_phiu):
    """Moment-space source of Eq. 18 (c = 1): (0, d_t(phi u), 0, 0, 0)."""
    z = np.zeros_like(dt_phiu[0])
    return np.array([z, dt_phiu[0], dt_phiu[1], dt_phiu[2], z, z, z])


def d3q15_s(u):
    """s_i(u) of Eq. 22."""
    cs2 = D3Q15_CS2
    cu = _dot_c(D3Q15_C, u)
    uu = np.sum(u * u, axis=0)
    w = D3Q15_W.reshape((-1,) + (1,) * (np.ndim(u) - 1))
    return w * (cu / cs2 + cu ** 2 / (2.0 * cs2 ** 2) - uu / (2.0 * cs2))


def d3q15_geq(p, rho, u):
    """g_i^eq of Eq. 21: p/c_s^2 (omega_0 - 1) + rho s_0 for i = 0,
    p/c_s^2 omega_i + rho s_i otherwise."""
    w = D3Q15_W.reshape((-1,) + (1,) * np.ndim(p))
    geq = p / D3Q15_CS2 * w + rho * d3q15_s(u)
    geq[0] = geq[0] - p / D3Q15_CS2
    return geq


def d3q15_mgeq(p, rho, u):
    """Moment-space equilibrium of Eq. 31 with c = 1."""
    ux, uy, uz = u
    uu = ux * ux + uy * uy + uz * uz
    z = np.zeros_like(p)
    return np.array([
        z,
        3.0 * p + rho * uu,
        -(45.0 * p + 5.0 * rho * uu),
        rho * ux, -7.0 * rho * ux / 3.0,
        rho * uy, -7.0 * rho * uy / 3.0,
        rho * uz, -7.0 * rho * uz / 3.0,
        rho * (2.0 * ux * ux - uy * uy - uz * uz),
        rho * (uy * uy - uz * uz),
        rho * ux * uy, rho * uy * uz, rho * ux * uz,
        z])


def d3q15_T(u, grad_rho, F):
    """T_i of Eq. 28: (c_i - u)/c_s^2 . [s_i grad(rho c_s^2) + F (s_i + omega_i)]."""
    cs2 = D3Q15_CS2
    s = d3q15_s(u)
    w = D3Q15_W.reshape((-1,) + (1,) * (np.ndim(u) - 1))
    X = cs2 * grad_rho
    cmu = D3Q15_C.astype(np.float64).reshape((15, 3) + (1,) * (np.ndim(u) - 1)) - u[None]
    vec = s[:, None] * X[None] + F[None] * (s + w)[:, None]
    return np.sum(cmu * vec, axis=1) / cs2


def d3q15_mT(u, grad_rho, F):
    """Moment-space source of Eq. 32 with c = 1; X = c_s^2 grad(rho).  The brace
    grouping of rows 11-13 is read as u_a (X_b + F_b) + u_b (X_a + F_a)."""
    cs2 = D3Q15_CS2
    X = cs2 * grad_rho
    ux, uy, uz = u
    Fx, Fy, Fz = F
    Yx, Yy, Yz = X[0] + Fx, X[1] + Fy, X[2] + Fz
    udX = ux * X[0] + uy * X[1] + uz * X[2]
    udF = ux * Fx + uy * Fy + uz * Fz
    udrho = ux * grad_rho[0] + uy * grad_rho[1] + uz * grad_rho[2]
    z = np.zeros_like(ux)
    return np.array([
        udrho,
        -udX + 2.0 * udF,
        -(7.0 * udX + 10.0 * udF),
        Fx, -7.0 * Fx / 3.0,
        Fy, -7.0 * Fy / 3.0,
        Fz, -7.0 * Fz / 3.0,
        4.0 * ux * Yx - 2.0 * uy * Yy - 2.0 * uz * Yz,
        2.0 * uy * Yy - 2.0 * uz * Yz,
        ux * Yy + uy * Yx,
        uy * Yz + uz * Yy,
        ux * Yz + uz * Yx,
        z])


# ----------------------------------------------------------------------------------
# Isotropic finite differences (Eqs. 35-36) on the D3Q15 stencil
# ----------------------------------------------------------------------------------

def neighbour(chi: np.ndarray, c: Sequence[int], walls_z: bool) -> np.ndarray:
    """chi(x + c) on the grid.  x and y are periodic; z is periodic, or walled with a
    ghost layer equal to the adjacent fluid node."""
    cx, cy, cz = (int(v) for v in c)
    out = np.roll(chi, shift=(-cy, -cx), axis=(-2, -1))
    if cz == 0:
        return out
    if not walls_z:
        return np.roll(out, shift=-cz, axis=-3)
    nz = chi.shape[-3]
    idx = np.clip(np.arange(nz) + cz, 0, nz - 1)
    return np.take(out, idx, axis=-3)


def _stencil_lattice(lattice: str):
    """(velocities, weights, c_s^2) of the lattice whose weights the schemes use: the
    D3Q15 flow lattice (default), or the D3Q7 lattice (weights A/2 with c_s^2 = A; the
    schemes then reduce to 7-point central differences for any A)."""
    if lattice == "d3q15":
        return D3Q15_C, D3Q15_W, D3Q15_CS2
    A = 0.25
    return D3Q7_C, d3q7_weights(A), A


def grad_iso(chi: np.ndarray, walls_z: bool, lattice: str = "d3q15") -> np.ndarray:
    """Eq. 35: grad chi = sum_{i != 0} omega_i c_i chi(x + c_i) / c_s^2."""
    C, W, cs2 = _stencil_lattice(lattice)
    out = np.zeros((3,) + chi.shape)
    for i in range(1, len(C)):
        nb = neighbour(chi, C[i], walls_z)
        for a in range(3):
            if C[i, a]:
                out[a] += W[i] * C[i, a] * nb
    return out / cs2


def lap_iso(chi: np.ndarray, walls_z: bool, lattice: str = "d3q15") -> np.ndarray:
    """Eq. 36: lap chi = sum_{i != 0} 2 omega_i [chi(x + c_i) - chi(x)] / c_s^2."""
    C, W, cs2 = _stencil_lattice(lattice)
    out = np.zeros_like(chi)
    for i in range(1, len(C)):
        out += 2.0 * W[i] * (neighbour(chi, C[i], walls_z) - chi)
    return out / cs2


# ----------------------------------------------------------------------------------
# Macroscopic quantities
# ----------------------------------------------------------------------------------

def order_parameter(f):
    """phi = sum_i f_i (Eq. 13)."""
    return np.sum(f, axis=0)


def density(phi, rho_l, rho_g):
    """rho = (1 + phi)/2 rho_l + (1 - phi)/2 rho_g (Eq. 14)."""
    return 0.5 * (1.0 + phi) * rho_l + 0.5 * (1.0 - phi) * rho_g


def chemical_potential(phi, lap_phi, beta, kappa):
    """mu = 4 beta phi (phi - 1)(phi + 1) - kappa lap phi (Eq. 2; the paper's k is
    called kappa here)."""
    return 4.0 * beta * phi * (phi - 1.0) * (phi + 1.0) - kappa * lap_phi


def velocity(g, rho, Fs, G, lap_mu, rho_l, rho_g, mobility):
    """Eq. 29: u = [sum_i c_i g_i + (F_s + G)/2] / [rho - (rho_l - rho_g) Mob lap mu / 4]."""
    j = np.einsum("ia,i...->a...", D3Q15_C.astype(np.float64), g)
    return (j + 0.5 * (Fs + G)) / (rho - 0.25 * (rho_l - rho_g) * mobility * lap_mu)


def pressure(g, u, grad_rho, rho):
    """Eq. 30: p = c_s^2/(1 - omega_0) [sum_{i != 0} g_i + u . grad rho / 2 + rho s_0(u)]."""
    s0 = d3q15_s(u)[0]
    return D3Q15_CS2 / (1.0 - D3Q15_W[0]) * (
        np.sum(g[1:], axis=0) + 0.5 * np.sum(u * grad_rho, axis=0) + rho * s0)


# ----------------------------------------------------------------------------------
# Collision and propagation
# ----------------------------------------------------------------------------------

def collide_moments(m, meq, rates, msrc):
    """Moment-space form of the collision (Eqs. 15 and 20 premultiplied by the moment
    matrix): m+ = m - S (m - m^eq) + (I - S/2) m_src, S diagonal."""
    return m - rates * (m - meq) + (1.0 - 0.5 * rates) * msrc


def stream(post: np.ndarray, C: np.ndarray, opp: np.ndarray, walls_z: bool) -> np.ndarray:
    """Propagation, Eq. 16, as a pull: f_i(x) = f_i^+(x - c_i).  With walls, a link
    whose source x - c_i lies beyond z = 0 or z = nz is closed by halfway bounce-back:
    f_i(x) = f_{opp(i)}^+(x)."""
    out = np.empty_like(post)
    nz = post.shape[1]
    for i, c in enumerate(C):
        cx, cy, cz = (int(v) for v in c)
        out[i] = np.roll(post[i], shift=(cz, cy, cx), axis=(0, 1, 2))
        if walls_z and cz != 0:
            src_z = np.arange(nz) - cz
            cut = (src_z < 0) | (src_z >= nz)
            out[i][cut] = post[opp[i]][cut]
    return out


# ----------------------------------------------------------------------------------
# Prescribed velocity fields of the interface-tracking tests (Sec. III A, B)
# ----------------------------------------------------------------------------------

def prescribed_velocity(kind: str, U: float, period: float, box, t: float,
                        coords=None) -> np.ndarray:
    """u(x, t) at the nodes x_i = i of a periodic box of size box = (NZ, NY, NX).

    "uniform": u = (U, 0, 0).
    "rotation" (Eq. 37): rigid rotation about the x axis through the box centre,
        v = -Omega (z - N/2), w = Omega (y - N/2), Omega = U pi / N with N = NY (the
        paper's 100^3 case: Omega = U pi / 100, one turn in 200/U steps); `period` unused.
    "deformation" (Eq. 41): with L = NX and the time factor cos(pi t / period),
        u = 2U sin^2(pi x/L) sin(2 pi y/L) sin(2 pi z/L),
        v = -U sin(2 pi x/L) sin^2(pi y/L) sin(2 pi z/L),
        w = -U sin(2 pi x/L) sin(2 pi y/L) sin^2(pi z/L).
    coords: optional (z, y, x) index arrays (broadcastable) of the nodes to evaluate;
    default the whole box.
    """
    NZ, NY, NX = box
    if coords is None:
        z, y, x = np.meshgrid(np.arange(NZ, dtype=np.float64), np.arange(NY, dtype=np.float64),
                              np.arange(NX, dtype=np.float64), indexing="ij")
    else:
        z, y, x = (np.asarray(c, dtype=np.float64) for c in coords)
        z, y, x = np.broadcast_arrays(z, y, x)
    u = np.zeros((3,) + z.shape)
    if kind == "uniform":
        u[0] = U
    elif kind == "rotation":
        omega = U * np.pi / NY
        u[1] = -omega * (z - NY / 2.0)
        u[2] = omega * (y - NY / 2.0)
    elif kind == "deformation":
        L = float(NX)
        a = np.cos(np.pi * t / period)
        sx, sy, sz = np.sin(np.pi * x / L), np.sin(np.pi * y / L), np.sin(np.pi * z / L)
        s2x, s2y, s2z = np.sin(2 * np.pi * x / L), np.sin(2 * np.pi * y / L), np.sin(2 * np.pi * z / L)
        u[0] = 2.0 * U * sx * sx * s2y * s2z * a
        u[1] = -U * s2x * sy * sy * s2z * a
        u[2] = -U * s2x * s2y * sz * sz * a
    else:
        raise ValueError(kind)
    return u


# ----------------------------------------------------------------------------------
# The coupled solver
# ----------------------------------------------------------------------------------

@dataclass
class Params:
    """Physical and lattice parameters (c = dx = dt = 1)."""

    nx: int
    ny: int
    nz: int
    walls_z: bool
    rho_l: float
    rho_g: float
    nu_l: float
    nu_g: float
    mobility: float
    D: float
    sigma: float
    g: Sequence[float]
    A: float = 0.25
    sf: Sequence[float] = (1.0, 1.25, 1.25, 1.25, 1.2, 1.0, 1.0)
    sg: Sequence[float] = (1.0,) * 15
    buoyancy: bool = False
    # interface tracking with a prescribed velocity instead of the flow lattice:
    # None (coupled), ("rotation", U) or ("deformation", U, period_in_steps)
    velocity: Optional[tuple] = None
    # the paper's comparison variants: single-relaxation-time flow lattice (every
    # lambda_k = the viscous rate), and the D3Q7 weights in the schemes of Eqs. 35-36
    srt_flow: bool = False
    stencil: str = "d3q15"

    @property
    def kappa(self):
        """k = 3 D sigma / 8 (text after Eq. 2)."""
        return 3.0 * self.D * self.sigma / 8.0

    @property
    def beta(self):
        """beta = 3 sigma / (4 D) (text after Eq. 2)."""
        return 3.0 * self.sigma / (4.0 * self.D)

    @property
    def eta(self):
        """eta from Mob = eta c_s^2 (tau_f - 1/2), tau_f = 1/s_1 (Eq. 19), c_s^2 = A."""
        return self.mobility / (self.A * (1.0 / self.sf[1] - 0.5))

    def viscous_rate(self, phi):
        """lambda_9..13 = 1/tau_g with nu = c_s^2 (tau_g - 1/2) (Eq. 33) and nu linear in phi."""
        nu = 0.5 * (1.0 + phi) * self.nu_l + 0.5 * (1.0 - phi) * self.nu_g
        return 1.0 / (nu / D3Q15_CS2 + 0.5)

    @classmethod
    def from_workload(cls, w) -> "Params":
        return cls(nx=w.nx, ny=w.ny, nz=w.nz, walls_z=bool(w.walls_z), rho_l=w.rho_l,
                   rho_g=w.rho_g, nu_l=w.nu_l, nu_g=w.nu_g, mobility=w.mobility, D=w.D,
                   sigma=w.sigma, g=tuple(w.g), A=w.A, sf=tuple(w.sf), sg=tuple(w.sg),
                   buoyancy=bool(w.buoyancy), velocity=getattr(w, "velocity", None),
                   srt_flow=bool(getattr(w, "srt_flow", False)),
                   stencil=getattr(w, "stencil", "d3q15"))


class Oracle:
    """The coupled D3Q7 (Cahn-Hilliard) + D3Q15 (Navier-Stokes) MRT scheme.

    State between steps: the populations f (7) and g (15) at time t just after
    propagation, the product phi u of the previous step, and the step count.

    With params.velocity set, only the interface lattice evolves (Eq. 4) and u is the
    prescribed field of Eq. 37 or Eq. 41 (Sec. III A, B); g is not used.
    """

    def __init__(self, params: Params, box=None, coords=None):
        """box, coords: for a patch cut out of a larger grid, the full box size and the
        global (z, y, x) indices of the patch's nodes (used by the prescribed velocity)."""
        if not (params.sf[1] == params.sf[2] == params.sf[3]):
            raise ValueError("Eq. 19 needs s_1 = s_2 = s_3")
        self.p = params
        self.box = box if box is not None else (params.nz, params.ny, params.nx)
        self.coords = coords
        self.f: Optional[np.ndarray] = None
        self.g: Optional[np.ndarray] = None
        self.phiu_prev: Optional[np.ndarray] = None
        self.t = 0

    # -- helpers -----------------------------------------------------------------
    def _force(self, rho):
        gv = np.asarray(self.p.g, dtype=np.float64).reshape((3,) + (1,) * rho.ndim)
        if self.p.buoyancy:
            return (rho - 0.5 * (self.p.rho_l + self.p.rho_g))[None] * gv
        return rho[None] * gv

    def _prescribed(self):
        v = self.p.velocity
        period = v[2] if len(v) > 2 else 1.0
        return prescribed_velocity(v[0], v[1], period, self.box, self.t, self.coords)

    def macroscopic(self):
        """All macroscopic fields at the current time from the current populations."""
        p = self.p
        wz, lat = p.walls_z, p.stencil
        phi = order_parameter(self.f)
        rho = density(phi, p.rho_l, p.rho_g)
        mu = chemical_potential(phi, lap_iso(phi, wz, lat), p.beta, p.kappa)
        if p.velocity is not None:
            return dict(phi=phi, rho=rho, mu=mu, u=self._prescribed(), p=np.zeros_like(phi))
        grad_phi = grad_iso(phi, wz, lat)
        grad_rho = grad_iso(rho, wz, lat)
        lap_mu = lap_iso(mu, wz, lat)
        Fs = mu[None] * grad_phi
        G = self._force(rho)
        u = velocity(self.g, rho, Fs, G, lap_mu, p.rho_l, p.rho_g, p.mobility)
        pr = pressure(self.g, u, grad_rho, rho)
        Fa = 0.5 * (p.rho_l - p.rho_g) * p.mobility * lap_mu[None] * u
        return dict(phi=phi, rho=rho, mu=mu, grad_phi=grad_phi, grad_rho=grad_rho,
                    lap_mu=lap_mu, Fs=Fs, G=G, Fa=Fa, F=Fs + Fa + G, u=u, p=pr)

    # -- public ------------------------------------------------------------------
    def init(self, phi0, u0=None, p0=None):
        """Populations at their equilibria (Eqs. 5 and 21) for the given phi0, u0, p0."""
        p = self.p
        shape = (p.nz, p.ny, p.nx)
        phi0 = np.asarray(phi0, dtype=np.float64).reshape(shape)
        u0 = np.zeros((3,) + shape) if u0 is None else np.asarray(u0, np.float64).reshape((3,) + shape)
        p0 = np.zeros(shape) if p0 is None else np.asarray(p0, np.float64).reshape(shape)
        mu0 = chemical_potential(phi0, lap_iso(phi0, p.walls_z, p.stencil), p.beta, p.kappa)
        rho0 = density(phi0, p.rho_l, p.rho_g)
        self.t = 0
        if p.velocity is not None:
            u0 = self._prescribed()
        self.f = d3q7_feq(phi0, mu0, u0, p.eta, p.A)
        self.g = d3q15_geq(p0, rho0, u0)
        self.phiu_prev = None

    def step(self, n: int = 1):
        for _ in range(n):
            self._step()

    def _step(self):
        p = self.p
        mac = self.macroscopic()
        phi, rho, u = mac["phi"], mac["rho"], mac["u"]

        # Flow lattice: collision in moment space (Eqs. 20, 27, 31, 32).
        g_post = None
        if p.velocity is None:
            rates_g = np.broadcast_to(np.asarray(p.sg, np.float64).reshape(15, 1, 1, 1),
                                      (15,) + phi.shape).copy()
            if p.srt_flow:
                rates_g[:] = p.viscous_rate(phi)[None]
            else:
                rates_g[9:14] = p.viscous_rate(phi)[None]
            mg = to_moments(GAMMA, self.g)
            mg_post = collide_moments(mg, d3q15_mgeq(mac["p"], rho, u), rates_g,
                                      d3q15_mT(u, mac["grad_rho"], mac["F"]))
            g_post = to_moments(GAMMA_INV, mg_post)

        # Interface lattice: backward time difference (Eq. 34), collision (Eqs. 15-18).
        phiu = phi[None] * u
        dt_phiu = np.zeros_like(phiu) if self.phiu_prev is None else phiu - self.phiu_prev
        self.phiu_prev = phiu
        rates_f = np.asarray(p.sf, np.float64).reshape(7, 1, 1, 1)
        mf = to_moments(M7, self.f)
        mf_post = collide_moments(mf, d3q7_mfeq(phi, mac["mu"], u, p.eta, p.A), rates_f,
                                  d3q7_mR(dt_phiu))
        f_post = to_moments(M7_INV, mf_post)

        # Propagation (Eq. 16).
        self.f = stream(f_post, D3Q7_C, OPP7, p.walls_z)
        if g_post is not None:
            self.g = stream(g_post, D3Q15_C, OPP15, p.walls_z)
        self.t += 1

    def fields(self):
        """phi, rho, p, u, mu at the current time."""
        mac = self.macroscopic()
        return {k: mac[k] for k in ("phi", "rho", "p", "u", "mu")}

    def totals(self):
        """sum_x phi and sum_x sum_i c_i g_i over the grid (pre-collision populations)."""
        j = np.einsum("ia,i...->a...", D3Q15_C.astype(np.float64), self.g)
        return float(np.sum(order_parameter(self.f))), j.reshape(3, -1).sum(axis=1)
