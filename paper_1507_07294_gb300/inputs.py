"""Seeded synthetic workloads for the 3D MRT lattice Boltzmann multiphase model.

This module builds what both the CUDA path and the FP64 oracle take as input: the
grid, the physical parameters of each test problem of the paper (Sec. III), and the
initial fields.  It holds none of the method's arithmetic -- no equilibria, moments,
stencils or collisions.  The only formulas here are the problem statements:

* the static droplet phi = tanh(2(R - r)/D) (interface profile of Eq. 43 around a sphere);
* the Rayleigh-Taylor interface h(x, y) of Eq. 42 and phi0 of Eq. 43;
* the dimensionless groups that fix nu and the mobility: Re (Eq. 44) and the Peclet
  number Pe = sqrt(gW) W / Mob for the Rayleigh-Taylor runs, Pe = U L / Mob (Eq. 39)
  for interface-tracking runs.

Node coordinates: along a periodic axis node i sits at i; along a walled z axis node k
sits at k + 1/2, with the walls at z = 0 and z = nz.

Arrays are float64, indexed [z, y, x] (x fastest), vectors as [3, z, y, x].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional, Tuple

import numpy as np

# Relaxation matrix of the order-parameter lattice used in the coupled runs (Eq. 45).
SF_COUPLED = (1.0, 1.25, 1.25, 1.25, 1.2, 1.0, 1.0)
# Relaxation matrix of the interface-tracking runs (Eq. 38).
SF_TRACKING = (1.0, 4.0 / 3.0, 4.0 / 3.0, 4.0 / 3.0, 1.2, 1.2, 1.2)
# Flow-lattice rates: all unity; the five viscous rates are set from nu(phi) by the solver.
SG_UNITY = (1.0,) * 15


@dataclass
class Workload:
    """One problem: grid, parameters and initial condition."""

    name: str
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
    g: Tuple[float, float, float]
    A: float = 0.25
    sf: Tuple[float, ...] = SF_COUPLED
    sg: Tuple[float, ...] = SG_UNITY
    buoyancy: bool = False
    steps: int = 100
    U: float = 1.0  # velocity scale used to normalise velocity errors
    # interface tracking with a prescribed velocity (no flow lattice):
    # None, ("uniform", U), ("rotation", U) or ("deformation", U, period_in_steps)
    velocity: Optional[tuple] = None
    # the paper's comparison variants (Sec. III A): SRT flow lattice; D3Q7 stencils
    srt_flow: bool = False
    stencil: str = "d3q15"
    phi0: Optional[np.ndarray] = field(default=None, repr=False)
    u0: Optional[np.ndarray] = field(default=None, repr=False)
    p0: Optional[np.ndarray] = field(default=None, repr=False)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


def node_coords(nx: int, ny: int, nz: int, walls_z: bool):
    """Broadcastable (z, y, x) node coordinates following the convention above."""
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    if walls_z:
        z = z + 0.5
    return x, y, z


def droplet(n: int = 32, R: float = 8.0, D: float = 4.0, sigma: float = 0.01,
            rho_l: float = 3.0, rho_g: float = 1.0, nu: float = 0.1,
            mobility: float = 0.1, steps: int = 500, nx: Optional[int] = None,
            ny: Optional[int] = None, nz: Optional[int] = None) -> Workload:
    """Static droplet of radius R centred in a periodic box; phi = +1 (rho_l) inside."""
    nx = n if nx is None else nx
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    x, y, z = node_coords(nx, ny, nz, False)
    r = np.sqrt((x - nx / 2) ** 2 + (y - ny / 2) ** 2 + (z - nz / 2) ** 2)
    phi0 = np.tanh(2.0 * (R - r) / D)
    return Workload(name=f"droplet{nx}x{ny}x{nz}_R{R:g}", nx=nx, ny=ny, nz=nz,
                    walls_z=False, rho_l=rho_l, rho_g=rho_g, nu_l=nu, nu_g=nu,
                    mobility=mobility, D=D, sigma=sigma, g=(0.0, 0.0, 0.0),
                    sf=SF_COUPLED, steps=steps, U=sigma / (rho_l * nu), phi0=phi0)


def rayleigh_taylor(W: int = 64, Re: float = 256.0, atwood: float = 0.5,
                    sqrt_gW: float = 0.04, D: float = 4.0, sigma: float = 1e-4,
                    Pe: float = 50.0, rho_g: float = 1.0, steps: int = 20000,
                    nz: Optional[int] = None, with_fields: bool = True) -> Workload:
    """Rayleigh-Taylor box W x W x 4W: heavy fluid (phi = +1) above z = 2W + h(x, y).

    Eq. 42 gives h, Eq. 43 phi0 and Eq. 44 Re = sqrt(gW) W / nu; the mobility follows
    from Pe = sqrt(gW) W / Mob.  Lateral boundaries periodic, z walled.  With
    with_fields False phi0 is left None (it depends on W, nz and D only; callers that
    make many runs of one grid build it once with rt_interface).
    """
    nz = 4 * W if nz is None else nz
    rho_l = rho_g * (1.0 + atwood) / (1.0 - atwood)
    gacc = sqrt_gW ** 2 / W
    nu = sqrt_gW * W / Re
    mob = sqrt_gW * W / Pe
    phi0 = rt_interface(W, nz, D) if with_fields else None
    return Workload(name=f"rt{W}x{W}x{nz}_Re{Re:g}", nx=W, ny=W, nz=nz, walls_z=True,
                    rho_l=rho_l, rho_g=rho_g, nu_l=nu, nu_g=nu, mobility=mob, D=D,
                    sigma=sigma, g=(0.0, 0.0, -gacc), sf=SF_COUPLED, steps=steps,
                    U=sqrt_gW, phi0=phi0)


def rt_interface(W: int, nz: int, D: float = 4.0) -> np.ndarray:
    """phi0 of Eq. 43 around the perturbed plane z = nz/2 + h(x, y) of Eq. 42."""
    x, y, z = node_coords(W, W, nz, True)
    h = 0.05 * W * (np.cos(2 * math.pi * x / W) + np.cos(2 * math.pi * y / W))
    phi0 = np.tanh(2.0 * (z - h - nz / 2.0) / D)
    return np.broadcast_to(phi0, (nz, W, W)).copy()


def flat_interface(nz: int = 32, nxy: int = 4, D: float = 4.0, sigma: float = 0.01,
                   rho_l: float = 3.0, rho_g: float = 1.0, nu: float = 0.1,
                   mobility: float = 0.1, steps: int = 2000) -> Workload:
    """Planar interface phi = tanh(2(z - nz/2)/D) between two z walls, no gravity."""
    x, y, z = node_coords(nxy, nxy, nz, True)
    phi0 = np.broadcast_to(np.tanh(2.0 * (z - nz / 2.0) / D), (nz, nxy, nxy)).copy()
    return Workload(name=f"flat{nxy}x{nxy}x{nz}", nx=nxy, ny=nxy, nz=nz, walls_z=True,
                    rho_l=rho_l, rho_g=rho_g, nu_l=nu, nu_g=nu, mobility=mobility, D=D,
                    sigma=sigma, g=(0.0, 0.0, 0.0), sf=SF_COUPLED, steps=steps,
                    U=sigma / (rho_l * nu), phi0=phi0)


def deformation(n: int = 128, U: float = 0.02, period: float = 3000.0, D: float = 2.0,
                sigma: float = 0.04, Pe: float = 400.0) -> Workload:
    """Deformation-flow test (Sec. III B, Eq. 41) scaled to an n^3 periodic box: sphere of
    radius 0.15 n centred at 0.35 n in each axis (15 and 35 in the paper's 100^3 box),
    velocity amplitude U, time factor cos(pi t / period) with t in steps; the mobility
    from Pe = U R / Mob (Eq. 39 with L = R); S^f of Eq. 38."""
    R = 0.15 * n
    c = 0.35 * n
    x, y, z = node_coords(n, n, n, False)
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    phi0 = np.tanh(2.0 * (R - r) / D)
    return Workload(name=f"deformation{n}", nx=n, ny=n, nz=n, walls_z=False, rho_l=1.0,
                    rho_g=1.0, nu_l=0.1, nu_g=0.1, mobility=U * R / Pe, D=D, sigma=sigma,
                    g=(0.0, 0.0, 0.0), sf=SF_TRACKING, steps=int(period), U=2.0 * U,
                    velocity=("deformation", U, float(period)), phi0=phi0)


def zalesak(n: int = 100, U: float = 0.02, D: float = 2.0, sigma: float = 0.04,
            Pe: float = 200.0, slot_depth: Optional[float] = None) -> Workload:
    """Zalesak's slotted sphere (Sec. III A, Eq. 37) scaled to an n^3 periodic box: radius
    0.4 n at the centre (40 of 100), a slot of width 0.16 n (16 of 100) along x cut from
    the bottom of the sphere, depth `slot_depth` (the paper gives none; default R, up to
    the centre).  Rigid rotation about the x axis, one turn in 2n/U steps; Pe = U R / Mob."""
    R = 0.4 * n
    half_w = 0.08 * n
    depth = R if slot_depth is None else slot_depth
    c = n / 2.0
    x, y, z = node_coords(n, n, n, False)
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    # signed distance to the slot box {|y - c| <= half_w, z <= c - R + depth} (outside > 0)
    qy = np.abs(y - c) - half_w
    qz = z - (c - R + depth)
    qy, qz = np.broadcast_arrays(qy, qz)
    outside = np.sqrt(np.maximum(qy, 0) ** 2 + np.maximum(qz, 0) ** 2)
    inside = np.minimum(np.maximum(qy, qz), 0.0)
    d_slot = np.broadcast_to(outside + inside, (n, n, n))
    d = np.minimum(R - r, d_slot)
    phi0 = np.tanh(2.0 * d / D)
    return Workload(name=f"zalesak{n}", nx=n, ny=n, nz=n, walls_z=False, rho_l=1.0, rho_g=1.0,
                    nu_l=0.1, nu_g=0.1, mobility=U * R / Pe, D=D, sigma=sigma,
                    g=(0.0, 0.0, 0.0), sf=SF_TRACKING, steps=int(round(2 * n / U)), U=U,
                    velocity=("rotation", U), phi0=np.ascontiguousarray(phi0))


def translating_slab(n: int = 64, U: float = 0.02, D: float = 2.0, sigma: float = 0.04,
                     mobility: float = 0.02) -> Workload:
    """A slab phi = +1 for n/4 < x < 3n/4 (two tanh interfaces) in a periodic n x 1 x 1
    box, carried by the uniform velocity (U, 0, 0)."""
    x = np.arange(n, dtype=np.float64)
    phi = np.tanh(2.0 * (x - n / 4) / D) - np.tanh(2.0 * (x - 3 * n / 4) / D) - 1.0
    return Workload(name=f"slab{n}", nx=n, ny=1, nz=1, walls_z=False, rho_l=1.0, rho_g=1.0,
                    nu_l=0.1, nu_g=0.1, mobility=mobility, D=D, sigma=sigma,
                    g=(0.0, 0.0, 0.0), sf=SF_TRACKING, steps=int(round(n / U)), U=U,
                    velocity=("uniform", U), phi0=phi.reshape(1, 1, n))


def perturbed(w: Workload, seed: int = 0, phi_amp: float = 0.0, u_amp: float = 0.0,
              p_amp: float = 0.0) -> Workload:
    """Copy of `w` with seeded random perturbations of phi0, u0 and p0.

    Parity runs use this so that every term of the update (velocity-dependent
    equilibria and sources, pressure) is exercised from the first step.  The phi
    perturbation is kept inside [-1, 1].
    """
    rng = np.random.default_rng(seed)
    phi0 = w.phi0.copy()
    if phi_amp:
        phi0 = np.clip(phi0 + phi_amp * rng.uniform(-1, 1, phi0.shape), -1.0, 1.0)
    u0 = None if not u_amp else u_amp * rng.uniform(-1, 1, (3,) + w.shape)
    p0 = None if not p_amp else p_amp * rng.uniform(-1, 1, w.shape)
    return replace(w, name=w.name + f"_pert{seed}", phi0=phi0, u0=u0, p0=p0)


def random_fields(shape, seed: int = 0, scale: float = 1.0) -> np.ndarray:
    """Uniform(-scale, scale) float64 array, seeded."""
    return scale * np.random.default_rng(seed).uniform(-1.0, 1.0, shape)
