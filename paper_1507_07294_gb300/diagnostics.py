"""Host-side diagnostics of simulation results (no part of the time step)."""
import numpy as np


def relative_error(phi_T, phi_0) -> float:
    """Global relative error of the order parameter, Eq. 40:
    Err = sum_x |phi(x, T) - phi(x, 0)| / sum_x |phi(x, 0)|."""
    phi_T = np.asarray(phi_T, dtype=np.float64)
    phi_0 = np.asarray(phi_0, dtype=np.float64)
    return float(np.abs(phi_T - phi_0).sum() / np.abs(phi_0).sum())


def interface_crossings(profile, coords):
    """Positions where a 1D profile changes sign, by linear interpolation."""
    p = np.asarray(profile, dtype=np.float64)
    c = np.asarray(coords, dtype=np.float64)
    k = np.flatnonzero(np.sign(p[:-1]) * np.sign(p[1:]) < 0)
    return c[k] - p[k] * (c[k + 1] - c[k]) / (p[k + 1] - p[k])


def rt_fronts(phi, W: int):
    """Bubble front and spike tip of a Rayleigh-Taylor run (heavy fluid, phi > 0, above
    the plane z = nz/2 + h(x, y) of Eq. 42), in units of W from the initial mean
    interface: the highest phi = 0 crossing along the column x = y = 0 (where h is
    largest: the light fluid rises there) and the lowest along x = y = W/2.  phi is
    indexed [z, y, x] with walls in z (node k at k + 1/2)."""
    phi = np.asarray(phi, dtype=np.float64)
    nz = phi.shape[0]
    z = np.arange(nz) + 0.5
    bubble = interface_crossings(phi[:, 0, 0], z).max()
    spike = interface_crossings(phi[:, W // 2, W // 2], z).min()
    return (bubble - nz / 2) / W, (spike - nz / 2) / W
