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
