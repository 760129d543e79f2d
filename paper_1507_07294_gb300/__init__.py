"""GB300 (sm_103a) implementation of the 3D MRT lattice Boltzmann multiphase model of
Liang, Shi & Chai (arXiv:1507.07294): a D3Q7 Cahn-Hilliard lattice coupled to a D3Q15
Navier-Stokes lattice, stepped by hand-written CUDA kernels behind a C ABI
(include/lbm.h).

Submodules:
    lbm      ctypes binding of liblbm.so (the C entry points, one to one) and Solver
    inputs   seeded synthetic workloads (grids, parameters, initial fields)
    _build   nvcc build of liblbm.so

The binding is imported lazily so that `inputs` can be used without CUDA.
"""

__all__ = ["lbm", "inputs"]


def __getattr__(name):
    if name in ("lbm", "inputs", "_build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
