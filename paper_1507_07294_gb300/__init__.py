"""GB300 (sm_103a) implementation of the 3D MRT lattice Boltzmann multiphase model of
Liang, Shi & Chai (arXiv:1507.07294): a D3Q7 Cahn-Hilliard lattice coupled to a D3Q15
Navier-Stokes lattice, stepped by hand-written CUDA kernels behind a C ABI
(include/lbm.h).

Submodules:
    lbm          ctypes binding of liblbm.so (the C entry points, one to one), Solver,
                 Batch
    serve        continuous-batching request loop over many runs
    tune         autotuning of the single-run prefetch distances
    inputs       seeded synthetic workloads (grids, parameters, initial fields)
    diagnostics  host-side measures of results (Err of Eq. 40, interface fronts)
    _build       nvcc build of liblbm.so

Submodules are imported lazily so that `inputs` and `diagnostics` can be used without
CUDA.
"""

__all__ = ["lbm", "serve", "tune", "inputs", "diagnostics"]


def __getattr__(name):
    if name in ("lbm", "serve", "tune", "inputs", "diagnostics", "_build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
