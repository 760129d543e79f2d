"""FP64 CPU oracle of the 3D MRT lattice Boltzmann multiphase model.

Test infrastructure only: imported by the tests, the package smoke check and the
benchmark's CPU-baseline leg, never by the product path.
"""
