"""FP64 CPU oracle of the phase-field WMRT lattice Boltzmann step.

Test infrastructure only: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the product library.
"""
