"""Seeded synthetic workloads (meshes, wavenumbers, tree depths, right-hand
sides) shared by the CPU oracle, the tests and the benchmark.  This package
holds no electromagnetic or fast-multipole arithmetic."""
from .meshes import icosphere, plate_with_strips, plate, cube, two_triangle_pairs  # noqa: F401
from .configs import WORKLOADS, Workload, get, rhs, rhs_complex  # noqa: F401
