"""Named workloads.  Each one fixes a mesh recipe, the wavenumber, the number
of tree levels (level 0 included, the convention of Table II's ``nlv``), the
digits of accuracy d0 in the excess-bandwidth formula for the truncation
number (Section V), the number of right-hand sides B and a seed.

Right-hand sides are real N(0, 1) columns drawn from NumPy's PCG64 generator,
float64, shape [N, B] with B innermost; a run at reduced precision casts them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Tuple

import numpy as np

from . import meshes


@dataclass(frozen=True)
class Workload:
    name: str
    mesh: Callable[[], Tuple[np.ndarray, np.ndarray]]
    k: float                 # free-space wavenumber, rad/m
    levels: int              # oct-tree levels including level 0
    digits: float            # d0
    batch: int               # right-hand sides per pass
    seed: int
    note: str = ""
    n_expected: int = field(default=0)


TWO_PI = 2.0 * math.pi

WORKLOADS = {
    # 1,280 triangles / 1,920 RWG, three levels (two-level FMM at level 2)
    "sphere-r0.5m-ico3": Workload("sphere-r0.5m-ico3", lambda: meshes.icosphere(3, 0.5),
                                  TWO_PI, 3, 3.0, 8, 1412175601,
                                  "PEC sphere r=0.5 m, wavelength 1 m", 1920),
    # 20,480 triangles / 30,720 RWG, five levels
    "sphere-r2m-ico5": Workload("sphere-r2m-ico5", lambda: meshes.icosphere(5, 2.0),
                                TWO_PI, 5, 3.0, 1, 1412175602,
                                "PEC sphere r=2 m, wavelength 1 m", 30720),
    # 6 m plate (7,200 triangles) plus 16 strips: 10,824 RWG
    "plate6m-strips": Workload("plate6m-strips", lambda: meshes.plate_with_strips(),
                               TWO_PI, 5, 3.0, 16, 1412175603,
                               "6x6 m plate + 4x4 strip array, wavelength 1 m", 10824),
    # 76,800 triangles / 115,200 RWG, seven levels
    "cube8m": Workload("cube8m", lambda: meshes.cube(8.0, 80), TWO_PI, 7, 3.0, 64, 1412175604,
                       "PEC cube side 8 m, wavelength 1 m", 115200),
    # the same cube with 6 levels (0.25 wavelength leaves, inside the paper's
    # 0.2-0.5 wavelength range) and d0 = 5
    "cube8m-6lv": Workload("cube8m-6lv", lambda: meshes.cube(8.0, 80), TWO_PI, 6, 5.0, 64, 1412175604,
                           "PEC cube side 8 m, 6 levels", 115200),
    # 1,310,720 triangles / 1,966,080 RWG, nine levels
    "sphere-r8m-ico8": Workload("sphere-r8m-ico8", lambda: meshes.icosphere(8, 8.0),
                                TWO_PI, 9, 3.0, 16, 1412175605,
                                "PEC sphere r=8 m, wavelength 1 m", 1966080),
    # the same sphere with 8 levels (0.125 wavelength leaves): the depth at
    # which Eq. (9) with d0 = 3 still delivers about 3 digits
    "sphere-r8m-ico8-8lv": Workload("sphere-r8m-ico8-8lv", lambda: meshes.icosphere(8, 8.0),
                                    TWO_PI, 8, 3.0, 16, 1412175605,
                                    "PEC sphere r=8 m, 8 levels", 1966080),
    # small sphere for fast tests: 320 triangles / 480 RWG
    "sphere-r0.5m-ico2": Workload("sphere-r0.5m-ico2", lambda: meshes.icosphere(2, 0.5),
                                  TWO_PI, 3, 3.0, 4, 1412175606,
                                  "PEC sphere r=0.5 m, coarse mesh", 480),
}


def get(name: str) -> Workload:
    return WORKLOADS[name]


def rhs(n: int, batch: int, seed: int) -> np.ndarray:
    """Real N(0, 1) right-hand sides, float64 [n, batch]."""
    g = np.random.Generator(np.random.PCG64(seed))
    return g.standard_normal((n, batch))


def rhs_complex(n: int, batch: int, seed: int) -> np.ndarray:
    """Complex right-hand sides with N(0, 1) real and imaginary parts."""
    g = np.random.Generator(np.random.PCG64(seed))
    return g.standard_normal((n, batch)) + 1j * g.standard_normal((n, batch))
