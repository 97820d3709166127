"""Writes sphere_30720_cm_values.txt: the 24 characteristic values nearest
zero (Section II, Eq. (GEP), with R = -Re Z and X = Im Z) of the oracle's
dense FP64 Galerkin EFIE matrix for the 30,720-unknown sphere (icosphere
subdivision 5, radius 2 m, k = 2 pi), by oracle.cm.cm_values_symmetric (one
dense symmetric eigenproblem, no iteration).  Calls only the oracle and the
mesh generator.  Needs ~32 GB of host memory; ~40 minutes on 8 cores.

    python tests/golden/make_sphere_30720_cm.py
"""
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads  # noqa: E402
from oracle import cm, efie  # noqa: E402

NEV = 24


def main():
    v, t = workloads.icosphere(5, 2.0)
    t0 = time.time()
    Z = efie.Problem(v, t, 2 * math.pi).dense()
    t_fill = time.time() - t0
    R = -Z.real
    X = Z.imag.copy()
    del Z
    t0 = time.time()
    lam = cm.cm_values_symmetric(R, X, NEV, overwrite=True)
    t_eig = time.time() - t0
    with open(os.path.join(HERE, "sphere_30720_cm_values.txt"), "w") as f:
        f.write("# The %d characteristic values nearest zero, sorted by magnitude, of X J = lambda R J\n" % NEV)
        f.write("# (Section II, Eq. (GEP); R = -Re Z, X = Im Z) for the oracle's dense FP64 Galerkin EFIE\n")
        f.write("# matrix of the sphere r = 2 m, icosphere subdivision 5 (30,720 RWG unknowns), k = 2 pi.\n")
        f.write("# Written by tests/golden/make_sphere_30720_cm.py (oracle.cm.cm_values_symmetric);\n")
        f.write("# dense fill %.0f s, eigensolve %.0f s.\n" % (t_fill, t_eig))
        for x in lam:
            f.write("%.12e\n" % x)
    print(lam)


if __name__ == "__main__":
    main()
