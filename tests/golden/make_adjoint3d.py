"""Writes adjoint3d_sphere.txt: the oracle's frozen-turbulence adjoint of a
3D case (a sphere placed off the grid's symmetry planes in a 16 x 8 x 8
channel, laminar, Re 20): J (pressure drop) and dJ/dlambda at the oracle's
converged state.  Calls only oracle/ (and the seeded geometry); the GPU
parity test of the 3D adjoint compares against it.

    python tests/golden/make_adjoint3d.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2606_06135_gb300 import geometry as G  # noqa: E402
from oracle import adjoint as A  # noqa: E402
from oracle import hfdib_oracle as O  # noqa: E402


def sphere_off_axis():
    case = G.case_sphere(16, 8, 8, model="laminar", Re=20.0)
    X, Y, Z = G.cell_centres(case["grid"])
    sig = np.sqrt((X - 4.3) ** 2 + (Y - 3.7) ** 2 + (Z - 4.2) ** 2) - 1.4
    case["sigma"] = sig
    case["lam"] = G.lambda_from_sigma(sig, O.Mesh(case["grid"]).h)
    case["ywall"] = np.maximum(sig, 0.0)
    return case


def main():
    case = sphere_off_axis()
    o = O.Oracle(case)
    it, res = o.solve(tol=1e-13, max_iter=4000)
    assert o.max_residual(res) <= 1e-13
    fs = A.FrozenSteady(o)
    assert fs.n_kinks == 0
    J, g, _ = fs.gradient()
    # text: J on the first line, then dJ/dlambda in cell order (x fastest)
    vals = np.concatenate([[J], np.asarray(g).ravel()])
    np.savetxt(os.path.join(HERE, "adjoint3d_sphere.txt"), vals, fmt="%.17e",
               header="oracle adjoint of the off-axis sphere: J, then dJ/dlambda (16 x 8 x 8, x fastest)")
    print("J = %.15f, |grad| = %.6e" % (J, np.linalg.norm(g)))


if __name__ == "__main__":
    main()
