"""Writes the oracle's frozen-turbulence adjoints of 3D cases, each file J
on the first line and then dJ/dlambda in cell order (x fastest), at the
oracle's converged state:

* adjoint3d_sphere.txt: a sphere placed off the grid's symmetry planes in a
  16 x 8 x 8 channel, laminar, Re 20, pressure drop;
* adjoint3d_sphere_drag.txt: the same state, drag objective;
* adjoint3d_sphere_keps_drag.txt: the same geometry with k-epsilon at Re
  200 (nu_t frozen at the converged state), drag objective.

Calls only oracle/ (and the seeded geometry); the GPU parity tests of the 3D
adjoint compare against them.

    python tests/golden/make_adjoint3d.py [which ...]   (default: all)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2606_06135_gb300 import geometry as G  # noqa: E402
from oracle import adjoint as A  # noqa: E402
from oracle import hfdib_oracle as O  # noqa: E402


def sphere_off_axis(model="laminar", Re=20.0):
    case = G.case_sphere(16, 8, 8, model=model, Re=Re)
    X, Y, Z = G.cell_centres(case["grid"])
    sig = np.sqrt((X - 4.3) ** 2 + (Y - 3.7) ** 2 + (Z - 4.2) ** 2) - 1.4
    case["sigma"] = sig
    case["lam"] = G.lambda_from_sigma(sig, O.Mesh(case["grid"]).h)
    case["ywall"] = np.maximum(sig, 0.0)
    return case


GOLDENS = {
    "adjoint3d_sphere.txt": ("laminar", 20.0, "pressure_drop"),
    "adjoint3d_sphere_drag.txt": ("laminar", 20.0, "drag"),
    "adjoint3d_sphere_keps_drag.txt": ("kepsilon", 200.0, "drag"),
}


def write(name):
    model, Re, objective = GOLDENS[name]
    case = sphere_off_axis(model, Re)
    o = O.Oracle(case)
    it, res = o.solve(tol=1e-13, max_iter=6000)
    assert o.max_residual(res) <= 1e-13, (it, res)
    fs = A.FrozenSteady(o, objective)
    assert fs.n_kinks == 0
    J, g, _ = fs.gradient()
    vals = np.concatenate([[J], np.asarray(g).ravel()])
    np.savetxt(os.path.join(HERE, name), vals, fmt="%.17e",
               header="oracle adjoint of the off-axis sphere (%s, Re %g, %s): J, then dJ/dlambda "
                      "(16 x 8 x 8, x fastest)" % (model, Re, objective))
    print("%s: J = %.15f, |grad| = %.6e, %d sweeps" % (name, J, np.linalg.norm(g), it))


def main():
    for name in (sys.argv[1:] or list(GOLDENS)):
        write(name)


if __name__ == "__main__":
    main()
