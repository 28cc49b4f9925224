"""Symmetries of the oracle's 3D sweep.

A sphere at the centre of the y-z cross-section of a box with equal y and z
sides and cubic cells: swapping the y and z axes maps the problem onto
itself (lambda, y_wall and the boundary conditions; v and w trade places),
and so do the reflections y -> L_y - y and z -> L_z - z (v, respectively w,
change sign). The oracle's inner solves are exact, so every sweep commutes
with these maps, and the iterates keep the symmetry to rounding from the
uniform start. A y/z-asymmetric mistake anywhere in the 3D path -- an index
of the wrong axis, a face area or a distance of the wrong direction, a
term dropped for one direction -- breaks one of them.

(An extruded 2D body is not such a pin: in 3D the momentum diagonal holds
the z-diffusion coefficients, which enter the under-relaxation and rAU and
through rAU the Rhie-Chow flux, so the extruded problem is a slightly
different discrete problem from the 2D one.)
"""
import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O


def swap_yz(f):
    """f[k, j, i] -> f[j, k, i]."""
    return np.transpose(np.asarray(f), (1, 0, 2))


def _sphere(model, sweeps):
    case = G.case_sphere(16, 8, 8, model=model)
    g = case["grid"]
    assert g["ny"] == g["nz"] and g["dy"] == g["dz"]
    o = O.Oracle(case)
    for _ in range(sweeps):
        o.sweep()
    return o


def _scale(f):
    return max(1.0, float(np.abs(f).max()))


@pytest.mark.parametrize("model", ["kepsilon", "komegasst"])
def test_sphere_sweeps_keep_the_y_z_swap(model):
    o = _sphere(model, 20)
    tol = 1e-13
    u, v, w = o.u
    assert np.abs(u - swap_yz(u)).max() <= tol * _scale(u)
    assert np.abs(v - swap_yz(w)).max() <= tol * _scale(v)
    assert np.abs(o.p - swap_yz(o.p)).max() <= tol * _scale(o.p)
    for name in ("k", "eps", "omega", "nut"):
        f = getattr(o, name)
        assert np.abs(f - swap_yz(f)).max() <= tol * _scale(f), name
    # the flow around the sphere is three-dimensional, not trivially so
    assert np.abs(v).max() > 1e-3 and np.abs(w).max() > 1e-3


def test_sphere_sweeps_keep_the_reflections():
    o = _sphere("kepsilon", 20)
    tol = 1e-13
    u, v, w = o.u
    for ax, odd in ((1, v), (0, w)):          # y is axis 1, z axis 0 of [nz, ny, nx]
        flip = lambda f: np.flip(f, axis=ax)
        assert np.abs(u - flip(u)).max() <= tol * _scale(u)
        assert np.abs(odd + flip(odd)).max() <= tol * _scale(odd)
        assert np.abs(o.p - flip(o.p)).max() <= tol * _scale(o.p)
        assert np.abs(o.k - flip(o.k)).max() <= tol * _scale(o.k)


def test_y_z_swap_pin_catches_a_one_direction_mistake(monkeypatch):
    """A mistake planted in the oracle on one axis only -- the z-face
    diffusion distance scaled by 1 + 1e-3 -- breaks the swap."""
    orig = O.Oracle.__init__

    def planted(self, case, opts=None):
        orig(self, case, opts)
        self.m.D = list(self.m.D)
        self.m.D[2] = self.m.D[2] * (1.0 + 1e-3)

    monkeypatch.setattr(O.Oracle, "__init__", planted)
    o = _sphere("laminar", 10)
    u, v, w = o.u
    err = max(np.abs(u - swap_yz(u)).max(), np.abs(v - swap_yz(w)).max())
    assert err > 1e-7
