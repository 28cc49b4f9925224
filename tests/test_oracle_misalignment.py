"""Misalignment of the immersed body with the mesh faces (App. C), on the
oracle.

A rectangle at zero angle of attack, rotated with its inflow by beta, in a
square domain with the inflow through x- and y- and the outflow through x+
and y+. Mirroring about the diagonal maps the problem at beta onto the
problem at 90 - beta: lambda, y_wall and the boundary conditions map exactly
(up to the rounding of cos and sin), and (u, v) maps to (v, u). On a square
grid of square cells every step of a sweep (the groups and interpolation of
the IB cells, the momentum and turbulence rows, the pressure equation, the
flux correction) treats x and y alike, so each sweep maps one problem's
iterate onto the other's. A transposed index, a dropped or wrong-signed term
in one direction only, or an x-first tie in the IB geometry breaks that.
"""
import math

import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O


def mirrored(f):
    """f of one 2D problem as the other problem sees it: transpose [ny, nx]."""
    return np.asarray(f)[0].T


def test_geometry_of_beta_mirrors_that_of_90_minus_beta():
    a = G.case_misaligned_box(30.0, 32, L=4.0)
    b = G.case_misaligned_box(60.0, 32, L=4.0)
    np.testing.assert_allclose(a["lam"][0], mirrored(b["lam"]), rtol=0, atol=1e-14)
    np.testing.assert_allclose(a["ywall"][0], mirrored(b["ywall"]), rtol=0, atol=1e-14)
    assert a["bc"]["xmin"] == b["bc"]["ymin"] == "inlet"
    assert a["bc"]["xmax"] == b["bc"]["ymax"] == "outlet"
    assert a["u_in"][0] == pytest.approx(b["u_in"][1], abs=1e-15)
    assert a["u_in"][1] == pytest.approx(b["u_in"][0], abs=1e-15)
    # the body: its area 1 x 0.25 whatever the angle (lambda sums to the
    # solid area in units of the cell area up to the smoothing of the band)
    for beta in (0.0, 15.0, 30.0, 45.0):
        c = G.case_misaligned_box(beta, 64, L=4.0)
        area = c["lam"].sum() * c["grid"]["dx"] * c["grid"]["dy"]
        assert area == pytest.approx(0.25, rel=0.03), (beta, area)
        # the inflow at unit speed along the body's long axis
        assert math.hypot(c["u_in"][0], c["u_in"][1]) == pytest.approx(1.0, abs=1e-15)


def _pair(model, Re, betas, sweeps=None, tol=None):
    out = []
    for beta in betas:
        o = O.Oracle(G.case_misaligned_box(beta, 16, L=4.0, model=model, Re=Re))
        if sweeps is None:
            _, res = o.solve(tol=tol, max_iter=4000)
            assert o.max_residual(res) <= tol
        else:
            for _ in range(sweeps):
                o.sweep()
        out.append(o)
    return out


def _assert_mirror(a, b, atol):
    np.testing.assert_allclose(a.u[0][0], mirrored(b.u[1]), rtol=0, atol=atol, err_msg="u <-> v")
    np.testing.assert_allclose(a.u[1][0], mirrored(b.u[0]), rtol=0, atol=atol, err_msg="v <-> u")
    for name in ("p", "k", "eps", "nut"):
        np.testing.assert_allclose(getattr(a, name)[0], mirrored(getattr(b, name)), rtol=0,
                                   atol=atol * max(1.0, np.abs(getattr(b, name)).max()), err_msg=name)


def test_converged_laminar_state_at_30_mirrors_the_state_at_60():
    a, b = _pair("laminar", 20.0, (30.0, 60.0), tol=1e-12)
    _assert_mirror(a, b, 1e-13)
    # and the flow is not trivially symmetric: at 30 degrees u != v^T
    assert np.abs(a.u[0][0] - mirrored(a.u[1])).max() > 1e-2


def test_k_epsilon_sweeps_at_30_mirror_the_sweeps_at_60():
    """Each sweep, not only the fixed point: 60 k-epsilon sweeps from the
    uniform start (the iteration itself commutes with the mirror)."""
    a, b = _pair("kepsilon", 1e4, (30.0, 60.0), sweeps=60)
    _assert_mirror(a, b, 1e-13)
    assert np.abs(a.nut).max() > 1e-4


def test_45_degrees_is_its_own_mirror():
    (s,) = _pair("kepsilon", 1e4, (45.0,), sweeps=60)
    _assert_mirror(s, s, 1e-13)


def test_mirror_pin_catches_a_one_direction_mistake(monkeypatch):
    """A mistake planted in the oracle in one direction only -- the y-face
    diffusion coefficient of the momentum rows scaled by 1 + 1e-3, a
    stand-in for a wrong index or factor on one axis -- breaks the
    mirror."""
    orig = O.Oracle.__init__

    def planted(self, case, opts=None):
        orig(self, case, opts)
        self.m.D = list(self.m.D)
        self.m.D[1] = self.m.D[1] * (1.0 + 1e-3)

    monkeypatch.setattr(O.Oracle, "__init__", planted)
    a, b = _pair("laminar", 20.0, (30.0, 60.0), sweeps=40)
    err = max(np.abs(a.u[0][0] - mirrored(b.u[1])).max(), np.abs(a.p[0] - mirrored(b.p)).max())
    assert err > 1e-6
