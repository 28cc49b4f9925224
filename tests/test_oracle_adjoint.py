"""Pins of the oracle's frozen-turbulence adjoint (oracle/adjoint.py).

* The residual form R(z; lambda) vanishes at the oracle's converged sweep
  fixed point: it states the same discrete equations as the sweep.
* Its geometry restatement reproduces ib_geometry for real lambda.
* The coloured complex-step Jacobian equals single complex-step
  Jacobian-vector products (the colouring attributes every entry).
* dJ/dlambda equals central finite differences of frozen-turbulence solves
  on perturbed lambda (integer decisions checked unchanged).
"""
import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O
from oracle import adjoint as A


@pytest.fixture(scope="module")
def grf_state():
    case = G.case_grf(32, 16, seed=1)
    o = O.Oracle(case)
    it, res = o.solve(tol=1e-13, max_iter=4000)
    assert o.max_residual(res) <= 1e-13
    return o


def test_residual_form_vanishes_at_sweep_fixed_point(grf_state):
    fs = A.FrozenSteady(grf_state)
    z = fs.state()
    r0 = np.abs(fs.residual(z)).max()
    # a 1% perturbation of the state gives the scale of a non-solution
    r1 = np.abs(fs.residual(z * 1.01)).max()
    assert r0 <= 1e-9 * r1, (r0, r1)


def test_geometry_restatement_matches_ib_geometry(grf_state):
    o = grf_state
    w = A.bc_weights(o.m, o.lam, o.geo)
    for key in ("n", "y_perp", "t1", "t2", "wS", "w1", "w2"):
        np.testing.assert_allclose(w[key], o.geo[key], rtol=1e-14, atol=1e-15, err_msg=key)


def test_colouring_equals_jacobian_vector_products(grf_state):
    fs = A.FrozenSteady(grf_state)
    z = fs.state()
    Rz = fs.jacobian_z(z)
    rng = np.random.default_rng(7)
    for _ in range(2):
        v = rng.standard_normal(len(z))
        # the faces whose flux is exactly zero (walls, slip, closed) sit on the
        # kink of the upwind max(F, 0): take the same side as the colouring
        v[z == 0.0] = np.abs(v[z == 0.0])
        jv = fs.residual(z + 1j * A.H_CS * v).imag / A.H_CS
        assert np.abs(Rz @ v - jv).max() <= 1e-13 * np.abs(jv).max()
    Rl = fs.jacobian_lambda(z)
    v = rng.standard_normal(grf_state.m.N)
    jv = fs.residual(z.astype(complex), (grf_state.lam.ravel() + 1j * A.H_CS * v).reshape(grf_state.m.shape))
    jv = jv.imag / A.H_CS
    assert np.abs(Rl @ v - jv).max() <= 1e-13 * np.abs(jv).max()


@pytest.mark.slow
def test_pressure_drop_gradient_matches_finite_differences(grf_state):
    o = grf_state
    fs = A.FrozenSteady(o)
    J, g, _ = fs.gradient()
    assert abs(J - fs.objective(fs.state())) == 0.0
    gf = g.ravel()
    lam = o.lam.ravel()
    cut = np.flatnonzero((lam > 0.05) & (lam < 0.95))
    pick = cut[np.argsort(-np.abs(gf[cut]))[:3]]
    fd = A.fd_gradient(o, pick, delta=1e-6)
    np.testing.assert_allclose(gf[pick], fd, rtol=1e-5)
    # the gradient lives where lambda moves the imposed velocities only
    assert np.count_nonzero(gf) < 0.2 * o.m.N


def test_symmetric_flow_has_zero_flux_faces():
    """A cylinder on the channel axis gives a mirror-symmetric flow whose
    centre-line faces carry no flux: the upwind switch sits on its kink there
    and the gradient is refused."""
    case = G.case_cylinder(32, 16, model="laminar", Re=20.0)
    o = O.Oracle(case)
    o.solve(tol=1e-12, max_iter=4000)
    fs = A.FrozenSteady(o)
    assert fs.n_kinks == 32
    with pytest.raises(ValueError):
        fs.gradient()


@pytest.mark.slow
def test_laminar_gradient_matches_finite_differences():
    """All bc cells imposed (laminar model): every cut cell moves u_ib.  A
    box rotated by 15 degrees keeps every interior face flux away from 0."""
    case = G.case_rotated_box(15.0, 16, model="laminar", Re=20.0)
    o = O.Oracle(case)
    it, res = o.solve(tol=1e-13, max_iter=4000)
    assert o.max_residual(res) <= 1e-13
    fs = A.FrozenSteady(o)
    assert fs.n_kinks == 0
    J, g, _ = fs.gradient()
    gf = g.ravel()
    lam = o.lam.ravel()
    cut = np.flatnonzero((lam > 0.05) & (lam < 0.95))
    pick = cut[np.argsort(-np.abs(gf[cut]))[:3]]
    fd = A.fd_gradient(o, pick, delta=1e-6)
    np.testing.assert_allclose(gf[pick], fd, rtol=1e-5)


@pytest.mark.slow
@pytest.mark.parametrize("which", ["grf", "box15"])
def test_drag_gradient_matches_finite_differences(which, grf_state):
    """Drag (the x force of the fluid on the body, minus the immersed-boundary
    forcing of the imposed rows): J_lambda - psi^T R_lambda against central
    differences of frozen-turbulence solves, and positive for flow in +x."""
    if which == "grf":
        o = grf_state
    else:
        o = O.Oracle(G.case_rotated_box(15.0, 16, model="laminar", Re=20.0))
        o.solve(tol=1e-13, max_iter=4000)
    fs = A.FrozenSteady(o, "drag")
    J, g, _ = fs.gradient()
    assert J > 0.0
    gf = g.ravel()
    lam = o.lam.ravel()
    cut = np.flatnonzero((lam > 0.05) & (lam < 0.95))
    pick = cut[np.argsort(-np.abs(gf[cut]))[:3]]
    fd = A.fd_gradient(o, pick, delta=1e-6, objective="drag")
    np.testing.assert_allclose(gf[pick], fd, rtol=1e-5)
