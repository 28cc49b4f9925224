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


def test_pressure_drop_gradient_on_the_64x32_check_grid():
    """The gradient check grid of the batched-gradient workload: a 64 x 32
    random-obstacle channel (seed 0, k-epsilon, Re 1000) converged to 1e-13;
    dJ/dlambda of the pressure drop at the three cut cells of largest
    gradient equals central differences of frozen-turbulence solves (step
    1e-6, integer decisions checked unchanged) within 1e-5 (measured
    2e-8 - 7e-8)."""
    o = O.Oracle(G.case_grf(64, 32, seed=0))
    _, res = o.solve(tol=1e-13, max_iter=8000)
    assert o.max_residual(res) <= 1e-13
    fs = A.FrozenSteady(o)
    J, g, _ = fs.gradient()
    gf = g.ravel()
    lam = o.lam.ravel()
    cut = np.flatnonzero((lam > 0.05) & (lam < 0.95))
    pick = cut[np.argsort(-np.abs(gf[cut]))[:3]]
    fd = A.fd_gradient(o, pick, delta=1e-6)
    np.testing.assert_allclose(gf[pick], fd, rtol=1e-5)


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


# ---------------------------------------------------------------- reading B
def box15_reading_b():
    case = G.case_rotated_box(15.0, 16, model="laminar", Re=20.0)
    o = O.Oracle(case, dict(continuity_mask="B"))
    it, res = o.solve(tol=1e-13, max_iter=4000)
    assert o.max_residual(res) <= 1e-13
    return o


def test_readings_agree_without_cut_cells():
    """With lambda in {0, 1} only, m = [lambda < 1] = 1 - lambda: both readings
    run the same arithmetic, bit for bit."""
    case = G.case_rotated_box(15.0, 16, model="laminar", Re=20.0)
    case["lam"] = np.where(case["lam"] >= 0.5, 1.0, 0.0)
    a = O.Oracle(case)
    b = O.Oracle(case, dict(continuity_mask="B"))
    for _ in range(5):
        a.sweep()
        b.sweep()
    for x, y in ((a.u[0], b.u[0]), (a.u[1], b.u[1]), (a.p, b.p)):
        assert np.array_equal(x, y)


def test_reading_b_scales_the_continuity_of_cut_cells():
    """At a reading-B fixed point the corrected flux keeps lambda times the
    divergence of phiHbyA in every cell: div phi = div phiH - (1 - lambda)
    div phiH (the pressure equation, Eq. hfdibrans_2 with m = 1 - lambda)."""
    o = box15_reading_b()
    fs = A.FrozenSteady(o)
    z = fs.state()
    assert np.abs(fs.residual(z)).max() <= 1e-9 * np.abs(fs.residual(z * 1.01)).max()
    # the fluid cells (lambda = 0) are divergence-free, the cut cells not
    div = o.divergence(o.phi)
    fluid = o.lam == 0.0
    cut = (o.lam > 0.05) & (o.lam < 0.95)
    scale = float(np.abs(o.phi[0]).max())
    assert np.abs(div[fluid]).max() <= 1e-10 * scale
    assert np.abs(div[cut]).max() > 1e-6 * scale


@pytest.mark.slow
def test_reading_b_gradient_matches_finite_differences():
    """Reading B differentiates m = 1 - lambda: the gradient in the cut cells,
    in-solid (0.5 <= lambda < 1) and bc, matches central differences, and it
    reaches fluid cells far from the body, where reading A has none (there
    lambda moves no imposed velocity)."""
    o = box15_reading_b()
    fs = A.FrozenSteady(o)
    assert fs.n_kinks == 0
    J, g, _ = fs.gradient()
    gf = g.ravel()
    lam = o.lam.ravel()
    ic_cut = np.flatnonzero((lam >= 0.5) & (lam < 0.95))
    bc_cut = np.flatnonzero((lam > 0.05) & (lam < 0.5))
    assert np.abs(gf[ic_cut]).max() > 1e-3 * np.abs(gf).max()
    pick = np.concatenate([ic_cut[np.argsort(-np.abs(gf[ic_cut]))[:2]],
                           bc_cut[np.argsort(-np.abs(gf[bc_cut]))[:2]]])
    fd = A.fd_gradient(o, pick, delta=1e-6)
    np.testing.assert_allclose(gf[pick], fd, rtol=1e-5)
    # fluid cells more than 3 cells from any lambda > 0
    from scipy.ndimage import binary_dilation
    near = binary_dilation(o.lam[0] > 0.0, iterations=3)
    far = np.flatnonzero(~near.ravel())
    assert far.size > 100
    assert np.count_nonzero(gf[far]) > 0.9 * far.size
    a = O.Oracle(o.case)
    a.solve(tol=1e-13, max_iter=4000)
    _, ga, _ = A.FrozenSteady(a).gradient()
    assert np.all(ga.ravel()[far] == 0.0)


@pytest.mark.slow
def test_3d_gradient_matches_finite_differences():
    """The residual form and its adjoint in 3D (7-point rows, trilinear
    interpolation along n): a sphere placed off the grid's symmetry planes
    (no zero-flux faces), laminar; the fixed point satisfies R = 0 and
    dJ/dlambda matches central differences of frozen solves."""
    case = G.case_sphere(16, 8, 8, model="laminar", Re=20.0)
    X, Y, Z = G.cell_centres(case["grid"])
    sig = np.sqrt((X - 4.3) ** 2 + (Y - 3.7) ** 2 + (Z - 4.2) ** 2) - 1.4
    case["sigma"] = sig
    case["lam"] = G.lambda_from_sigma(sig, O.Mesh(case["grid"]).h)
    case["ywall"] = np.maximum(sig, 0.0)
    o = O.Oracle(case)
    it, res = o.solve(tol=1e-13, max_iter=4000)
    assert o.max_residual(res) <= 1e-13
    fs = A.FrozenSteady(o)
    assert fs.n_kinks == 0
    z = fs.state()
    assert np.abs(fs.residual(z)).max() <= 1e-9 * np.abs(fs.residual(z * 1.01)).max()
    J, g, _ = fs.gradient()
    gf = g.ravel()
    lam = o.lam.ravel()
    cut = np.flatnonzero((lam > 0.05) & (lam < 0.95))
    pick = cut[np.argsort(-np.abs(gf[cut]))[:3]]
    fd = A.fd_gradient(o, pick, delta=1e-6)
    np.testing.assert_allclose(gf[pick], fd, rtol=1e-5)
