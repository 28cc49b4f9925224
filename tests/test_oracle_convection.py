"""Pins of the oracle's convection schemes for momentum (App. B), applied as
a deferred correction of the bounded upwind rows.

* linearUpwind reproduces the exact face value of a linear field (the
  Gauss-linear cell gradient is exact there), for either flow direction.
* vanLeer is central on a linear field (r = 1, psi = 1), falls back to
  upwind at a local extremum (r < 0, psi = 0), and keeps every face value
  between its upwind and downwind cell values (TVD: 0 <= psi < 2).
* The correction only moves momentum between cells: a converged
  linearUpwind state still puts the momentum balance on the domain boundary
  (the force equals the boundary flux), and the symmetric cylinder stays
  mirror-symmetric under both schemes.
"""
import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O
from oracle import forces as Fo


def mesh(nx=12, ny=9):
    case = G.case_uniform(nx, ny)
    return O.Mesh(case["grid"]), case


def grad(m, f):
    spec = {key: (np.zeros(m.slab(f, *key).shape, bool), 0.0) for key in
            [(d, hi) for d in range(m.dims) for hi in (0, 1)]}
    return O.gauss_grad(m, f, spec)


def interior(arr, ax, n):
    """Faces whose both cells are one away from the domain edge along ax."""
    sl = [slice(None)] * 3
    sl[ax] = slice(1, n - 2)
    return arr[tuple(sl)]


@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("scheme", ["linearUpwind", "vanLeer"])
def test_linear_field_gets_its_exact_face_value(scheme, sign):
    m, _ = mesh()
    X, Y, _ = G.cell_centres(G.case_uniform(12, 9)["grid"])
    f = 0.7 * X - 1.3 * Y + 0.2
    g = grad(m, f)
    for d, a in ((0, 0.7), (1, -1.3)):
        ax = 2 - d
        n = m.n[d]
        shp = list(m.shape)
        shp[ax] = n + 1
        phi_d = np.full(shp, sign)
        face_corr = O.face_correction(m, phi_d, f, g[d], d, scheme)
        # exact face value minus the upwind cell value: +-a Delta/2
        expect = sign * a * 0.5 * m.D[d]
        np.testing.assert_allclose(interior(face_corr, ax, n), expect, rtol=1e-12, atol=1e-14)


def test_vanleer_is_upwind_at_an_extremum_and_bounded():
    m, _ = mesh(16, 5)
    X, _, _ = G.cell_centres(G.case_uniform(16, 5)["grid"])
    # a V-shaped profile along x with its minimum in cell 7
    xc = X[0, 0, 7]
    f = np.abs(X - xc)
    g = grad(m, f)
    phi_x = np.ones((1, 5, 17))
    corr = O.face_correction(m, phi_x, f, g[0], 0, "vanLeer")
    # face 7|8 has U = cell 7 (the minimum): zero central gradient there, r = -1
    assert np.all(corr[0, :, 7] == 0.0)
    # TVD: face values between the upwind and downwind values on random data
    rng = np.random.default_rng(3)
    f = rng.standard_normal(m.shape)
    g = grad(m, f)
    for sign in (1.0, -1.0):
        corr = O.face_correction(m, sign * phi_x, f, g[0], 0, "vanLeer")
        fL, fH = f[..., :-1], f[..., 1:]
        fU, fD = (fL, fH) if sign > 0 else (fH, fL)
        face = fU + corr
        assert np.all(face >= np.minimum(fU, fD) - 1e-15)
        assert np.all(face <= np.maximum(fU, fD) + 1e-15)


@pytest.mark.parametrize("scheme", ["linearUpwind", "vanLeer"])
def test_symmetric_cylinder_stays_symmetric(scheme):
    case = G.case_cylinder(48, 24, model="laminar", Re=40.0)
    o = O.Oracle(case, dict(convection=scheme))
    it, res = o.solve(tol=1e-10, max_iter=3000)
    assert o.max_residual(res) <= 1e-10
    ux, uy = o.u[0][0], o.u[1][0]
    assert np.abs(ux - ux[::-1]).max() < 1e-10
    assert np.abs(uy + uy[::-1]).max() < 1e-10
    # and differs from the upwind solution (the correction is active)
    a = O.Oracle(case)
    a.solve(tol=1e-10, max_iter=3000)
    assert np.abs(o.u[0] - a.u[0]).max() > 1e-3


def test_linear_upwind_keeps_the_momentum_balance():
    """The correction is a sum of face fluxes, equal and opposite in the two
    cells of a face: with it the force is still the momentum leaving the
    domain (the global balance of the force pin)."""
    from test_oracle_forces import boundary_momentum_flux
    case = G.case_rotated_box(15.0, 16, model="laminar", Re=20.0)
    o = O.Oracle(case, dict(convection="linearUpwind"))
    it, res = o.solve(tol=1e-13, max_iter=8000)
    assert o.max_residual(res) <= 1e-13
    o.imposed_fields()
    F = sum(Fo.ib_force(o))
    B = boundary_momentum_flux(o)
    scale = np.abs(B).max() + np.abs(F).max()
    assert np.abs(F + B).max() <= 1e-9 * scale


def test_adjoint_refuses_other_schemes():
    from oracle import adjoint as A
    case = G.case_rotated_box(15.0, 16, model="laminar", Re=20.0)
    o = O.Oracle(case, dict(convection="vanLeer"))
    o.sweep()
    with pytest.raises(ValueError):
        A.FrozenSteady(o)


def test_cell_limiter_keeps_extrapolations_within_the_neighbour_bounds():
    """Barth-Jespersen: l grad f extrapolated to each face stays within the
    min/max of the cell and its neighbours; on a linear field the interior
    limiter is 1 (the neighbours are a full cell away, the faces half)."""
    m, _ = mesh(16, 9)
    rng = np.random.default_rng(5)
    f = rng.standard_normal(m.shape)
    g = grad(m, f)
    lim = O.cell_limiter(m, f, g)
    assert np.all(lim >= 0.0) and np.all(lim <= 1.0)
    fmax, fmin = f.copy(), f.copy()
    for ax, n in ((2, m.nx), (1, m.ny)):
        sl = lambda a, b: tuple(slice(a, b) if i == ax else slice(None) for i in range(3))
        fmax[sl(0, n - 1)] = np.maximum(fmax[sl(0, n - 1)], f[sl(1, n)])
        fmax[sl(1, n)] = np.maximum(fmax[sl(1, n)], f[sl(0, n - 1)])
        fmin[sl(0, n - 1)] = np.minimum(fmin[sl(0, n - 1)], f[sl(1, n)])
        fmin[sl(1, n)] = np.minimum(fmin[sl(1, n)], f[sl(0, n - 1)])
    for d in range(2):
        for sgn in (1.0, -1.0):
            face = f + lim * sgn * 0.5 * m.D[d] * g[d]
            assert np.all(face <= fmax + 1e-14) and np.all(face >= fmin - 1e-14)
    X, Y, _ = G.cell_centres(G.case_uniform(16, 9)["grid"])
    f = 0.7 * X - 1.3 * Y
    lim = O.cell_limiter(m, f, grad(m, f))
    assert np.all(lim[0, 1:-1, 1:-1] == 1.0)


def test_limited_linear_upwind_keeps_symmetry_and_the_momentum_balance():
    from test_oracle_forces import boundary_momentum_flux
    case = G.case_cylinder(48, 24, model="laminar", Re=40.0)
    o = O.Oracle(case, dict(convection="linearUpwindLimited"))
    it, res = o.solve(tol=1e-10, max_iter=3000)
    assert o.max_residual(res) <= 1e-10
    assert np.abs(o.u[0][0] - o.u[0][0, ::-1]).max() < 1e-10
    box = G.case_rotated_box(15.0, 16, model="laminar", Re=20.0)
    o = O.Oracle(box, dict(convection="linearUpwindLimited"))
    it, res = o.solve(tol=1e-13, max_iter=8000)
    assert o.max_residual(res) <= 1e-13
    o.imposed_fields()
    F = sum(Fo.ib_force(o))
    B = boundary_momentum_flux(o)
    assert np.abs(F + B).max() <= 1e-9 * (np.abs(B).max() + np.abs(F).max())
