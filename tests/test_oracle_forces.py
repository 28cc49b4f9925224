"""Pins of the oracle's force on the body (Eqs. dragcoeff, dlcoeffs) and wall
shear stress (Sec. 3.3) against what the momentum balance fixes.

* At a converged state, the force on the body is the momentum that leaves the
  domain through its boundary, written here face by face from the boundary
  values alone: convective flux, wall and inlet diffusion, the explicit
  transpose flux, and the boundary pressure.
* Mirror images (a box rotated by +beta and -beta about the channel's axis)
  have the same drag and opposite lift; a body symmetric about the axis has
  no lift; no body, no force.
* In developed laminar flow between two domain walls, the wall shear of the
  discrete equations has the closed form 6 nu U H / (H^2 + 2 Delta^2) and
  balances the pressure gradient: tau_bottom + tau_top = -H dp/dx.
"""
import math

import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O
from oracle import forces as Fo


def converged(case, tol=1e-13, max_iter=8000):
    o = O.Oracle(case)
    it, res = o.solve(tol=tol, max_iter=max_iter)
    assert o.max_residual(res) <= tol, (it, res)
    # the imposed fields of the converged state, as the next sweep would set them
    o.imposed_fields()
    return o


def _face(arr, d, hi, m):
    ax = 2 - d
    n = arr.shape[ax]
    sl = [slice(None)] * 3
    sl[ax] = slice(n - 1, n) if hi else slice(0, 1)
    return arr[tuple(sl)]


def boundary_momentum_flux(o):
    """Sum over the domain's boundary faces of the momentum leaving through
    them (the terms every row's interior faces cancel down to)."""
    m = o.m
    nu_eff = o.nu + o.nut
    G_ = o.velocity_grad(o.u)          # G_[q][a] = d u_a / d x_q
    B = np.zeros(3)
    for d in range(m.dims):
        for hi in (0, 1):
            kind = o.bnd.kind[(d, hi)]
            closed = o.bnd.closed[(d, hi)]
            sgn = 1.0 if hi else -1.0
            Fout = sgn * _face(o.phi[d], d, hi, m)
            nuP = m.slab(nu_eff, d, hi)
            pP = m.slab(o.p, d, hi)
            pb = np.full(pP.shape, o.bnd.p_out) if kind == "outlet" else pP
            for q in range(m.dims):
                uP = m.slab(Fo.imposed_velocity(o, q), d, hi)
                if kind == "inlet":
                    fixed, val = ~closed, o.bnd.u_in[q]
                elif kind == "wall":
                    fixed, val = ~closed, 0.0
                elif kind == "slip":
                    fixed, val = ~closed & (q == d), 0.0
                else:
                    fixed, val = np.zeros(closed.shape, bool), 0.0
                # convection: upwind, the boundary value where it flows in
                ub = np.where(fixed & (Fout < 0.0), val, uP)
                conv = Fout * ub
                # diffusion through a face with a fixed value (half-cell distance)
                diff = np.where(fixed, nuP * m.S[d] * (uP - val) / (0.5 * m.D[d]), 0.0)
                # explicit div(nu_eff (grad u)^T): the cell's d u_d / d x_q on the face
                trans = -sgn * nuP * m.slab(G_[q][d], d, hi) * m.S[d]
                press = sgn * pb * m.S[d] if q == d else 0.0 * pb
                B[q] += float(np.sum(conv + diff + trans + press))
    return B


CASES = {
    "box15_laminar": lambda: G.case_rotated_box(15.0, 16, model="laminar", Re=20.0),
    "grf_keps_32x16": lambda: G.case_grf(32, 16, seed=1),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_force_is_the_momentum_leaving_through_the_domain_boundary(name):
    o = converged(CASES[name]())
    Fn, Ft = Fo.ib_force(o)
    F = Fn + Ft
    B = boundary_momentum_flux(o)
    scale = np.abs(B).max() + np.abs(F).max()
    print(name, "F", F, "boundary", -B)
    assert np.abs(F + B).max() <= 1e-9 * scale
    assert abs(F[0]) > 1e-3 * scale


def test_mirror_images_have_equal_drag_and_opposite_lift():
    a = converged(G.case_rotated_box(15.0, 16, model="laminar", Re=20.0))
    b = converged(G.case_rotated_box(-15.0, 16, model="laminar", Re=20.0))
    Fa = sum(Fo.ib_force(a))
    Fb = sum(Fo.ib_force(b))
    print("F(+15)", Fa, "F(-15)", Fb)
    assert abs(Fa[1]) > 0.05 * abs(Fa[0])
    assert abs(Fa[0] - Fb[0]) <= 1e-9 * abs(Fa[0])
    assert abs(Fa[1] + Fb[1]) <= 1e-9 * abs(Fa[0])


def test_symmetric_body_has_no_lift():
    o = converged(G.case_cylinder(32, 16, model="laminar", Re=10.0))
    Fn, Ft = Fo.ib_force(o)
    F = Fn + Ft
    assert F[0] > 0.0
    assert abs(F[1]) <= 1e-10 * F[0]
    # pressure and viscous parts both push the body downstream at Re = 10
    assert Fn[0] > 0.0 and Ft[0] > 0.0


def test_no_body_no_force():
    o = O.Oracle(G.case_uniform(16, 8, model="laminar"))
    for _ in range(3):
        o.sweep()
    o.imposed_fields()
    Fn, Ft = Fo.ib_force(o)
    assert not Fo.imposed_rows(o).any()
    assert np.all(Fn == 0.0) and np.all(Ft == 0.0)


def test_force_coefficients_formula():
    # q = 0.5 A_ref |u_in|^2 = 1
    Cd, Cl = Fo.force_coefficients([2.0, 1.0, 0.0], 0.5, (2.0, 0.0, 0.0))
    assert Cd == 2.0 and Cl == 1.0
    g = math.radians(30.0)
    Cd, Cl = Fo.force_coefficients([2.0, 1.0, 0.0], 0.5, (2.0, 0.0, 0.0), gamma=g)
    assert Cd == 2.0
    assert abs(Cl - (-math.sin(g) * 2.0 + math.cos(g) * 1.0)) <= 1e-15


def duct_case(nx=64, ny=8, L=8.0, H=1.0, Re=10.0):
    g = G.make_grid(nx, ny, 1, 0.0, 0.0, L, H)
    X, _, _ = G.cell_centres(g)
    far = np.full(X.shape, 1e3)
    return G._base_case("duct", g, far, far, "laminar", Re,
                        G.bc2d(ymin="wall", ymax="wall"), lt_in=0.1)


def test_developed_duct_wall_shear_closed_form():
    """Developed laminar flow: the discrete profile is A y(H-y) + A Delta^2/4
    (central differences are exact for the quadratic, the wall row with its
    half-cell distance fixes the offset), with A = 6U/(H^2 + 2 Delta^2) from
    the flow rate, so tau_w = nu A H."""
    H, ny, Re = 1.0, 8, 10.0
    o = converged(duct_case(ny=ny, H=H, Re=Re))
    m = o.m
    nu = o.nu
    U = 1.0
    dy = H / ny
    expect = 6.0 * nu * U * H / (H * H + 2.0 * dy * dy)
    tb = Fo.wall_shear(o, "ymin")
    tt = Fo.wall_shear(o, "ymax")
    xs = m.x0 + (np.arange(m.nx) + 0.5) * m.dx
    sel = (xs > 4.0) & (xs < 6.0)
    # tau_x = nu du_x/dn with n pointing into the fluid: positive on both
    # walls for flow in +x
    assert np.abs(tb[0][sel] - expect).max() <= 1e-7 * expect
    assert np.abs(tt[0][sel] - expect).max() <= 1e-7 * expect
    assert np.all(tb[1] == 0.0) and np.all(tb[2] == 0.0)
    # force balance of a developed column: both walls against the pressure drop
    gradp = O.gauss_grad(m, o.p, o.bnd.pressure_spec())[0][0, 0]
    assert np.abs((tb[0] + tt[0])[sel] + H * gradp[sel]).max() <= 1e-7 * expect


def test_wall_shear_rejects_non_wall_sides():
    o = O.Oracle(duct_case(nx=16, ny=4))
    with pytest.raises(ValueError):
        Fo.wall_shear(o, "xmin")


def test_reattachment_interpolates_the_last_upward_zero():
    x = np.arange(10.0)
    # corner vortex (+), main bubble (-), reattached (+)
    t = np.array([0.5, 0.2, -0.1, -0.4, -0.3, -0.2, 0.2, 0.4, 0.5, 0.6])
    assert abs(Fo.reattachment(x, t) - 5.5) <= 1e-15
    assert Fo.reattachment(x, np.abs(t) + 0.1) is None


@pytest.mark.parametrize("model", ["komegasst", "kepsilon"])
def test_recirculation_ends_at_the_reattachment_point(model):
    """Behind the step the furthest recirculating cell sits on the bottom
    wall, where tau_x has the sign of u_x: its centre L and the zero of tau_x
    satisfy L <= x_reat < L + dx (two definitions of Sec. 3.3 and 3.6)."""
    o = converged(G.case_bfs(64, 16, model=model), tol=1e-8, max_iter=3000)
    m = o.m
    xs = m.x0 + (np.arange(m.nx) + 0.5) * m.dx
    x_reat = Fo.reattachment(xs, Fo.wall_shear(o, "ymin")[0])
    L, V, n = Fo.recirculation(o, 0.0)
    assert n > 0 and abs(V - n * m.V) <= 1e-15 * V
    assert L <= x_reat < L + m.dx, (L, x_reat)
    # nothing recirculates upstream of the step's rear end inside the solid
    L0, V0, n0 = Fo.recirculation(o, 1e9)
    assert (L0, V0, n0) == (0.0, 0.0, 0)
