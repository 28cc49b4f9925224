"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: hand-derived
cell groups and distances (Sec. 2.3-2.4), closed forms of the wall functions
(Eqs. kws, frictionvel, omegaws), exact properties of the discrete operators
(linear fields, a linear pressure), the lambda == 0 uniform flow, the laminar
Poiseuille profile between immersed walls, mass conservation at convergence
(App. D) and mirror symmetry.
"""
import math
import os

import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def flat_wall_case(yw, nx=8, ny=8, dx=1.0, dy=1.0):
    g = G.make_grid(nx, ny, 1, 0.0, 0.0, nx * dx, ny * dy)
    X, Y, _ = G.cell_centres(g)
    sigma = Y - yw
    return G._base_case("flat", g, sigma, np.maximum(sigma, 0), "kepsilon", 100.0, G.bc2d())


def read_golden_tags():
    rows = {}
    for line in open(os.path.join(GOLDEN, "flat_wall_2d.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        a, b = line.split()
        if a.isdigit():
            rows[int(a)] = int(b)
        else:
            rows[a] = float(b)
    return rows


# ---------------------------------------------------------------- lambda, sigma
def test_lambda_sigma_round_trip():
    """sigma = h atanh(1 - 2 lambda(sigma)) inside the band (Eqs. lambda, yorthoaux)."""
    case = G.case_cylinder(64, 32)
    m = O.Mesh(case["grid"])
    lam = case["lam"]
    band = (lam > 0) & (lam < 1)
    assert band.sum() >= 16
    s_back = np.array([O.sigma_of_lambda(m, v) for v in lam[band]])
    np.testing.assert_allclose(s_back, case["sigma"][band], rtol=1e-12, atol=1e-13)
    assert np.all(lam[case["sigma"] >= 0.75 * m.h] == 0.0)
    assert np.all(lam[case["sigma"] <= -0.75 * m.h] == 1.0)


# ---------------------------------------------------------------- a0 pins
def test_flat_wall_groups_and_case_a():
    gold = read_golden_tags()
    case = flat_wall_case(2.3)
    m = O.Mesh(case["grid"])
    tag = O.classify(m, case["lam"])
    for j in range(8):
        assert np.all(tag[0, j, :] == gold[j]), j
    geo = O.ib_geometry(m, case["lam"], tag)
    assert np.all(geo["case"] == 0)
    np.testing.assert_allclose(geo["y_perp"], gold["yperp_row2"], rtol=1e-13)
    np.testing.assert_array_equal(geo["n"], np.tile([0.0, 1.0, 0.0], (8, 1)))
    # face neighbour straight below
    cells = geo["cell"]
    np.testing.assert_array_equal(geo["nbr"], cells - 8)
    np.testing.assert_allclose(geo["y_eff"], 0.5 * (0.2 + 0.5), rtol=1e-13)


@pytest.mark.parametrize("yw,row,yperp", [(2.9, 3, 0.6), (3.0, 3, 0.5)])
def test_flat_wall_other_offsets(yw, row, yperp):
    case = flat_wall_case(yw)
    m = O.Mesh(case["grid"])
    tag = O.classify(m, case["lam"])
    assert np.all(tag[0, row - 1] == O.TAG_IC) and np.all(tag[0, row] == O.TAG_BC)
    assert np.all(tag[0, row + 1:] == O.TAG_FC)
    geo = O.ib_geometry(m, case["lam"], tag)
    np.testing.assert_allclose(geo["y_perp"], yperp, rtol=1e-12)


def test_case_b_true_distance():
    """lambda_P = 0, lambda_N in [.5, 1): n_N.[P - (N + |sigma_N| n_N)] = 0.8."""
    case = flat_wall_case(1.7)
    m = O.Mesh(case["grid"])
    tag = O.classify(m, case["lam"])
    geo = O.ib_geometry(m, case["lam"], tag)
    row2 = geo["cell"] // 8 == 2
    assert np.all(geo["case"][row2] == 1)
    np.testing.assert_allclose(geo["y_perp"][row2], 0.8, rtol=1e-12)


def test_case_c_shared_vertices():
    """lambda_P = 0, lambda_N = 1 on dx=0.5, dy=2 cells: y_perp = dy/2."""
    case = flat_wall_case(2.0, nx=8, ny=6, dx=0.5, dy=2.0)
    m = O.Mesh(case["grid"])
    assert abs(m.h - 1.0) < 1e-15
    tag = O.classify(m, case["lam"])
    geo = O.ib_geometry(m, case["lam"], tag)
    assert np.all(geo["case"] == 2)
    np.testing.assert_allclose(geo["y_perp"], 1.0, rtol=1e-14)
    np.testing.assert_array_equal(geo["nbr"], geo["cell"] - 8)


def test_interpolation_weights_reproduce_quadratics():
    """The quadratic through S, X1, X2 is exact for any quadratic profile."""
    case = G.case_cylinder(64, 32)
    m = O.Mesh(case["grid"])
    tag = O.classify(m, case["lam"])
    geo = O.ib_geometry(m, case["lam"], tag)
    h = m.h
    for coeffs in ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.3, -2.0, 5.0)):
        f = lambda d: coeffs[0] + coeffs[1] * d + coeffs[2] * d * d
        yp = geo["y_perp"]
        val = geo["wS"] * f(0.0) + geo["w1"] * f(yp + h) + geo["w2"] * f(yp + 2 * h)
        np.testing.assert_allclose(val, f(yp), rtol=1e-11, atol=1e-12)


def test_bilinear_interpolation_exact_for_linear_fields():
    case = G.case_cylinder(64, 32)
    m = O.Mesh(case["grid"])
    tag = O.classify(m, case["lam"])
    geo = O.ib_geometry(m, case["lam"], tag)
    X, Y, _ = G.cell_centres(case["grid"])
    f = 2.0 * X - 3.0 * Y + 1.0
    v = O.interp_at(m, f, geo["base1"], geo["t1"])
    # reconstruct X1 from the stencil and compare with the linear function
    x1 = m.x0 + (geo["base1"][:, 0] + 0.5 + geo["t1"][:, 0]) * m.dx
    y1 = m.y0 + (geo["base1"][:, 1] + 0.5 + geo["t1"][:, 1]) * m.dy
    np.testing.assert_allclose(v, 2 * x1 - 3 * y1 + 1.0, rtol=1e-12, atol=1e-12)
    # and X1 = P + h n
    k = geo["cell"]
    P = np.stack([X.ravel()[k], Y.ravel()[k]], 1)
    np.testing.assert_allclose(np.stack([x1, y1], 1), P + m.h * geo["n"][:, :2], atol=1e-12)


# ---------------------------------------------------------------- wall functions
@pytest.fixture(scope="module")
def cyl_converged():
    case = G.case_cylinder(64, 32)
    o = O.Oracle(case)
    it, res = o.solve(tol=1e-12, max_iter=600)
    assert o.max_residual(res) <= 1e-12, res
    return o


def test_imposed_values_follow_wall_functions(cyl_converged):
    """At convergence: in log-branch bc cells nu_t = k/omega_ib = kappa u_tau y_eff;
    in ic cells u = u_s before the update, k = 0, eps = max over bc u fc."""
    o = cyl_converged
    o.imposed_fields()
    cells = o.geo["cell"]
    k = o.k.ravel()[cells]
    ut = O.C_MU ** 0.25 * np.sqrt(k)
    yp = o.geo["y_eff"] * ut / o.nu
    logb = yp > O.YPLUS_LAM
    lamb = ~logb
    assert lamb.any()
    nut = o.nut.ravel()[cells]
    eps = o.eps.ravel()[cells]
    # eps_ib = C_mu k omega_ib with omega_ib of Eq. omegaws
    wl = 6.0 * o.nu / (O.BETA1_WF * o.geo["y_eff"] ** 2)
    np.testing.assert_allclose(eps[lamb], np.maximum(O.C_MU * k[lamb] * wl[lamb], O.EPS_MIN),
                               rtol=1e-9)
    if logb.any():
        np.testing.assert_allclose(nut[logb], O.KAPPA * ut[logb] * o.geo["y_eff"][logb],
                                   rtol=1e-9)
    assert np.all(o.k[o.ic] == 0.0)
    assert np.all(o.nut[o.ic] == 0.0)
    np.testing.assert_allclose(o.eps[o.ic], o.eps[~o.ic].max(), rtol=1e-9)


def test_log_branch_nut_on_bfs():
    """High-Re case (all bc cells log branch): nu_t = kappa u_tau y_eff (Sec. 1)."""
    case = G.case_bfs(64, 16, model="kepsilon")
    o = O.Oracle(case)
    it, res = o.solve(tol=1e-11, max_iter=800)
    assert o.max_residual(res) <= 1e-11
    o.imposed_fields()
    cells = o.geo["cell"]
    assert not o.lam_branch.any()
    k = o.k.ravel()[cells]
    ut = O.C_MU ** 0.25 * np.sqrt(k)
    np.testing.assert_allclose(o.nut.ravel()[cells], O.KAPPA * ut * o.geo["y_eff"], rtol=1e-8)


# ---------------------------------------------------------------- operators
def test_transport_operator_exact_on_linear_field():
    """Upwind convection of a linear field with uniform flux is exact; the
    diffusion of a linear field vanishes (interior cells)."""
    case = G.case_uniform(12, 8)
    m = O.Mesh(case["grid"])
    X, Y, _ = G.cell_centres(case["grid"])
    U, Vv = 0.7, -0.3
    phi = [np.full((1, 8, 13), U * m.S[0]), np.full((1, 9, 12), Vv * m.S[1])]
    gamma = np.full(m.shape, 0.05)
    spec = {key: (np.zeros((1, 1, 1), bool), 0.0) for key in O.SIDE_NAMES}
    aP, aM, aPl, b = O.assemble_transport(m, phi, gamma, spec)
    f = 1.0 + 2.0 * X - 5.0 * Y
    Af = aP * f + O.apply_offdiag(m, aM, aPl, f)
    inner = (slice(None), slice(1, -1), slice(1, -1))
    np.testing.assert_allclose(Af[inner], (U * 2.0 + Vv * (-5.0)) * m.V, rtol=1e-12)


def test_pressure_operator_linear_pressure():
    """-laplacian(rAU, p) of p = g (x_out - x) is zero inside and matches the
    outlet Dirichlet term (half-cell distance), so A p = rhs_outlet exactly;
    the zero-gradient inlet column sees one face flux rAU S g."""
    case = G.case_uniform(16, 8)
    o = O.Oracle(case)
    m = o.m
    X, _, _ = G.cell_centres(case["grid"])
    xo = m.x0 + m.nx * m.dx
    p = 3.0 * (xo - X)
    rAU = np.full(m.shape, 0.37)
    coef, aP, aM, aPl, rhs = o.pressure_operator(rAU)
    Ap = aP * p + O.apply_offdiag(m, aM, aPl, p)
    # the inlet column is zero-gradient (no boundary flux), the rest is exact
    np.testing.assert_allclose(Ap[..., 1:], rhs[..., 1:], atol=1e-12)
    np.testing.assert_allclose(Ap[..., 0], 0.37 * m.S[0] / m.dx * 3.0 * m.dx, rtol=1e-12)
    # the corrected flux of that pressure is uniform: rAU g S
    phi = o.correct_flux([np.zeros((1, 8, 17)), np.zeros((1, 9, 16))], coef, p)
    np.testing.assert_allclose(phi[0][0, :, 1:], 0.37 * 3.0 * m.S[0], rtol=1e-12)


# ---------------------------------------------------------------- flows
def test_uniform_flow_stays_uniform():
    """lambda == 0: u = (U, 0), p = 0 to round-off; k, eps depend on x only
    and decay downstream."""
    case = G.case_uniform(48, 8, Re=1e5, I_in=0.05)
    o = O.Oracle(case)
    for _ in range(40):
        o.sweep()
    assert np.abs(o.u[0] - 1.0).max() < 1e-13
    assert np.abs(o.u[1]).max() < 1e-13
    assert np.abs(o.p).max() < 1e-12
    assert np.abs(o.k - o.k[:, :1, :]).max() < 1e-9 * o.k.max()
    kx = o.k[0, 0]
    assert np.all(np.diff(kx) < 0)


def test_homogeneous_decay_exponent():
    """lambda == 0, tiny nu: k(x) follows decaying homogeneous turbulence,
    k ~ (x + x0)^(-1/(C2 - 1)) (dk/dt = -eps, deps/dt = -C2 eps^2/k)."""
    case = G.case_uniform(400, 4, Re=1e8, I_in=0.1)
    case["lt_in"] = 0.02
    o = O.Oracle(case)
    it, res = o.solve(tol=1e-12, max_iter=400)
    X, _, _ = G.cell_centres(case["grid"])
    k = o.k[0, 0]
    e = o.eps[0, 0]
    # virtual origin from the inlet state: t0 = k/((C2-1) eps)
    n_exp = 1.0 / (O.KE_C2 - 1.0)
    t = X[0, 0]
    sel = (t > 0.5) & (t < 1.8)
    slope = np.polyfit(np.log(t[sel] + o.k_in / ((O.KE_C2 - 1) * o.eps_in)), np.log(k[sel]), 1)[0]
    assert abs(-slope - n_exp) / n_exp < 0.03, slope


def test_poiseuille_between_immersed_walls():
    """Laminar channel (Sec. 3.1 geometry): the developed profile approaches
    (3/2) U (1 - (2y/H - 1)^2) under refinement; dp/dx -> -12 nu U / H^2."""
    errs = []
    for ny in (8, 16, 32):
        case = G.case_channel(ny_in=ny, nx=4 * ny, Re=10.0)
        o = O.Oracle(case)
        it, res = o.solve(tol=1e-10, max_iter=3000)
        assert o.max_residual(res) <= 1e-10
        X, Y, _ = G.cell_centres(case["grid"])
        col = -ny
        y = Y[0, :, col]
        fl = (y > 0) & (y < 1)
        exact = 1.5 * (1 - (2 * y - 1) ** 2)
        errs.append(np.abs(o.u[0][0, fl, col] - exact[fl]).max())
        dpdx = (o.p[0, ny // 2 + 3, col + 1] - o.p[0, ny // 2 + 3, col - 1]) / (2 * o.m.dx)
        nu = 1.0 / case["Re"]
        if ny == 32:
            assert abs(dpdx - (-12 * nu)) / (12 * nu) < 0.05, dpdx
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 0.03, errs


def test_continuity_and_symmetry(cyl_converged):
    """App. D: sum m |div phi| -> 0 at convergence; the cylinder in a
    y-symmetric channel gives u_x even, u_y odd in y."""
    o = cyl_converged
    inflow = float(np.abs(o.phi[0][..., 0]).sum())
    assert o.history[-1]["cont"] / inflow < 1e-10
    ux, uy, p = o.u[0][0], o.u[1][0], o.p[0]
    assert np.abs(ux - ux[::-1]).max() < 1e-9
    assert np.abs(uy + uy[::-1]).max() < 1e-9
    assert np.abs(p - p[::-1]).max() < 1e-9
    assert np.abs(o.k[0] - o.k[0, ::-1]).max() < 1e-9


def test_production_of_simple_shear():
    """u = (s y, 0): 2 S:S = s^2, so G = nu_t s^2 in interior fluid cells."""
    case = G.case_uniform(12, 10)
    o = O.Oracle(case)
    _, Y, _ = G.cell_centres(case["grid"])
    s = 0.8
    o.u = [s * Y, np.zeros_like(Y)]
    o.nut = np.full(o.m.shape, 0.02)
    o.imposed_fields()
    _, S2, Gk, _ = o._production()
    inner = (slice(None), slice(1, -1), slice(1, -1))
    np.testing.assert_allclose(S2[inner], s * s, rtol=1e-12)
    np.testing.assert_allclose(Gk[inner], 0.02 * s * s, rtol=1e-12)


def test_transpose_term_linear_velocity():
    """div(nu (grad u)^T) for u = (a x, -a y) and nu = nu0 + c x is
    (c a, 0) per unit volume in interior cells (grad u^T is constant)."""
    case = G.case_uniform(12, 10)
    o = O.Oracle(case)
    X, Y, _ = G.cell_centres(case["grid"])
    a, c = 0.6, 0.3
    u = [a * X, -a * Y]
    nu = 0.01 + c * X
    Gt = o.velocity_grad(u)
    inner = (slice(None), slice(2, -2), slice(2, -2))
    Tx = o.transpose_source(Gt, nu, 0)
    Ty = o.transpose_source(Gt, nu, 1)
    np.testing.assert_allclose(Tx[inner], c * a * o.m.V, rtol=1e-10)
    np.testing.assert_allclose(Ty[inner], 0.0, atol=1e-13)


def test_keps_wall_eps_uses_the_imposed_k():
    """k-eps wall value: eps_ib = C_mu k omega_ib (Eq. omegaws) with k the value
    the cell takes this sweep, so in laminar-branch cells the eddy viscosity
    C_mu k_ib^2 / eps_ib is k_ib / omega_ib = k_ib beta1 y_eff^2 / (6 nu),
    whatever the old k_P was (here set to the 1e-14 floor)."""
    case = G.case_grf(64, 32, seed=1)
    o = O.Oracle(case)
    cells = o.geo["cell"]
    kf = o.k.ravel().copy()
    kf[cells] = O.K_MIN
    o.k = kf.reshape(o.m.shape)
    o.imposed_fields()
    lam = o.lam_branch
    assert lam.all()
    kib = o.k_ib.ravel()[cells]
    eib = o.eps_ib.ravel()[cells]
    ye = o.geo["y_eff"]
    wl = 6.0 * o.nu / (O.BETA1_WF * ye ** 2)
    np.testing.assert_allclose(eib, O.C_MU * kib * wl, rtol=1e-14)
    sel = kib > 0
    assert sel.sum() > 10
    np.testing.assert_allclose(O.C_MU * kib[sel] ** 2 / eib[sel], kib[sel] / wl[sel], rtol=1e-12)


@pytest.mark.slow
def test_keps_random_obstacle_converges():
    """k-eps channel with a random smooth obstacle reaches a steady state with
    vanishing continuity error (it diverged with eps_ib built from a stale
    k_P)."""
    case = G.case_grf(64, 32, seed=1)
    o = O.Oracle(case)
    it, res = o.solve(tol=1e-6, max_iter=400)
    assert o.max_residual(res) <= 1e-6, (it, res)
    assert res["cont"] < 1e-12
    assert np.isfinite(o.nut).all() and o.nut.max() < 1.0


@pytest.mark.parametrize("wall_distance", ["y_eff", "y_perp"])
def test_wall_distance_option_on_the_flat_wall(wall_distance):
    """y+ (Eq. yplus) and the laminar-branch omega_ib (Eq. omegaws) use y_eff =
    (y_perp + h/2)/2 by default and y_perp under the App. A option; on the
    flat wall y_perp = 0.2 (golden) and h = 1, so y_eff = 0.35."""
    gold = read_golden_tags()
    case = flat_wall_case(2.3)
    case["model"] = "komegasst"
    o = O.Oracle(case, dict(wall_distance=wall_distance))
    o.k = np.full(o.m.shape, 0.01)
    o.imposed_fields()
    y = gold["yperp_row2"] if wall_distance == "y_perp" else 0.5 * (gold["yperp_row2"] + 0.5)
    ut = O.C_MU ** 0.25 * math.sqrt(0.01)
    np.testing.assert_allclose(o.yplus_bc, y * ut / o.nu, rtol=1e-13)
    cells = o.geo["cell"]
    lam = o.lam_branch
    assert lam.all()                         # y+ < 11 at nu = 0.01: laminar branch
    np.testing.assert_allclose(o.omega_ib.ravel()[cells], 6.0 * o.nu / (O.BETA1_WF * y * y), rtol=1e-13)


def test_wall_distance_option_changes_the_step():
    """On the k-eps step the two distances give different sweeps (the option
    reaches omega_ib / eps_ib and the branch of Eq. alphauk)."""
    case = G.case_bfs(64, 16, model="kepsilon")
    a = O.Oracle(case)
    b = O.Oracle(case, dict(wall_distance="y_perp"))
    for _ in range(3):
        a.sweep()
        b.sweep()
    assert np.linalg.norm(a.eps - b.eps) > 1e-3 * np.linalg.norm(a.eps)
