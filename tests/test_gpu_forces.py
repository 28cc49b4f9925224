"""Force on the body (hfdib_ib_force, Eqs. dragcoeff and dlcoeffs) and wall
shear stress (hfdib_wall_shear, Sec. 3.3) through the C ABI, against the
oracle and the closed form of developed duct flow.

* The force of each side's converged state agrees within 1e-9 (relative to
  |F|), component by component and for both parts (pressure, the rest); its
  x component is the drag objective of hfdib_adjoint_grad.
* Wall shear after three sweeps with exact inner solves agrees face by face
  within 1e-9 (relative to max |tau|), on a k-omega SST and a k-epsilon
  backward-facing step, including the closed faces under the step.
* Developed laminar duct flow on the GPU: tau_w = 6 nu U H / (H^2 + 2 Delta^2).
* Recirculation (hfdib_recirculation, Sec. 3.6) on identical inputs: the
  same cells as the oracle's definition, bit for bit, on the 64 x 16 and the
  1024 x 256 step.
"""
import math

import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O
from oracle import forces as Fo

pytestmark = pytest.mark.gpu

TIGHT = dict(tol=1e-12, max_iter=40000, check_every=20)
EXACT = dict(n_u=600, n_turb=600, p_reltol=1e-15, p_maxiter=4000)


def gpu_converged(case, **opts):
    from paper_2606_06135_gb300.hfdib import Solver
    s = Solver(case, **opts)
    rc, it, res = s.solve(**TIGHT)
    assert rc == 0, (rc, it, res)
    return s


def oracle_converged(case, tol=1e-13):
    o = O.Oracle(case)
    it, res = o.solve(tol=tol, max_iter=8000)
    assert o.max_residual(res) <= tol
    o.imposed_fields()
    return o


FORCE_CASES = {
    "box15_laminar": lambda: G.case_rotated_box(15.0, 16, model="laminar", Re=20.0),
    "grf_keps_32x16": lambda: G.case_grf(32, 16, seed=1),
    "cylinder_keps_48x24": lambda: G.case_cylinder(48, 24),
}


@pytest.mark.parametrize("name", sorted(FORCE_CASES))
def test_force_matches_oracle(name):
    case = FORCE_CASES[name]()
    o = oracle_converged(case)
    Fn_o, Ft_o = Fo.ib_force(o)
    s = gpu_converged(case)
    Fn, Ft = s.force()
    scale = np.abs(Fn_o + Ft_o).max()
    print("%s: F gpu %s oracle %s" % (name, Fn + Ft, Fn_o + Ft_o))
    assert np.abs(Fn - Fn_o).max() <= 1e-9 * scale
    assert np.abs(Ft - Ft_o).max() <= 1e-9 * scale
    # C_d, C_l with the default reference area l_ref * dz
    A_ref = case["l_ref"] * case["grid"]["dz"]
    Cd, Cl = s.force_coefficients()
    Cd_o, Cl_o = Fo.force_coefficients(Fn_o + Ft_o, A_ref, case["u_in"])
    assert abs(Cd - Cd_o) <= 1e-9 * (abs(Cd_o) + abs(Cl_o))
    assert abs(Cl - Cl_o) <= 1e-9 * (abs(Cd_o) + abs(Cl_o))
    # a rotated lift direction and an explicit reference area (Eq. dlcoeffs)
    Cd, Cl = s.force_coefficients(A_ref=0.7, gamma=0.3)
    Cd_o, Cl_o = Fo.force_coefficients(Fn_o + Ft_o, 0.7, case["u_in"], gamma=0.3)
    assert abs(Cd - Cd_o) <= 1e-9 * (abs(Cd_o) + abs(Cl_o))
    assert abs(Cl - Cl_o) <= 1e-9 * (abs(Cd_o) + abs(Cl_o))
    # hfdib_ib_force leaves the state a fixed point: the next sweep's residual stays converged
    res = s.sweep()
    assert max(res[:4]) <= 1e-11
    s.close()


def test_force_x_is_the_drag_objective():
    s = gpu_converged(G.case_grf(32, 16, seed=1))
    Fn, Ft = s.force()
    J = s.objective("drag")
    assert abs((Fn[0] + Ft[0]) - J) <= 1e-12 * abs(J)
    s.close()


def test_force_on_no_body_is_zero():
    from paper_2606_06135_gb300.hfdib import Solver
    s = Solver(G.case_uniform(32, 16, model="laminar"))
    s.sweep(3)
    Fn, Ft = s.force()
    assert np.all(Fn == 0.0) and np.all(Ft == 0.0)
    s.close()


SHEAR_CASES = {
    "bfs_sst_64x16": lambda: G.case_bfs(64, 16),
    "bfs_keps_64x16": lambda: G.case_bfs(64, 16, model="kepsilon"),
}


@pytest.mark.parametrize("name", sorted(SHEAR_CASES))
def test_wall_shear_matches_oracle(name):
    from paper_2606_06135_gb300.hfdib import Solver
    case = SHEAR_CASES[name]()
    o = O.Oracle(case)
    s = Solver(case, **EXACT)
    for _ in range(3):
        o.sweep()
        s.sweep()
    o.imposed_fields()
    ref = Fo.wall_shear(o, "ymin")
    got = s.wall_shear("ymin").cpu().numpy()
    assert got.shape == ref.shape
    # the faces under the step are closed: exactly zero on both sides
    assert np.array_equal(got == 0.0, ref == 0.0)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    s.close()


def duct_case(nx=64, ny=8, L=8.0, H=1.0, Re=10.0):
    g = G.make_grid(nx, ny, 1, 0.0, 0.0, L, H)
    X, _, _ = G.cell_centres(g)
    far = np.full(X.shape, 1e3)
    return G._base_case("duct", g, far, far, "laminar", Re,
                        G.bc2d(ymin="wall", ymax="wall"), lt_in=0.1)


def test_developed_duct_wall_shear_closed_form():
    H, ny, Re = 1.0, 8, 10.0
    case = duct_case(ny=ny, H=H, Re=Re)
    s = gpu_converged(case)
    nu = case["u_ref"] * case["l_ref"] / Re
    dy = H / ny
    expect = 6.0 * nu * 1.0 * H / (H * H + 2.0 * dy * dy)
    g = case["grid"]
    xs = g["x0"] + (np.arange(g["nx"]) + 0.5) * g["dx"]
    sel = (xs > 4.0) & (xs < 6.0)
    for side in ("ymin", "ymax"):
        tau = s.wall_shear(side).cpu().numpy()
        assert tau.shape == (3, g["nx"])
        assert np.abs(tau[0][sel] - expect).max() <= 1e-7 * expect
        assert np.all(tau[1] == 0.0) and np.all(tau[2] == 0.0)
    s.close()


def test_wall_shear_rejects_non_wall_sides():
    from paper_2606_06135_gb300.hfdib import HfdibError, Solver
    s = Solver(duct_case(nx=16, ny=4))
    for side in ("xmin", "xmax", 7):
        with pytest.raises(HfdibError):
            s.wall_shear(side)
    s.close()
    s = Solver(G.case_cylinder(32, 16))
    with pytest.raises(HfdibError):
        s.wall_shear("ymin")          # slip, not a wall
    with pytest.raises(HfdibError):
        s.wall_shear("zmin")          # beyond a 2D grid
    s.close()


def test_recirculation_matches_oracle_on_the_same_state():
    """Integer decisions (u_x < 0, x_c > x_rear) on identical inputs: the
    oracle's converged step loaded into the GPU solver gives the same cells,
    hence the same count, volume and length, bit for bit."""
    from paper_2606_06135_gb300.hfdib import Solver
    case = G.case_bfs(64, 16, model="komegasst")
    o = oracle_converged(case, tol=1e-8)
    s = Solver(case)
    for name, val in (("ux", o.u[0]), ("uy", o.u[1]), ("p", o.p), ("k", o.k), ("omega", o.omega)):
        s.set_field(name, val)
    for x_rear in (0.0, 1.0, 1e9):
        got = s.recirculation(x_rear)
        ref = Fo.recirculation(o, x_rear)
        assert got[2] == ref[2] and got[0] == ref[0] and got[1] == ref[1], (x_rear, got, ref)
    assert s.recirculation(0.0)[2] > 0
    s.close()


class _State:
    """The oracle's view (mesh, in-solid mask, velocity) of a GPU state."""
    def __init__(self, case, s):
        self.m = O.Mesh(case["grid"])
        tags, _ = s.tags()
        self.ic = tags == O.TAG_IC
        f = s.fields()
        self.u = [f["ux"], f["uy"]]


def test_recirculation_on_the_full_step():
    """1024 x 256 step after 2000 sweeps: the GPU metric equals the oracle's
    definition applied to the GPU's own fields."""
    from paper_2606_06135_gb300.hfdib import Solver
    case = G.case_bfs(1024, 256)
    s = Solver(case, precision=1, freeze_switch=300)
    s.sweep(2000, read=False)
    st = _State(case, s)
    got = s.recirculation(0.0)
    ref = Fo.recirculation(st, 0.0)
    assert got[2] == ref[2] and got[0] == ref[0] and got[1] == ref[1], (got, ref)
    assert got[2] > 100
    s.close()


def test_force_with_linear_upwind_matches_oracle():
    """The force includes the deferred convection correction of the imposed
    rows' momentum (App. B scheme)."""
    case = G.case_rotated_box(15.0, 16, model="laminar", Re=20.0)
    o = O.Oracle(case, dict(convection="linearUpwind"))
    it, res = o.solve(tol=1e-13, max_iter=8000)
    assert o.max_residual(res) <= 1e-13
    o.imposed_fields()
    Fref = sum(Fo.ib_force(o))
    s = gpu_converged(case, convection=1)
    F = sum(s.force())
    assert np.abs(F - Fref).max() <= 1e-9 * np.abs(Fref).max()
    s.close()
