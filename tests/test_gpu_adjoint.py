"""Frozen-turbulence adjoint on the GPU (hfdib_adjoint_grad) against the
oracle's sparse complex-step adjoint and against central finite differences
of frozen-turbulence GPU solves.

* dJ/dlambda of the GPU reverse sweep equals the oracle's gradient of the
  same discrete equations (each side at its own converged state).
* The gradient does not depend on how the sweep is iterated: the reverse pass
  of a sweep with 1, 2 or 3 red-black momentum passes gives the same gradient
  on one state (the fixed point, not the iteration, is differentiated).
* Central differences of J over frozen-turbulence GPU solves agree within 1e-4
  relative.
* The torch.autograd.Function delivers the same gradient to lambda.grad.
"""
import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O
from oracle import adjoint as A

pytestmark = pytest.mark.gpu

TIGHT = dict(tol=1e-12, max_iter=40000, check_every=20)


def gpu_converged(case, **opts):
    from paper_2606_06135_gb300.hfdib import Solver
    s = Solver(case, **opts)
    rc, it, res = s.solve(**TIGHT)
    assert rc == 0, (rc, it, res)
    return s


def oracle_gradient(case):
    o = O.Oracle(case)
    it, res = o.solve(tol=1e-13, max_iter=6000)
    assert o.max_residual(res) <= 1e-13
    fs = A.FrozenSteady(o)
    assert fs.n_kinks == 0
    J, g, _ = fs.gradient()
    return J, g.ravel()


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = {
    "grf_keps_32x16": lambda: G.case_grf(32, 16, seed=1),
    "box15_laminar": lambda: G.case_rotated_box(15.0, 16, model="laminar", Re=20.0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_adjoint_gradient_matches_oracle(name):
    case = CASES[name]()
    Jo, go = oracle_gradient(case)
    s = gpu_converged(case)
    J, g, it, ch, rc = s.adjoint_grad(tol=1e-12, max_iter=40000)
    assert rc == 0, (it, ch)
    g = g.cpu().numpy().ravel()
    e = rel(g, go)
    print("%s: J gpu %.15f oracle %.15f, grad rel-L2 %.2e, %d adjoint iterations" % (name, J, Jo, e, it))
    assert abs(J - Jo) <= 1e-10 * abs(Jo)
    assert e <= 1e-10
    # the support is the same: only cells that move an imposed velocity
    assert set(np.flatnonzero(np.abs(go) > 1e-12 * np.abs(go).max())) <= set(np.flatnonzero(g))
    s.close()


def test_gmres_and_reverse_fixed_point_agree():
    """GMRES on (I - G_x^T) psi = J_x^T with exact pressure solves and the
    reverse fixed point psi <- G_x^T psi + J_x^T with warm-started loose ones
    reach the same adjoint."""
    case = G.case_grf(32, 16, seed=1)
    s = gpu_converged(case)
    _, gk, itk, chk, rck = s.adjoint_grad(tol=1e-11, max_iter=4000, gmres_restart=40)
    _, gf, itf, chf, rcf = s.adjoint_grad(tol=1e-12, max_iter=40000, gmres_restart=0)
    assert rck == 0 and rcf == 0, (itk, chk, itf, chf)
    print("GMRES(40): %d transposed sweeps (residual %.1e); fixed point: %d (change %.1e)" % (itk, chk, itf, chf))
    assert rel(gk.cpu().numpy(), gf.cpu().numpy()) <= 1e-9
    s.close()


def test_gradient_independent_of_inner_sweeps():
    from paper_2606_06135_gb300.hfdib import Solver
    case = G.case_grf(32, 16, seed=1)
    base = gpu_converged(case)
    st = base.get_state()
    grads = []
    for n_u in (1, 2, 3):
        s = Solver(case, n_u=n_u)
        s.set_state(st)
        J, g, it, ch, rc = s.adjoint_grad(tol=1e-12, max_iter=40000)
        assert rc == 0, (n_u, it, ch)
        grads.append(g.cpu().numpy().ravel())
        s.close()
    base.close()
    assert rel(grads[0], grads[1]) <= 1e-9
    assert rel(grads[2], grads[1]) <= 1e-9


def test_adjoint_matches_gpu_finite_differences():
    from paper_2606_06135_gb300.hfdib import Solver
    case = G.case_grf(32, 16, seed=1)
    base = gpu_converged(case)
    J0, g, it, ch, rc = base.adjoint_grad(tol=1e-12, max_iter=40000)
    assert rc == 0
    g = g.cpu().numpy().ravel()
    st = base.get_state()
    tags0, _ = base.tags()
    lam = case["lam"].ravel()
    cut = np.flatnonzero((lam > 0.05) & (lam < 0.95))
    pick = cut[np.argsort(-np.abs(g[cut]))[:2]]
    delta = 1e-6
    for c in pick:
        Js = []
        for sgn in (1.0, -1.0):
            cs = dict(case)
            cs["lam"] = case["lam"].copy()
            cs["lam"].reshape(-1)[c] += sgn * delta
            s = Solver(cs, frozen_turbulence=1)
            tags, _ = s.tags()
            assert np.array_equal(tags, tags0)
            s.set_state(st)
            rc, it2, res = s.solve(**TIGHT)
            assert rc == 0, (rc, it2, res)
            Js.append(s.objective())
            s.close()
        fd = (Js[0] - Js[1]) / (2 * delta)
        print("cell %d: adjoint %.10e fd %.10e" % (c, g[c], fd))
        assert abs(fd - g[c]) <= 1e-4 * abs(fd)
    base.close()


def test_mixed_precision_handle_differentiates_the_fp64_sweep():
    from paper_2606_06135_gb300.hfdib import Solver
    case = G.case_grf(32, 16, seed=1)
    a = gpu_converged(case)
    st = a.get_state()
    b = Solver(case, precision=1)
    b.set_state(st)
    _, ga, _, _, rca = a.adjoint_grad(tol=1e-12, max_iter=40000)
    _, gb, _, _, rcb = b.adjoint_grad(tol=1e-12, max_iter=40000)
    assert rca == 0 and rcb == 0
    assert rel(gb.cpu().numpy(), ga.cpu().numpy()) <= 1e-9
    a.close()
    b.close()


def test_autograd_function_delivers_the_gradient():
    import torch
    from paper_2606_06135_gb300.autograd import pressure_drop
    case = G.case_grf(32, 16, seed=1)
    lam = torch.tensor(case["lam"], dtype=torch.float64, device="cuda", requires_grad=True)
    J = pressure_drop(lam, case, solve_tol=1e-12, adj_tol=1e-11)
    J.backward()
    s = gpu_converged(case)
    Jd, g, _, _, rc = s.adjoint_grad(tol=1e-12, max_iter=40000)
    assert rc == 0
    assert abs(J.item() - Jd) <= 1e-12 * abs(Jd)
    assert rel(lam.grad.cpu().numpy(), g.cpu().numpy()) <= 1e-9
    s.close()


@pytest.mark.parametrize("golden_name", ["adjoint3d_sphere.txt", "adjoint3d_sphere_drag.txt",
                                         "adjoint3d_sphere_keps_drag.txt"])
def test_3d_gradient_matches_oracle(golden_name):
    """3D (trilinear stencils, 26-neighbour normals): the GPU adjoint of a
    sphere placed off the grid's symmetry planes against the oracle's, for the
    pressure drop and the drag (laminar) and the drag with frozen k-epsilon
    turbulence (goldens written from oracle/ alone by
    tests/golden/make_adjoint3d.py)."""
    import importlib.util
    import os
    golden = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location("make_adjoint3d", os.path.join(golden, "make_adjoint3d.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    model, Re, objective = mk.GOLDENS[golden_name]
    case = mk.sphere_off_axis(model, Re)
    vals = np.loadtxt(os.path.join(golden, golden_name))
    Jo, go = vals[0], vals[1:]
    s = gpu_converged(case)
    J, g, it, ch, rc = s.adjoint_grad(tol=1e-12, max_iter=40000, objective=objective)
    assert rc == 0, (it, ch)
    g = g.cpu().numpy().ravel()
    e = rel(g, go)
    print("3D sphere %s: J gpu %.15f oracle %.15f, grad rel-L2 %.2e, %d adjoint iterations"
          % (golden_name, J, Jo, e, it))
    assert abs(J - Jo) <= 1e-10 * abs(Jo)
    assert e <= 1e-9
    s.close()


def test_adjoint_rejects_unknown_objective_and_other_schemes():
    from paper_2606_06135_gb300.hfdib import HfdibError, Solver
    s = Solver(G.case_grf(32, 16, seed=1))
    with pytest.raises(HfdibError):
        s.adjoint_grad(max_iter=10, objective=7)
    s.close()
    s = Solver(G.case_grf(32, 16, seed=1), convection=1)
    with pytest.raises(HfdibError):
        s.adjoint_grad(max_iter=10)
    s.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_drag_gradient_matches_oracle(name):
    """Drag (minus the immersed-boundary forcing of the imposed rows): value
    and dJ/dlambda = J_lambda - psi^T R_lambda against the oracle."""
    case = CASES[name]()
    o = O.Oracle(case)
    it, res = o.solve(tol=1e-13, max_iter=6000)
    assert o.max_residual(res) <= 1e-13
    fs = A.FrozenSteady(o, "drag")
    Jo, go, _ = fs.gradient()
    go = go.ravel()
    s = gpu_converged(case)
    J, g, it, ch, rc = s.adjoint_grad(tol=1e-12, max_iter=40000, objective="drag")
    assert rc == 0, (it, ch)
    g = g.cpu().numpy().ravel()
    e = rel(g, go)
    print("%s drag: J gpu %.15f oracle %.15f, grad rel-L2 %.2e, %d iterations" % (name, J, Jo, e, it))
    assert abs(J - Jo) <= 1e-9 * abs(Jo)
    assert abs(s.objective("drag") - J) <= 1e-14 * abs(J)
    assert e <= 1e-10
    s.close()


def test_autograd_drag_delivers_the_gradient():
    import torch
    from paper_2606_06135_gb300.autograd import drag
    case = G.case_grf(32, 16, seed=1)
    lam = torch.tensor(case["lam"], dtype=torch.float64, device="cuda", requires_grad=True)
    J = drag(lam, case, solve_tol=1e-12, adj_tol=1e-12)
    J.backward()
    s = gpu_converged(case)
    Jd, g, _, _, rc = s.adjoint_grad(tol=1e-12, max_iter=40000, objective="drag")
    assert rc == 0
    assert abs(J.item() - Jd) <= 1e-12 * abs(Jd)
    assert rel(lam.grad.cpu().numpy(), g.cpu().numpy()) <= 1e-9
    s.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_reading_b_gradient_matches_oracle(name):
    """Reading B of the continuity mask (m = 1 - lambda): the converged states
    and the gradients, which now include ps div(phiHbyA) in every cell, agree
    with the oracle's residual-form adjoint."""
    from paper_2606_06135_gb300.hfdib import Solver
    case = CASES[name]()
    o = O.Oracle(case, dict(continuity_mask="B"))
    it, res = o.solve(tol=1e-13, max_iter=6000)
    assert o.max_residual(res) <= 1e-13
    fs = A.FrozenSteady(o)
    assert fs.n_kinks == 0
    Jo, go, _ = fs.gradient()
    go = go.ravel()
    s = gpu_converged(case, continuity_mask=1)
    J, g, it, ch, rc = s.adjoint_grad(tol=1e-12, max_iter=40000)
    assert rc == 0, (it, ch)
    g = g.cpu().numpy().ravel()
    e = rel(g, go)
    print("%s reading B: J gpu %.15f oracle %.15f, grad rel-L2 %.2e, %d iterations" % (name, J, Jo, e, it))
    assert abs(J - Jo) <= 1e-10 * abs(Jo)
    assert e <= 1e-10
    # the gradient reaches the fluid far from the body
    assert np.count_nonzero(g) > 0.9 * g.size
    s.close()


def test_batched_autograd_matches_single_designs():
    """pressure_drops: two designs of different size solved as one batch; the
    gradients of sum(J) are each design's own adjoint gradient."""
    import torch
    from paper_2606_06135_gb300.autograd import pressure_drop, pressure_drops
    cases = [G.case_grf(32, 16, seed=1), G.case_grf(40, 20, seed=2)]
    lams = [torch.tensor(c["lam"], dtype=torch.float64, device="cuda", requires_grad=True) for c in cases]
    J = pressure_drops(lams, cases, solve_tol=1e-12, adj_tol=1e-11)
    assert J.shape == (2,)
    J.sum().backward()
    for c, lam, Jb in zip(cases, lams, J.detach().cpu().numpy()):
        ls = torch.tensor(c["lam"], dtype=torch.float64, device="cuda", requires_grad=True)
        Js = pressure_drop(ls, c, solve_tol=1e-12, adj_tol=1e-11)
        Js.backward()
        assert abs(Js.item() - Jb) <= 1e-10 * abs(Jb)
        assert rel(lam.grad.cpu().numpy(), ls.grad.cpu().numpy()) <= 1e-8
