"""Pins of the oracle's Wilcox k-omega (Eq. hfdibkomega) and realizable
k-epsilon models against closed forms.

* Decaying homogeneous turbulence (lambda == 0, uniform flow, no shear):
  k-omega gives omega = 1/(beta (t + t0)) and k ~ (t + t0)^(-beta*/beta);
  realizable k-eps with nu -> 0 gives k ~ (t + t0)^(-1/(C2 - 1)) and, with
  no strain, C_mu = 1/A0.
* The realizable C_mu coefficients for pure shear, plane strain, axisymmetric
  strain and solid-body rotation (Shih et al.: A_s = sqrt(6) cos(phi),
  phi = arccos(sqrt(6) W)/3).
* Both models converge with immersed bodies, and keep the mirror symmetry of
  a cylinder in a symmetric channel.
"""
import math

import numpy as np
import pytest

from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O


def decayed(model, nx=400, sweeps=900):
    case = G.case_uniform(nx, 4, Re=1e8, I_in=0.1, model=model)
    case["lt_in"] = 0.02
    o = O.Oracle(case)
    for _ in range(sweeps):
        res = o.sweep()
    w = "omega" if model == "komega" else "eps"
    assert res["k"] <= 1e-12 and res[w] <= 1e-12, res
    X, _, _ = G.cell_centres(case["grid"])
    return o, X[0, 0]


def fit_exponent(t, k, t0):
    sel = (t > 0.5) & (t < 1.8)
    return -np.polyfit(np.log(t[sel] + t0), np.log(k[sel]), 1)[0]


def test_komega_homogeneous_decay():
    o, t = decayed("komega")
    c = O.KW
    t0 = 1.0 / (c["beta"] * o.omega_in)
    expo = c["bstar"] / c["beta"]
    got = fit_exponent(t, o.k[0, 0], t0)
    assert abs(got - expo) <= 5e-3 * expo, (got, expo)
    # d omega/dt = -beta omega^2: omega (t + t0) beta = 1
    sel = (t > 0.5) & (t < 1.8)
    prod = o.omega[0, 0][sel] * (t[sel] + t0) * c["beta"]
    assert np.abs(prod - 1.0).max() <= 5e-3, prod
    # nu_t = k/omega, eps = C_mu k omega
    np.testing.assert_allclose(o.nut, o.k / o.omega, rtol=1e-14)
    np.testing.assert_allclose(o.eps, O.C_MU * o.k * o.omega, rtol=1e-14)


def test_realizable_ke_homogeneous_decay():
    o, t = decayed("realizableke")
    c = O.RKE
    t0 = o.k_in / ((c["C2"] - 1.0) * o.eps_in)
    expo = 1.0 / (c["C2"] - 1.0)
    got = fit_exponent(t, o.k[0, 0], t0)
    assert abs(got - expo) <= 5e-3 * expo, (got, expo)
    # the standard model's exponent is 2 % away: the pin tells them apart
    assert abs(got - 1.0 / (O.KE_C2 - 1.0)) > 1e-2 * expo
    # no strain: C_mu = 1/A0
    # (rounding-level strain in the uniform flow moves it by ~1e-13)
    np.testing.assert_allclose(o.nut, o.k ** 2 / (c["A0"] * o.eps), rtol=1e-11)


def rke_at(G3):
    """A_s U* and S of one velocity gradient G3[a][b] = d u_b/d x_a."""
    d = len(G3)
    case = G.case_uniform(4, 4) if d == 2 else G.case_sphere(4, 4, 4)
    o = O.Oracle(case)
    Gf = [[np.full(o.m.shape, float(G3[a][b])) for b in range(d)] for a in range(d)]
    AsUs, S = o.rke_coefficients(Gf)
    return float(AsUs.ravel()[0]), float(S.ravel()[0])


def test_realizable_cmu_closed_forms():
    s = 0.8
    # pure shear u = (s y, 0): W = 0, A_s = 3/sqrt(2), U* = s, S = s
    AsUs, S = rke_at([[0.0, 0.0], [s, 0.0]])
    assert abs(AsUs - 3.0 / math.sqrt(2.0) * s) <= 1e-14
    assert abs(S - s) <= 1e-15
    # plane strain u = (a x, -a y): W = 0, U* = sqrt(2) a, S = 2 a
    a = 0.3
    AsUs, S = rke_at([[a, 0.0], [0.0, -a]])
    assert abs(AsUs - 3.0 / math.sqrt(2.0) * math.sqrt(2.0) * a) <= 1e-14
    assert abs(S - 2.0 * a) <= 1e-15
    # axisymmetric strain diag(2a, -a, -a): sqrt(6) W = 1, phi = 0, A_s = sqrt(6), U* = sqrt(6) a
    AsUs, S = rke_at([[2 * a, 0.0, 0.0], [0.0, -a, 0.0], [0.0, 0.0, -a]])
    assert abs(AsUs - 6.0 * a) <= 1e-14
    # its mirror diag(-2a, a, a): sqrt(6) W = -1, phi = pi/3, A_s = sqrt(6)/2
    AsUs, S = rke_at([[-2 * a, 0.0, 0.0], [0.0, a, 0.0], [0.0, 0.0, a]])
    assert abs(AsUs - 3.0 * a) <= 1e-14
    # solid-body rotation: S = 0 (W taken as 0), U* = |Omega| = sqrt(2) w
    w = 0.5
    AsUs, S = rke_at([[0.0, w], [-w, 0.0]])
    assert S == 0.0
    assert abs(AsUs - 3.0 / math.sqrt(2.0) * math.sqrt(2.0) * w) <= 1e-14


@pytest.mark.parametrize("model", ["komega", "realizableke"])
def test_model_converges_with_a_body_and_keeps_symmetry(model):
    case = G.case_cylinder(32, 16, model=model)
    o = O.Oracle(case)
    it, res = o.solve(tol=1e-10, max_iter=3000)
    assert o.max_residual(res) <= 1e-10, (it, res)
    ux, uy, k = o.u[0][0], o.u[1][0], o.k[0]
    assert np.abs(ux - ux[::-1]).max() < 1e-8
    assert np.abs(uy + uy[::-1]).max() < 1e-8
    assert np.abs(k - k[::-1]).max() < 1e-8 * k.max()
    # k = 0 in the solid (k_ib of ic cells), positive in the fluid
    assert np.all(o.nut >= 0.0) and np.all(o.k >= 0.0) and np.all(o.k[~o.ic] > 0.0)
