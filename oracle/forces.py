"""Force on the immersed body, force coefficients and wall shear stress, FP64.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference arm may import this module; the product path never
does and shares no code with it.

Force (Eq. dragcoeff, Eq. dlcoeffs).  The paper integrates the surface
traction f_tot = f_n + f_t over the fluid-solid interface Gamma_sf.  On the
HFDIB grid that interface is not a set of faces, so the integral is read
through the momentum balance of the cells whose velocity the immersed boundary
imposes (ic cells and laminar-branch bc cells).  In those rows the discrete
momentum equation holds only with the forcing f_ib of Eq. hfdibrans_1 added,
so f_ib V is the row residual at the imposed values ut,

    r_q = aP ut_P + sum_N a_N ut_N - b0_q + V dp/dx_q,

and the force of the fluid on the body is -sum r over those rows: the
reaction to the forcing.  Its interior faces cancel, so it is the flux of
momentum through the faces that bound the imposed cells.
  * F_n = -sum V dp/dx_q is the pressure part (the Gauss gradient sums to
    p_f S_f n over those faces): the f_n term.
  * F_t = the rest: viscous stress, plus the convective momentum flux through
    those faces.  It stands in for the f_t term.
The density drops out (kinematic pressure).  The coefficients are then
C_d = 2 F.v_d / (A_ref |u_in|^2) and C_l = 2 F.v_l / (A_ref |u_in|^2), with
v_d = (1, 0, 0) and v_l = (-sin gamma, cos gamma, 0).

Wall shear stress (Sec. 3.3).  The paper's definition is nu du_x/dy at the
wall.  Along a no-slip domain wall it is read as the shear the discrete
momentum equation applies at the wall face: nu_eff,P (u_P - u_wall)/(Delta/2)
for each tangential component, with nu_eff,P = nu + nu_t,P as on the face.
C_f = 2 tau_w / |u_in|^2.  The reattachment point is the downstream end of
the main recirculation: the last sign change of tau_x from negative to
positive, located by linear interpolation between cell centres.

Recirculation region (Sec. 3.6): the cells with negative u_x behind the body.
Read as cells outside the solid (not ic) whose centre lies downstream of the
body's rear end x_rear; its length is the largest distance from x_rear to
such a cell centre, its volume the sum of their volumes.
"""
from __future__ import annotations

import math

import numpy as np

from . import hfdib_oracle as O


def imposed_rows(o):
    """Cells whose momentum row the immersed boundary imposes: ic cells and
    bc cells in the laminar branch (alpha_u = 1)."""
    return o.alpha_u > 0.5


def imposed_velocity(o, c):
    """Velocity component c with the imposed value in the imposed rows (u_s in
    ic, u_ib in laminar-branch bc cells) and u elsewhere."""
    return np.where(imposed_rows(o), o.u_ib[c], o.u[c])


def ib_force(o):
    """(F_n, F_t): the pressure part and the rest of the force of the fluid on
    the body, each a length-3 array (zero beyond the grid's dimensions), at
    the oracle's current state (the rows of its next sweep)."""
    m = o.m
    fixed = imposed_rows(o)
    nu_eff = o.nu + o.nut
    G = o.velocity_grad(o.u)
    gradp = O.gauss_grad(m, o.p, o.bnd.pressure_spec())
    Fn = np.zeros(3)
    Ft = np.zeros(3)
    for c in range(m.dims):
        ut = imposed_velocity(o, c)
        aP, aM, aPl, b = O.assemble_transport(m, o.phi, nu_eff, o.bnd.velocity_spec(c))
        b = b + o.transpose_source(G, nu_eff, c) + o.momentum_convection_correction(G, c)
        rm = aP * ut + O.apply_offdiag(m, aM, aPl, ut) - b
        Ft[c] = -float(np.sum(rm[fixed]))
        Fn[c] = -float(np.sum((m.V * gradp[c])[fixed]))
    return Fn, Ft


def force_coefficients(F, A_ref, u_in, gamma=0.0):
    """(C_d, C_l) of Eqs. dragcoeff and dlcoeffs from the total force F."""
    F = np.asarray(F, dtype=np.float64)
    q = 0.5 * A_ref * float(np.dot(u_in, u_in))
    vd = np.array([1.0, 0.0, 0.0])
    vl = np.array([-math.sin(gamma), math.cos(gamma), 0.0])
    return float(F @ vd) / q, float(F @ vl) / q


SIDES = ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")


def wall_shear(o, side):
    """tau_w on the faces of one no-slip domain side: array [3, n_faces] (the
    component normal to the wall is zero), faces in the order of the cells
    next to the wall (x fastest, then y, then z)."""
    m = o.m
    s = SIDES.index(side)
    d, hi = s >> 1, s & 1
    if d >= m.dims or o.bnd.kind[(d, hi)] != "wall":
        raise ValueError("not a no-slip domain wall: %s" % side)
    nu_eff = m.slab(o.nu + o.nut, d, hi)
    # a closed face (wall inside the solid) carries no flux
    open_ = ~o.bnd.closed[(d, hi)]
    tau = np.zeros((3,) + nu_eff.shape)
    for c in range(m.dims):
        if c == d:
            continue
        uP = m.slab(imposed_velocity(o, c), d, hi)
        tau[c] = np.where(open_, nu_eff * uP / (0.5 * m.D[d]), 0.0)
    return tau.reshape(3, -1)


def reattachment(x, tau_x):
    """x of the last sign change of tau_x from negative to positive (linear
    interpolation between the two cell centres), or None."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(tau_x, dtype=np.float64)
    idx = np.flatnonzero((t[:-1] < 0.0) & (t[1:] >= 0.0))
    if idx.size == 0:
        return None
    i = int(idx[-1])
    return float(x[i] - t[i] * (x[i + 1] - x[i]) / (t[i + 1] - t[i]))


def recirculation(o, x_rear):
    """(length, volume, cells) of the recirculation region behind x_rear."""
    m = o.m
    X = m.x0 + (np.arange(m.nx) + 0.5) * m.dx
    X = np.broadcast_to(X[None, None, :], m.shape)
    sel = (~o.ic) & (X > x_rear) & (o.u[0] < 0.0)
    n = int(sel.sum())
    length = float((X[sel] - x_rear).max()) if n else 0.0
    return length, n * m.V, n
