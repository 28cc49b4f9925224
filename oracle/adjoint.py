"""Frozen-turbulence discrete adjoint of a converged HFDIB-SIMPLE state (oracle).

TEST INFRASTRUCTURE, like hfdib_oracle: only tests/, the smoke check and the
CPU arms of the benchmark may import it.  Plain FP64 (complex128 for the
complex-step derivatives), numpy/scipy, 2D and 3D grids.

What is differentiated.  A converged state is a fixed point of the extended
SIMPLE sweep (Fig. simplehfdibrans).  Hold fixed the turbulence fields (nu_t,
k, eps/omega), the cell groups (Sec. 2.3), the wall-function branch of each bc
cell (alpha_u, Eq. alphauk), the closed boundary faces, the continuity mask m
(under reading A, m = [lambda < 1]; under reading B, m = 1 - lambda is smooth
and differentiated) and the integer choices of the bc-cell geometry
(in-solid neighbour, y_perp case, interpolation cells, clamps).  The fixed point z = (u, p, phi) then
solves the steady equations R(z; lambda) = 0:

  momentum, every cell and component:
      aavg (u - ut) - rlx aP (u - ut) + aP ut + sum_N a_N ut_N - b0(u, phi)
        + V dp/dx = 0
  pressure:  L(rAU) p + m div(phiHbyA) - b_out = 0
  face flux: phi - [phiHbyA - rAU_f S (p_N - p_P) / Delta] = 0

with ut = u_ib(u; lambda) in imposed rows (ic: u_s; laminar-branch bc cells:
the quadratic interpolation along n, Sec. 2.5) and ut = u elsewhere,
rlx = (1 - alpha_u_relax)/alpha_u_relax, aavg the component-averaged relaxed
diagonal and HbyA = (b0 + rlx aP u - sum a_N ut_N - (aP/alpha - aavg) ut)/aavg.
In free rows ut = u and the first line is the steady momentum equation; in
imposed rows it is the velocity update u = HbyA - rAU grad p of a8 at the
fixed point.  Each line is assembled from the oracle's own blocks.

lambda enters R through u_ib: the normal n = -grad(lambda)/|grad(lambda)|
(Eq. yorthoaux), y_perp (Eq. yortho with sigma = h atanh(1 - 2 lambda)) and
through them the interpolation fractions and the quadratic weights; under
reading B also through m in the pressure line.

Objectives.  Pressure drop: J = mean p over the cells on open inlet faces
minus mean p over the cells on outlet faces.  Drag: J = minus the sum over
the imposed rows of the x-momentum row residual aP ut + sum a_N ut_N - b0
+ V dp/dx, the forcing the immersed boundary applies to the fluid there (the
divergence-form terms telescope to fluxes through the boundary of the imposed
region, so this is the force of the fluid on the body).  The adjoint psi
solves R_z^T psi = J_z^T and dJ/dlambda = J_lambda - psi^T R_lambda (J_lambda
is zero for the pressure drop; for the drag it is the explicit dependence
through u_ib).  R_z and R_lambda are
exact sparse Jacobians from complex-step derivatives (imaginary step 1e-20),
one evaluation of R per colour of a distance colouring of the grid.

Parity pinned by: R(z*) = 0 at the oracle's converged sweep fixed point; the
colouring against single complex-step Jacobian-vector products; the
geometry restatement against ib_geometry; dJ/dlambda against central finite
differences of frozen-turbulence solves.
"""
from __future__ import annotations

import copy

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import hfdib_oracle as O

H_CS = 1e-20     # complex-step size (no subtraction, so any tiny step is exact)
REACH = 6        # cells over which one entry of z or lambda can change a row of R


def _absr(x):
    """|x| by the sign of the real part (complex-step safe)."""
    return x if x.real >= 0 else -x


def _normal(m, lam, i, j, k):
    """n = -grad(lambda)/|grad(lambda)| (Eq. yorthoaux); where the real-valued
    gradient vanishes the oracle's fall-back normal (a constant) is used."""
    nr, fb = O.surface_normal(m, lam.real, i, j, k)
    if fb:
        return nr
    gx, gy, gz = O._grad_lambda(m, lam, i, j, k)
    mag = ((gx * gx + gy * gy) + gz * gz) ** 0.5
    return (-gx / mag, -gy / mag, -gz / mag)


def bc_weights(m, lam, geo):
    """Normal, y_perp, interpolation fractions and quadratic weights of the bc
    cells recomputed from lambda (real or complex) with the integer choices of
    `geo` (from hfdib_oracle.ib_geometry) held fixed."""
    cells = geo["cell"]
    nb = len(cells)
    dt = np.result_type(lam.dtype, np.float64)
    out = dict(n=np.zeros((nb, 3), dt), y_perp=np.zeros(nb, dt), t1=np.zeros((nb, 3), dt),
               t2=np.zeros((nb, 3), dt), wS=np.zeros(nb, dt), w1=np.zeros(nb, dt), w2=np.zeros(nb, dt))
    h = m.h
    for q, c in enumerate(cells):
        k, rem = divmod(int(c), m.ny * m.nx)
        j, i = divmod(rem, m.nx)
        P = m.centre(i, j, k)
        nP = tuple(geo["n"][q]) if geo["fallback"][q] else _normal(m, lam, i, j, k)
        case = geo["case"][q]
        if geo["clamped"][q]:
            yp = 1e-3 * h
        elif case == 0:
            yp = _absr(h * np.arctanh(1.0 - 2.0 * lam[k, j, i]))
        elif case == 1:
            kk, r2 = divmod(int(geo["nbr"][q]), m.ny * m.nx)
            jj, ii = divmod(r2, m.nx)
            nN = _normal(m, lam, ii, jj, kk)
            sN = _absr(h * np.arctanh(1.0 - 2.0 * lam[kk, jj, ii]))
            Nc = m.centre(ii, jj, kk)
            Q = [Nc[d] + sN * nN[d] for d in range(3)]
            yp = (nN[0] * (P[0] - Q[0]) + nN[1] * (P[1] - Q[1])) + nN[2] * (P[2] - Q[2])
        else:
            yp = geo["y_perp"][q]
        out["n"][q] = nP
        out["y_perp"][q] = yp
        for key, base, dist in (("t1", geo["base1"][q], h), ("t2", geo["base2"][q], 2.0 * h)):
            for d in range(3):
                if m.n[d] == 1:
                    continue
                xi = (P[d] + dist * nP[d] - m.o[d]) / m.D[d] - 0.5
                td = xi - base[d]
                if td.real < 0.0:
                    td = 0.0
                elif td.real > 1.0:
                    td = 1.0
                out[key][q, d] = td
        d1 = yp + h
        d2 = yp + 2.0 * h
        out["wS"][q] = ((yp - d1) * (yp - d2)) / ((0.0 - d1) * (0.0 - d2))
        out["w1"][q] = ((yp - 0.0) * (yp - d2)) / ((d1 - 0.0) * (d1 - d2))
        out["w2"][q] = ((yp - 0.0) * (yp - d1)) / ((d2 - 0.0) * (d2 - d1))
    return out


class FrozenSteady:
    """The steady equations R(z; lambda) around a converged oracle state `o`
    (an hfdib_oracle.Oracle whose sweeps have converged)."""

    def __init__(self, o, objective="pressure_drop"):
        if objective not in ("pressure_drop", "drag"):
            raise ValueError("objective: pressure_drop or drag")
        self.kind = objective
        m = o.m
        if o.opts.get("convection", "upwind") != "upwind":
            raise ValueError("the oracle adjoint covers the upwind scheme")
        self.o = copy.deepcopy(o)
        o = self.o
        o.imposed_fields()          # branch and masks the next sweep would use
        self.m = m
        self.lam0 = o.lam.copy()
        self.geo = o.geo
        self.sel = o.lam_branch.copy() if o.model != "laminar" else np.ones(len(o.geo["cell"]), bool)
        self.nu_eff = o.nu + o.nut
        # imposed rows: ic cells and the laminar-branch bc cells
        fixed = o.ic.copy()
        fixed.reshape(-1)[o.geo["cell"][self.sel]] = True
        self.fixed = fixed
        shapes = [m.shape] * m.dims + [m.shape]
        for d in range(m.dims):
            shp = list(m.shape)
            shp[2 - d] += 1
            shapes.append(tuple(shp))
        self.shapes = shapes
        self.sizes = [int(np.prod(s)) for s in shapes]
        self.offs = np.concatenate([[0], np.cumsum(self.sizes)])
        # objective weights: cells on open inlet faces, cells on outlet faces
        w = np.zeros(m.shape)
        for (d, hi), kind in o.bnd.kind.items():
            if kind not in ("inlet", "outlet"):
                continue
            sl = O._sl(2 - d, m.n[d] - 1, m.n[d]) if hi else O._sl(2 - d, 0, 1)
            sel = np.zeros(m.slab(w, d, hi).shape, bool)
            if kind == "inlet":
                sel = ~o.bnd.closed[(d, hi)]
            else:
                sel[...] = True
            cnt = int(sel.sum())
            if cnt:
                w[sl] += np.where(sel, (1.0 if kind == "inlet" else -1.0) / cnt, 0.0)
        self.jw = w
        # interior faces with (near) zero flux sit on the kink of the upwind
        # switch max(F, 0): J is not differentiable there (a symmetry plane
        # of a symmetric flow is the usual case); dJ/dlambda needs none
        fmax = max(float(np.abs(o.phi[d]).max()) for d in range(m.dims))
        self.n_kinks = 0
        for d in range(m.dims):
            inner = o.phi[d][O._sl(2 - d, 1, m.n[d])]
            self.n_kinks += int(np.sum(np.abs(inner) < 1e-10 * fmax))

    # ---------------------------------------------------------------- packing
    def pack(self, u, p, phi):
        return np.concatenate([np.asarray(a).ravel() for a in list(u) + [p] + list(phi)])

    def unpack(self, z):
        parts = [z[self.offs[b]:self.offs[b + 1]].reshape(self.shapes[b]) for b in range(len(self.shapes))]
        d = self.m.dims
        return parts[:d], parts[d], parts[d + 1:]

    def state(self):
        o = self.o
        return self.pack(o.u[:self.m.dims], o.p, o.phi[:self.m.dims])

    # ---------------------------------------------------------------- equations
    def _momentum_pieces(self, z, lam):
        """ut (u with the imposed values in imposed rows), the momentum rows
        aP, aM, aPl, the explicit right-hand sides b0 and grad p."""
        m, o = self.m, self.o
        lam = self.lam0 if lam is None else lam
        u, p, phi = self.unpack(z)
        geo = dict(self.geo)
        geo.update(bc_weights(m, lam, self.geo))
        cells = geo["cell"][self.sel]
        ut = []
        for c in range(m.dims):
            v1 = O.interp_at(m, u[c], geo["base1"], geo["t1"])
            v2 = O.interp_at(m, u[c], geo["base2"], geo["t2"])
            uib = geo["wS"] * o.u_s[c] + geo["w1"] * v1 + geo["w2"] * v2
            x = np.array(u[c], dtype=np.result_type(u[c], uib))
            x[o.ic] = o.u_s[c]
            x.reshape(-1)[cells] = uib[self.sel]
            ut.append(x)
        G = o.velocity_grad(u)
        gradp = O.gauss_grad(m, p, o.bnd.pressure_spec())
        aP, b0 = [], []
        for c in range(m.dims):
            aPc, aM, aPl, bc = O.assemble_transport(m, phi, self.nu_eff, o.bnd.velocity_spec(c))
            aP.append(aPc)
            b0.append(bc + o.transpose_source(G, self.nu_eff, c))
        return u, p, phi, ut, aP, aM, aPl, b0, gradp

    def residual(self, z, lam=None):
        m, o = self.m, self.o
        lam = self.lam0 if lam is None else lam
        au = o.opts["urf_u"]
        rlx = (1.0 - au) / au
        u, p, phi, ut, aP, aM, aPl, b0, gradp = self._momentum_pieces(z, lam)
        aavg = sum(a / au for a in aP) / m.dims
        Rm, H = [], []
        for c in range(m.dims):
            off = O.apply_offdiag(m, aM, aPl, ut[c])
            du = u[c] - ut[c]
            Rm.append(aavg * du - rlx * aP[c] * du + aP[c] * ut[c] + off - b0[c] + m.V * gradp[c])
            H.append((b0[c] + rlx * aP[c] * u[c] - off - (aP[c] / au - aavg) * ut[c]) / aavg)
        rAU = m.V / aavg
        phiH = o._flux_of(H)
        coef, pA_P, pA_M, pA_Pl, prhs = o.pressure_operator(rAU)
        if o.opts.get("continuity_mask", "A") == "B":
            cm = 1.0 - lam
        else:
            cm = np.where(o.mask_m, 1.0, 0.0)
        Rp = pA_P * p + O.apply_offdiag(m, pA_M, pA_Pl, p) + cm * o.divergence(phiH) - prhs
        phin = o.correct_flux(phiH, coef, p)
        Rf = [phi[d] - phin[d] for d in range(m.dims)]
        return self.pack(Rm, Rp, Rf)

    def drag_rows(self, z, lam=None):
        """The x-momentum row residual aP ut + sum a_N ut_N - b0 + V dp/dx of
        the imposed rows (ic and laminar-branch bc cells), zero elsewhere,
        laid out like R.  In an imposed row this is the force the immersed
        boundary applies to the fluid (the f_ib of Eq. hfdibrans_1)."""
        m = self.m
        lam = self.lam0 if lam is None else lam
        u, p, phi, ut, aP, aM, aPl, b0, gradp = self._momentum_pieces(z, lam)
        r = aP[0] * ut[0] + O.apply_offdiag(m, aM, aPl, ut[0]) - b0[0] + m.V * gradp[0]
        r = np.where(self.fixed, r, 0.0)
        zero = np.zeros(m.shape, dtype=r.dtype)
        faces = [np.zeros(self.shapes[m.dims + 1 + d], dtype=r.dtype) for d in range(m.dims)]
        return self.pack([r] + [zero] * (m.dims - 1), zero, faces)

    def objective(self, z, lam=None):
        if self.kind == "drag":
            # the force of the fluid on the body: minus the forcing applied to the fluid
            return float(-np.sum(self.drag_rows(z, lam).real))
        _, p, _ = self.unpack(z)
        return float(np.sum(self.jw * p.real))

    def objective_grad(self, z=None):
        """(J_z, J_lambda) as dense vectors."""
        if self.kind == "drag":
            z = self.state() if z is None else z
            Fz = self._colour_jacobian(lambda x: self.drag_rows(x), z.astype(complex), self.shapes, self.offs)
            zc = z.astype(complex)
            shp = self.m.shape
            Fl = self._colour_jacobian(lambda l: self.drag_rows(zc, l.reshape(shp)),
                                       self.lam0.ravel().astype(complex), [shp], np.array([0, self.m.N]))
            return -np.asarray(Fz.sum(axis=0)).ravel().real, -np.asarray(Fl.sum(axis=0)).ravel().real
        g = np.zeros(self.offs[-1])
        b = self.m.dims
        g[self.offs[b]:self.offs[b + 1]] = self.jw.ravel()
        return g, np.zeros(self.m.N)

    # ---------------------------------------------------------------- Jacobians
    def _colour_jacobian(self, f, x0, shapes, offs):
        """Sparse Jacobian of f at x0 (columns laid out as blocks of grid
        arrays `shapes`) by complex steps over a distance colouring: columns of
        one block whose grid indices agree mod 2*REACH+1 share an evaluation;
        a row is attributed to the unique such column within REACH of it."""
        K = 2 * REACH + 1
        rows_sh = self.shapes
        rows_off = self.offs
        R_, C_, V_ = [], [], []
        for b, shp in enumerate(shapes):
            kc = [range(min(K, s)) for s in shp]
            for ck in kc[0]:
                for cj in kc[1]:
                    for ci in kc[2]:
                        mask = np.zeros(shp, bool)
                        mask[ck::K, cj::K, ci::K] = True
                        dx = np.zeros(offs[-1], complex)
                        dx[offs[b]:offs[b + 1]] = mask.ravel() * (1j * H_CS)
                        y = f(x0 + dx)
                        jac = y.imag / H_CS
                        for rb, rshp in enumerate(rows_sh):
                            seg = jac[rows_off[rb]:rows_off[rb + 1]]
                            nz = np.flatnonzero(seg)
                            if len(nz) == 0:
                                continue
                            rk, rj, ri = np.unravel_index(nz, rshp)
                            col = []
                            for r, cc, ext in ((rk, ck, shp[0]), (rj, cj, shp[1]), (ri, ci, shp[2])):
                                off = (r - cc) % K
                                v = np.where(off <= REACH, r - off, r + (K - off))
                                if ext == 1:
                                    v = np.zeros_like(r)
                                col.append(v)
                            ok = (col[0] >= 0) & (col[0] < shp[0]) & (col[1] >= 0) & (col[1] < shp[1]) & \
                                 (col[2] >= 0) & (col[2] < shp[2])
                            inside = mask[np.clip(col[0], 0, shp[0] - 1), np.clip(col[1], 0, shp[1] - 1),
                                          np.clip(col[2], 0, shp[2] - 1)]
                            if not np.all(ok & inside):
                                raise RuntimeError("colouring reach exceeded")
                            cidx = np.ravel_multi_index((col[0], col[1], col[2]), shp) + offs[b]
                            R_.append(nz + rows_off[rb])
                            C_.append(cidx)
                            V_.append(seg[nz])
        n_rows = rows_off[-1]
        return sp.csr_matrix((np.concatenate(V_), (np.concatenate(R_), np.concatenate(C_))),
                             shape=(n_rows, offs[-1]))

    def jacobian_z(self, z=None):
        z = self.state() if z is None else z
        return self._colour_jacobian(lambda x: self.residual(x), z.astype(complex), self.shapes, self.offs)

    def jacobian_lambda(self, z=None):
        z = self.state() if z is None else z
        zc = z.astype(complex)
        shp = self.m.shape
        return self._colour_jacobian(lambda l: self.residual(zc, l.reshape(shp)),
                                     self.lam0.ravel().astype(complex), [shp], np.array([0, self.m.N]))

    def gradient(self):
        """(J, dJ/dlambda, psi) at the converged state."""
        if self.n_kinks:
            raise ValueError("%d interior faces carry zero flux: J is not differentiable" % self.n_kinks)
        z = self.state()
        Rz = self.jacobian_z(z)
        Rl = self.jacobian_lambda(z)
        Jz, Jl = self.objective_grad(z)
        psi = spla.spsolve(Rz.T.tocsc(), Jz)
        g = Jl - (Rl.T @ psi).real
        return self.objective(z), g.reshape(self.m.shape), psi


# ---------------------------------------------------------------- finite differences
def frozen_solve(o, tol=1e-13, max_iter=20000):
    """Frozen-turbulence sweeps until the momentum and pressure scaled
    residuals are at or below tol."""
    for it in range(max_iter):
        res = o.sweep(frozen_turbulence=True)
        r = max(res["U%d" % c] for c in range(o.m.dims))
        if max(r, res["p"]) <= tol:
            return it + 1, res
    return max_iter, res


def with_lambda(o, lam_new):
    """A copy of the converged oracle on a perturbed lambda, with every
    integer decision checked unchanged (cell groups, mask, closed faces,
    geometry choices)."""
    m = o.m
    tag = O.classify(m, lam_new)
    if not np.array_equal(tag, o.tag):
        raise ValueError("perturbation changes the cell groups")
    if o.opts.get("continuity_mask", "A") != "B" and not np.array_equal(lam_new < 1.0, o.mask_m):
        raise ValueError("perturbation changes the continuity mask")
    bnd = O.Boundaries(m, o.case, lam_new)
    for key in o.bnd.closed:
        if not np.array_equal(bnd.closed[key], o.bnd.closed[key]):
            raise ValueError("perturbation changes the closed faces")
    geo = O.ib_geometry(m, lam_new, tag)
    for key in ("cell", "nbr", "case", "base1", "base2", "clamped", "fallback"):
        if not np.array_equal(geo[key], o.geo[key]):
            raise ValueError("perturbation changes the bc-cell geometry choice " + key)
    q = copy.deepcopy(o)
    q.lam = lam_new
    q.geo = geo
    return q


def fd_gradient(o, cells, delta=1e-6, tol=1e-13, objective="pressure_drop"):
    """Central differences of J over frozen-turbulence solves started from
    the converged state, for the flat cell indices `cells`."""
    fs = FrozenSteady(o, objective)
    out = []
    for c in cells:
        vals = []
        for sgn in (1.0, -1.0):
            lam = o.lam.copy()
            lam.reshape(-1)[c] += sgn * delta
            q = with_lambda(o, lam)
            q.imposed_fields()
            if not np.array_equal(q.lam_branch, fs.o.lam_branch if o.model != "laminar" else q.lam_branch):
                raise ValueError("perturbation flips a wall-function branch")
            frozen_solve(q, tol=tol)
            if objective == "drag":
                fq = FrozenSteady(q, objective)
                vals.append(fq.objective(fq.state()))
            else:
                vals.append(float(np.sum(fs.jw * q.p)))
        out.append((vals[0] - vals[1]) / (2.0 * delta))
    return np.array(out)
