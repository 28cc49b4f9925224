"""Plain FP64 CPU oracle of the HFDIB steady-RANS SIMPLE sweep.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference arm may import this module; the product path never
does and shares no code with it.

It follows the paper step by step (Sec. 2, Fig. "simplehfdibrans"):

  a0  cell groups ic/bc/fc from lambda (Sec. 2.3), normal n = -grad(lambda)/
      |grad(lambda)| and in-solid neighbour (Eq. yorthoaux), y_perp three
      cases (Eq. yortho), y_eff (Eq. yplus), interpolation points along n
      (Sec. 2.5, Fig. interpolation)
  a1  max over bc u fc of omega_old / eps_old (Eq. imval)
  a2  u_tau (Eq. frictionvel), y+ (Eq. yplus), masks alpha_u = alpha_k
      (Eq. alphauk), u_ib, k_ib by quadratic interpolation with the wall
      function surface k (Eq. kws), omega_ib (Eq. omegaws)
  a3  momentum assembly of Eq. (hfdibrans)_1 with the IB source realised as
      rows u = u_ib where alpha_u = 1, implicit under-relaxation
  a4  momentum solve (exact sparse LU: the fixed point does not depend on
      the inner solver)
  a5  correction u = u + alpha_u (u_ib - u) (Eq. corru)
  a6  rAU, HbyA, face flux phiHbyA (standard SIMPLE, Sec. 2.5.1)
  a7  pressure equation laplacian(rAU_f, p) = m div(phiHbyA) with m = 1
      where lambda < 1 (lambda-masked continuity, Eq. hfdibrans_2; reading
      B, an option: m = 1 - lambda)
  a8  flux / pressure relaxation / velocity update
  a9  production, P_ib assignment (Eq. omegaws)
  a10 eps/omega equation with rows eps = eps_ib (omega = omega_ib) where
      alpha_omega = 1 (Eq. alphaomega, matrix manipulation)
  a11 k equation with rows k = k_ib where alpha_k = 1, then the k correction
  a12 nu_t and scaled residuals

Every linear system is assembled as a scipy.sparse matrix and solved with
scipy's sparse LU.  Floating point is FP64 throughout; the geometry step a0
uses plain IEEE double operations in a fixed order so that its integer
decisions (tags, chosen neighbour, interpolation cells) are reproducible.

Turbulence models (Sec. 2.1 names four): standard k-epsilon, k-omega SST,
the k-omega model written out in Eq. hfdibkomega, and realizable
k-epsilon.  All four share the HFDIB treatment: imposed eps/omega rows in ic
and bc cells, imposed k rows where alpha_k = 1, P_ib in bc cells.

Readings where the paper is silent are stated at each function; the wall
function and turbulence-model constants are the standard published values
(Wilcox; Launder-Spalding; Menter; Shih et al.), which the paper names but
does not print.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# wall-function constants (Sec. 2.5; values not printed in the paper)
C_MU = 0.09        # C_nu in Eq. frictionvel
KAPPA = 0.41
E_WF = 9.8
BETA1_WF = 0.075   # beta_1 in Eq. omegaws
C_WF = 11.0        # C in Eq. kws
C_EPS2 = 1.9       # C_eps2 in Eq. kws
YPLUS_LAM = 11.0   # Sec. 2.3

# standard k-epsilon (Launder & Spalding)
KE_C1, KE_C2, KE_SIGK, KE_SIGE = 1.44, 1.92, 1.0, 1.3

# k-omega SST (Menter), standard coefficients
SST = dict(ak1=0.85, ak2=1.0, aw1=0.5, aw2=0.856, g1=5.0 / 9.0, g2=0.44,
           b1=0.075, b2=0.0828, bstar=0.09, a1=0.31, bb1=1.0, c1=10.0)

# k-omega (Wilcox), Eq. hfdibkomega: sink beta* k omega in the k equation,
# source C_alpha1 (omega/k) P_k and sink C_beta1 omega^2 in the omega
# equation, diffusivities nu + nu_t/sigma; nu_t = k/omega.  The printed form
# has no cross-diffusion and no stress limiter.  Coefficients: the standard
# high-Reynolds set (beta* 0.09, beta 0.072, alpha 0.52, 1/sigma_k =
# 1/sigma_omega = 0.5).
KW = dict(bstar=0.09, beta=0.072, gamma=0.52, ak=0.5, aw=0.5)

# realizable k-epsilon (Shih, Liou, Shabbir, Yang, Zhu 1995): variable C_mu =
# 1/(A0 + A_s U* k/eps), eps source C1 S eps with C1 = max(0.43, eta/(eta+5)),
# eta = S k/eps, sink C2 eps^2/(k + sqrt(nu eps))
RKE = dict(A0=4.0, C2=1.9, sigk=1.0, sige=1.2)

K_MIN = 1e-14
EPS_MIN = 1e-14
OMEGA_MIN = 1e-14

TAG_FC, TAG_BC, TAG_IC = 0, 1, 2

# wall_distance: "y_eff" (Eq. yplus, default) or "y_perp", the distance the
# wall functions use in y+ and omega_ib (the comparison of App. A)
# continuity_mask: "A" (default) m = 1 where lambda < 1, else 0; "B" m = 1 - lambda
# convection: scheme of the momentum convection term, "upwind" (Sec. 3.1,
# default) or, by deferred correction, "linearUpwind" / "vanLeer" /
# "linearUpwindLimited" (App. B; the last with a cell-limited gradient)
DEFAULT_OPTS = dict(urf_u=0.7, urf_p=0.3, urf_turb=0.85, freeze_switch=0, wall_distance="y_eff",
                    continuity_mask="A", convection="upwind")


def _zeros(shape, *like):
    """Zeros in float64, or complex128 when any of `like` is complex (the
    adjoint checks differentiate these blocks by the complex step; real
    inputs take exactly the float64 path)."""
    dt = np.result_type(np.float64, *[np.asarray(a).dtype for a in like])
    return np.zeros(shape, dtype=dt)


def _sl(ax, a, b):
    s = [slice(None)] * 3
    s[ax] = slice(a, b)
    return tuple(s)


class Mesh:
    """Uniform Cartesian grid; arrays are [nz, ny, nx], x fastest."""

    def __init__(self, grid):
        self.nx, self.ny, self.nz = grid["nx"], grid["ny"], grid["nz"]
        self.x0, self.y0, self.z0 = grid["x0"], grid["y0"], grid["z0"]
        self.dx, self.dy, self.dz = grid["dx"], grid["dy"], grid["dz"]
        self.dims = 2 if self.nz == 1 else 3
        self.n = (self.nx, self.ny, self.nz)
        self.D = (self.dx, self.dy, self.dz)
        self.o = (self.x0, self.y0, self.z0)
        self.S = (self.dy * self.dz, self.dx * self.dz, self.dx * self.dy)
        self.V = self.dx * self.dy * self.dz
        # V^(1/3); one-cell-thick 2D grids use dz := sqrt(dx*dy)
        if self.dims == 2:
            self.h = math.sqrt(self.dx * self.dy)
        else:
            self.h = math.pow(self.dx * self.dy * self.dz, 1.0 / 3.0)
        self.shape = (self.nz, self.ny, self.nx)
        self.N = self.nx * self.ny * self.nz

    @staticmethod
    def ax(d):
        return 2 - d

    def slab(self, arr, d, hi):
        n = self.n[d]
        return arr[_sl(2 - d, n - 1, n)] if hi else arr[_sl(2 - d, 0, 1)]

    def centre(self, i, j, k):
        return (self.x0 + (i + 0.5) * self.dx, self.y0 + (j + 0.5) * self.dy,
                self.z0 + (k + 0.5) * self.dz)

    def lin(self, i, j, k):
        return (k * self.ny + j) * self.nx + i


SIDE_NAMES = {(0, 0): "xmin", (0, 1): "xmax", (1, 0): "ymin", (1, 1): "ymax",
              (2, 0): "zmin", (2, 1): "zmax"}


# ==========================================================================
# a0: cell groups and boundary-cell geometry (Sec. 2.3-2.5)
# ==========================================================================
def classify(m: Mesh, lam):
    """Cell groups of Sec. 2.3: ic if lambda >= 0.5; bc if 0 < lambda < 0.5 or
    lambda == 0 with an ic cell among the neighbours sharing >= 1 vertex;
    fc otherwise.  Returns uint8 tags (0 fc, 1 bc, 2 ic)."""
    ic = lam >= 0.5
    pad = np.pad(ic, 1, mode="constant", constant_values=False)
    any_ic = np.zeros(m.shape, dtype=bool)
    oz_range = (-1, 0, 1) if m.dims == 3 else (0,)
    for oz in oz_range:
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                if ox == 0 and oy == 0 and oz == 0:
                    continue
                any_ic |= pad[1 + oz:1 + oz + m.nz, 1 + oy:1 + oy + m.ny, 1 + ox:1 + ox + m.nx]
    bc = ((lam > 0.0) & (lam < 0.5)) | ((lam == 0.0) & any_ic)
    tag = np.full(m.shape, TAG_FC, dtype=np.uint8)
    tag[bc] = TAG_BC
    tag[ic] = TAG_IC
    return tag


def _moore(m: Mesh, i, j, k):
    """In-domain vertex neighbours of (i,j,k) in increasing linear index."""
    out = []
    for oz in ((-1, 0, 1) if m.dims == 3 else (0,)):
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                if ox == 0 and oy == 0 and oz == 0:
                    continue
                ii, jj, kk = i + ox, j + oy, k + oz
                if 0 <= ii < m.nx and 0 <= jj < m.ny and 0 <= kk < m.nz:
                    out.append((ox, oy, oz, ii, jj, kk))
    return out


def _grad_lambda(m: Mesh, lam, i, j, k):
    """Central differences of lambda (one-sided at the domain edges)."""
    idx = (i, j, k)
    g = []
    for d in range(3):
        n = m.n[d]
        if n == 1:
            g.append(0.0)
            continue
        lo = list(idx)
        hi = list(idx)
        if idx[d] == 0:
            hi[d] += 1
            g.append((lam[hi[2], hi[1], hi[0]] - lam[k, j, i]) / m.D[d])
        elif idx[d] == n - 1:
            lo[d] -= 1
            g.append((lam[k, j, i] - lam[lo[2], lo[1], lo[0]]) / m.D[d])
        else:
            hi[d] += 1
            lo[d] -= 1
            g.append((lam[hi[2], hi[1], hi[0]] - lam[lo[2], lo[1], lo[0]]) / (2.0 * m.D[d]))
    return g


def surface_normal(m: Mesh, lam, i, j, k):
    """n = -grad(lambda)/|grad(lambda)| (Eq. yorthoaux).

    Reading: where |grad lambda| < 1e-12/h the normal is taken from the
    vertex neighbour with the largest lambda to P (ties: most shared
    vertices, then lowest index).
    """
    gx, gy, gz = _grad_lambda(m, lam, i, j, k)
    mag = math.sqrt((gx * gx + gy * gy) + gz * gz)
    if mag < 1e-12 / m.h:
        best = None
        for ox, oy, oz, ii, jj, kk in _moore(m, i, j, k):
            nz_off = abs(ox) + abs(oy) + abs(oz)
            lv = lam[kk, jj, ii]
            if best is None or lv > best[0] or (lv == best[0] and nz_off < best[4]):
                best = (lv, ox, oy, oz, nz_off)
        vx, vy, vz = -best[1] * m.dx, -best[2] * m.dy, -best[3] * m.dz
        nv = math.sqrt((vx * vx + vy * vy) + vz * vz)
        return (vx / nv, vy / nv, vz / nv), True
    return (-gx / mag, -gy / mag, -gz / mag), False


def sigma_of_lambda(m: Mesh, lam_v):
    """sigma_perp = V^(1/3) atanh(1 - 2 lambda) (Eq. yorthoaux)."""
    return m.h * math.atanh(1.0 - 2.0 * lam_v)


def _interp_stencil(m: Mesh, X):
    """Cells and weights of bi/trilinear interpolation of a cell-centred
    field at point X (clamped to the cell-centre lattice)."""
    base = []
    t = []
    for d in range(3):
        n = m.n[d]
        if n == 1:
            base.append(0)
            t.append(0.0)
            continue
        xi = (X[d] - m.o[d]) / m.D[d] - 0.5
        i0 = math.floor(xi)
        i0 = min(max(i0, 0), n - 2)
        td = xi - i0
        td = min(max(td, 0.0), 1.0)
        base.append(int(i0))
        t.append(td)
    return base, t


def ib_geometry(m: Mesh, lam, tag):
    """Per-bc-cell geometry (Sec. 2.4-2.5), as a dict of arrays sorted by cell.

    For each bc cell P:
      n_P       outer unit normal (Eq. yorthoaux)
      N         in-solid neighbour: argmin over ic vertex neighbours of
                -n_P.(P - N) (Sec. 2.4).  Reading for exact ties (an
                axis-aligned wall): the neighbour sharing the most vertices
                (face, then edge, then corner), then the lowest linear index.
                -1 when P has no ic neighbour (only possible in case (a))
      case      0: lambda_P in (0, .5) -> |sigma_P|
                1: lambda_P = 0, lambda_N in [.5, 1) -> n_N.[P - (N + |sigma_N| n_N)]
                2: lambda_P = 0, lambda_N = 1 -> |P - mean of shared vertices|
      y_perp    clamped below at 1e-3 h (reading: the paper leaves y_perp <= 0
                of case (b) open)
      y_eff     0.5 [y_perp + 0.5 h] (Eq. yplus)
      interpolation: surface point S = P - y_perp n_P, free-stream points
                X1 = P + h n_P, X2 = P + 2h n_P; quadratic Lagrange weights
                (wS, w1, w2) of the profile through (0, d1 = y_perp + h,
                d2 = y_perp + 2h) evaluated at y_perp (Fig. interpolation);
                X1, X2 values by bi/trilinear interpolation.
    """
    cells = np.flatnonzero(tag.ravel() == TAG_BC)
    nb = len(cells)
    out = dict(cell=cells.astype(np.int64), nbr=np.full(nb, -1, np.int64),
               case=np.zeros(nb, np.int32), n=np.zeros((nb, 3)), y_perp=np.zeros(nb),
               y_eff=np.zeros(nb), wS=np.zeros(nb), w1=np.zeros(nb), w2=np.zeros(nb),
               base1=np.zeros((nb, 3), np.int64), t1=np.zeros((nb, 3)),
               base2=np.zeros((nb, 3), np.int64), t2=np.zeros((nb, 3)),
               clamped=np.zeros(nb, bool), fallback=np.zeros(nb, bool))
    h = m.h
    for q, c in enumerate(cells):
        k, rem = divmod(int(c), m.ny * m.nx)
        j, i = divmod(rem, m.nx)
        P = m.centre(i, j, k)
        nP, fb = surface_normal(m, lam, i, j, k)
        out["fallback"][q] = fb
        best = None
        for ox, oy, oz, ii, jj, kk in _moore(m, i, j, k):
            if tag[kk, jj, ii] != TAG_IC:
                continue
            s = (nP[0] * (ox * m.dx) + nP[1] * (oy * m.dy)) + nP[2] * (oz * m.dz)
            nz_off = abs(ox) + abs(oy) + abs(oz)
            if best is None or s < best[0] or (s == best[0] and nz_off < best[4]):
                best = (s, ii, jj, kk, nz_off)
        lp = lam[k, j, i]
        if best is not None:
            _, ii, jj, kk, _ = best
            out["nbr"][q] = m.lin(ii, jj, kk)
        if lp > 0.0:
            case = 0
            yp = abs(sigma_of_lambda(m, lp))
        else:
            _, ii, jj, kk, _ = best
            lN = lam[kk, jj, ii]
            Nc = m.centre(ii, jj, kk)
            if lN < 1.0:
                case = 1
                nN, _ = surface_normal(m, lam, ii, jj, kk)
                sN = abs(sigma_of_lambda(m, lN))
                Q = (Nc[0] + sN * nN[0], Nc[1] + sN * nN[1], Nc[2] + sN * nN[2])
                yp = (nN[0] * (P[0] - Q[0]) + nN[1] * (P[1] - Q[1])) + nN[2] * (P[2] - Q[2])
            else:
                case = 2
                v = (0.5 * (P[0] + Nc[0]), 0.5 * (P[1] + Nc[1]), 0.5 * (P[2] + Nc[2]))
                ex, ey, ez = P[0] - v[0], P[1] - v[1], P[2] - v[2]
                yp = math.sqrt((ex * ex + ey * ey) + ez * ez)
        if yp < 1e-3 * h:
            yp = 1e-3 * h
            out["clamped"][q] = True
        out["case"][q] = case
        out["n"][q] = nP
        out["y_perp"][q] = yp
        out["y_eff"][q] = 0.5 * (yp + 0.5 * h)
        X1 = (P[0] + h * nP[0], P[1] + h * nP[1], P[2] + h * nP[2])
        h2 = 2.0 * h
        X2 = (P[0] + h2 * nP[0], P[1] + h2 * nP[1], P[2] + h2 * nP[2])
        b1, t1 = _interp_stencil(m, X1)
        b2, t2 = _interp_stencil(m, X2)
        out["base1"][q], out["t1"][q] = b1, t1
        out["base2"][q], out["t2"][q] = b2, t2
        # quadratic Lagrange basis through d = 0 (S), d1 (X1), d2 (X2) at d = y_perp
        d1 = yp + h
        d2 = yp + h2
        dp = yp
        out["wS"][q] = ((dp - d1) * (dp - d2)) / ((0.0 - d1) * (0.0 - d2))
        out["w1"][q] = ((dp - 0.0) * (dp - d2)) / ((d1 - 0.0) * (d1 - d2))
        out["w2"][q] = ((dp - 0.0) * (dp - d1)) / ((d2 - 0.0) * (d2 - d1))
    return out


def interp_at(m: Mesh, f, base, t):
    """Bi/trilinear interpolation of cell field f with precomputed stencils."""
    f = np.asarray(f)
    val = np.zeros(len(base))
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                w = np.ones(len(base))
                idx = []
                for d, c in ((0, cx), (1, cy), (2, cz)):
                    if m.n[d] == 1:
                        if c == 1:
                            w = w * 0.0
                        idx.append(base[:, d])
                    else:
                        w = w * (t[:, d] if c == 1 else (1.0 - t[:, d]))
                        idx.append(base[:, d] + c)
                val = val + w * f[idx[2], idx[1], idx[0]]
    return val


# ==========================================================================
# boundary description
# ==========================================================================
class Boundaries:
    """Boundary kind per side and the 'closed' faces of Sec. 3.1: a wall
    face whose adjacent cell has lambda > 0 (a wall inside the solid) gets
    zero gradient for every variable and no flux.  Readings: slip sides are
    treated like walls; an inlet face is closed where its cell is in-solid
    (lambda >= 0.5), so no inflow is forced into the body; outlet faces keep
    p = p_out."""

    def __init__(self, m: Mesh, case, lam):
        self.m = m
        self.kind = {}
        self.closed = {}
        for d in range(m.dims):
            for hi in (0, 1):
                name = SIDE_NAMES[(d, hi)]
                kind = case["bc"][name]
                self.kind[(d, hi)] = kind
                sl = m.slab(lam, d, hi)
                if kind == "outlet":
                    self.closed[(d, hi)] = np.zeros(sl.shape, bool)
                elif kind == "inlet":
                    self.closed[(d, hi)] = sl >= 0.5
                else:
                    self.closed[(d, hi)] = sl > 0.0
        self.u_in = np.array(case["u_in"], dtype=np.float64)
        self.p_out = float(case["p_out"])

    def velocity_spec(self, c):
        """Per side (fixed_mask, value) for velocity component c."""
        spec = {}
        for key, kind in self.kind.items():
            d, hi = key
            cl = self.closed[key]
            if kind == "inlet":
                spec[key] = (~cl, self.u_in[c])
            elif kind == "wall":
                spec[key] = (~cl, 0.0)
            elif kind == "slip":
                spec[key] = (~cl & (c == d), 0.0)
            else:  # outlet
                spec[key] = (np.zeros(cl.shape, bool), 0.0)
        return spec

    def scalar_spec(self, inlet_value):
        spec = {}
        for key, kind in self.kind.items():
            cl = self.closed[key]
            if kind == "inlet":
                spec[key] = (~cl, inlet_value)
            else:
                spec[key] = (np.zeros(cl.shape, bool), 0.0)
        return spec

    def pressure_spec(self):
        spec = {}
        for key, kind in self.kind.items():
            cl = self.closed[key]
            if kind == "outlet":
                spec[key] = (np.ones(cl.shape, bool), self.p_out)
            else:
                spec[key] = (np.zeros(cl.shape, bool), 0.0)
        return spec


# ==========================================================================
# finite-volume building blocks (Sec. 3.1 "Numerical schemes": upwind)
# ==========================================================================
def face_values(m: Mesh, f, spec):
    """Face values of a cell field along each direction: linear interpolation
    inside, the fixed value or the cell value (zero gradient) on the boundary.
    Returns list over d of arrays with n_d + 1 entries along that axis."""
    out = []
    for d in range(m.dims):
        ax = 2 - d
        n = m.n[d]
        shp = list(f.shape)
        shp[ax] = n + 1
        F = _zeros(shp, f)
        F[_sl(ax, 1, n)] = 0.5 * (f[_sl(ax, 0, n - 1)] + f[_sl(ax, 1, n)])
        for hi in (0, 1):
            fm, val = spec[(d, hi)]
            cellv = m.slab(f, d, hi)
            bv = np.where(fm, val, cellv)
            F[_sl(ax, n, n + 1) if hi else _sl(ax, 0, 1)] = bv
        out.append(F)
    return out


def gauss_grad(m: Mesh, f, spec):
    """Gauss gradient with linear interpolation: (f_+ - f_-)/Delta per axis."""
    Fs = face_values(m, f, spec)
    g = [np.zeros(m.shape) for _ in range(3)]
    for d in range(m.dims):
        ax = 2 - d
        n = m.n[d]
        g[d] = (Fs[d][_sl(ax, 1, n + 1)] - Fs[d][_sl(ax, 0, n)]) / m.D[d]
    return g


def assemble_transport(m: Mesh, phi, gamma, spec):
    """Integrated steady transport operator div(phi f) - f div(phi) -
    div(gamma grad f) with upwind convection (bounded form) and central
    diffusion; face gamma is the arithmetic mean.

    Returns aP, aM[d], aPl[d], b with aP f_P + sum aM f_minus + aPl f_plus = b.
    phi[d] holds the volumetric flux through each d-face in the +d direction.
    """
    like = [phi[d] for d in range(m.dims)] + [gamma]
    aP = _zeros(m.shape, *like)
    b = _zeros(m.shape, *like)
    aM = [_zeros(m.shape, *like) for _ in range(3)]
    aPl = [_zeros(m.shape, *like) for _ in range(3)]
    for d in range(m.dims):
        ax = 2 - d
        n = m.n[d]
        S = m.S[d]
        Dl = m.D[d]
        F = phi[d]
        Fint = F[_sl(ax, 1, n)]                    # interior faces, +d flux
        gf = 0.5 * (gamma[_sl(ax, 0, n - 1)] + gamma[_sl(ax, 1, n)])
        Dif = gf * S / Dl
        # owner side (cell below the face): outward flux = +F
        lo = _sl(ax, 0, n - 1)
        up = _sl(ax, 1, n)
        aPl[d][lo] = np.minimum(Fint, 0.0) - Dif
        aP[lo] += np.maximum(-Fint, 0.0) + Dif
        # neighbour side (cell above the face): outward flux = -F
        aM[d][up] = np.minimum(-Fint, 0.0) - Dif
        aP[up] += np.maximum(Fint, 0.0) + Dif
        for hi in (0, 1):
            fm, val = spec[(d, hi)]
            Fb = F[_sl(ax, n, n + 1)] if hi else F[_sl(ax, 0, 1)]
            Fout = Fb if hi else -Fb
            gP = m.slab(gamma, d, hi)
            Db = gP * S / (0.5 * Dl)
            coef = np.where(fm, Db + np.maximum(-Fout, 0.0), 0.0)
            cs = _sl(ax, n - 1, n) if hi else _sl(ax, 0, 1)
            aP[cs] += coef
            b[cs] += coef * val
    return aP, aM, aPl, b


CONV_SCHEMES = ("upwind", "linearUpwind", "vanLeer", "linearUpwindLimited")


def cell_limiter(m: Mesh, f, G):
    """Cell-limited gradient factor l_P in [0, 1] (the Barth-Jespersen rule):
    the largest l <= 1 for which every face extrapolation f_P + l grad f_P .
    (x_f - x_P) = f_P +- l (Delta_d/2) df/dx_d stays within the minimum and
    maximum of f over P and its interior neighbours.  G[d] = df/dx_d."""
    fmax = f.copy()
    fmin = f.copy()
    for d in range(m.dims):
        ax = 2 - d
        n = m.n[d]
        lo, hi = _sl(ax, 0, n - 1), _sl(ax, 1, n)
        fmax[lo] = np.maximum(fmax[lo], f[hi])
        fmin[lo] = np.minimum(fmin[lo], f[hi])
        fmax[hi] = np.maximum(fmax[hi], f[lo])
        fmin[hi] = np.minimum(fmin[hi], f[lo])
    lim = np.ones(m.shape)
    for d in range(m.dims):
        for sgn in (1.0, -1.0):
            delta = sgn * 0.5 * m.D[d] * G[d]
            up = delta > 0.0
            dn = delta < 0.0
            with np.errstate(divide="ignore", invalid="ignore"):
                lim = np.where(up, np.minimum(lim, (fmax - f) / np.where(up, delta, 1.0)), lim)
                lim = np.where(dn, np.minimum(lim, (fmin - f) / np.where(dn, delta, 1.0)), lim)
    return lim


def face_correction(m: Mesh, phi_d, f, dfdx_d, d, scheme):
    """Scheme face value minus the upwind value, f_face - f_U, on the interior
    faces normal to d (App. B: schemes for the convection term of momentum).
    U is the upwind cell of the face (flux phi_d >= 0: the low cell), D the
    other, s = +1 when D lies at +d from U.
      linearUpwind: f_face = f_U + grad f_U . (x_face - x_U) = f_U + s (Delta/2) df/dx_d|U
      vanLeer (TVD): f_face = f_U + psi(r) (f_D - f_U)/2, psi(r) = (r + |r|)/(1 + |r|),
                     r = 2 (x_D - x_U) . grad f_U / (f_D - f_U) - 1 (0 where f_D = f_U)
    with the cell gradient of the Gauss-linear scheme."""
    ax = 2 - d
    n = m.n[d]
    F = phi_d[_sl(ax, 1, n)]
    fL, fH = f[_sl(ax, 0, n - 1)], f[_sl(ax, 1, n)]
    gL, gH = dfdx_d[_sl(ax, 0, n - 1)], dfdx_d[_sl(ax, 1, n)]
    pos = F >= 0.0
    fU = np.where(pos, fL, fH)
    fD = np.where(pos, fH, fL)
    gU = np.where(pos, gL, gH)
    s = np.where(pos, 1.0, -1.0)
    if scheme == "linearUpwind":
        return s * (0.5 * m.D[d]) * gU
    if scheme == "vanLeer":
        dd = fD - fU
        nz = dd != 0.0
        r = np.where(nz, 2.0 * (s * m.D[d]) * gU / np.where(nz, dd, 1.0) - 1.0, 0.0)
        psi = (r + np.abs(r)) / (1.0 + np.abs(r))
        return np.where(nz, 0.5 * psi * dd, 0.0)
    raise ValueError("convection scheme: " + str(scheme))


def convection_correction(m: Mesh, phi, f, G, scheme):
    """Deferred correction of the upwind convection of f (one velocity
    component): the rows keep the bounded upwind operator and take
    -sum_faces F_out (f_face - f_U) as an explicit source, so a converged
    state solves the scheme's equations.  G[d] = d f / d x_d.  Boundary faces
    keep their upwind / boundary values."""
    out = _zeros(m.shape, f, *phi[:m.dims])
    if scheme == "upwind":
        return out
    if scheme == "linearUpwindLimited":
        # linearUpwind with each cell's gradient scaled by its limiter
        lim = cell_limiter(m, f, G)
        G = [lim * G[d] for d in range(m.dims)]
        scheme = "linearUpwind"
    for d in range(m.dims):
        ax = 2 - d
        n = m.n[d]
        corr = phi[d][_sl(ax, 1, n)] * face_correction(m, phi[d], f, G[d], d, scheme)
        out[_sl(ax, 0, n - 1)] -= corr     # the face is the high face of the low cell
        out[_sl(ax, 1, n)] += corr         # and the low face (outward flux -F) of the high cell
    return out


def to_sparse(m: Mesh, aP, aM, aPl):
    idx = np.arange(m.N).reshape(m.shape)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [aP.ravel()]
    for d in range(m.dims):
        ax = 2 - d
        n = m.n[d]
        up = _sl(ax, 1, n)
        lo = _sl(ax, 0, n - 1)
        rows += [idx[up].ravel(), idx[lo].ravel()]
        cols += [idx[lo].ravel(), idx[up].ravel()]
        vals += [aM[d][up].ravel(), aPl[d][lo].ravel()]
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(m.N, m.N))


def apply_offdiag(m: Mesh, aM, aPl, f):
    """sum over neighbours a_N f_N."""
    out = _zeros(m.shape, f, *aM[:m.dims], *aPl[:m.dims])
    for d in range(m.dims):
        ax = 2 - d
        n = m.n[d]
        out[_sl(ax, 1, n)] += aM[d][_sl(ax, 1, n)] * f[_sl(ax, 0, n - 1)]
        out[_sl(ax, 0, n - 1)] += aPl[d][_sl(ax, 0, n - 1)] * f[_sl(ax, 1, n)]
    return out


def scaled_residual(m: Mesh, aP, aM, aPl, b, x, rows, fixed_val=None):
    """Normalised residual sum|b - Ax| / (sum|Ax - xbar A1| + sum|b - xbar A1|)
    over the solved rows, xbar the mean of x (the usual OpenFOAM measure,
    App. D).  Rows outside `rows` are fixed rows; there x takes `fixed_val`
    (the value the system imposes) before A x is formed."""
    if fixed_val is not None:
        x = np.where(rows, x, fixed_val)
    Ax = aP * x + apply_offdiag(m, aM, aPl, x)
    A1 = aP + apply_offdiag(m, aM, aPl, np.ones(m.shape))
    xbar = x.mean()
    r = np.abs(b - Ax)[rows].sum()
    nf = (np.abs(Ax - A1 * xbar)[rows].sum() + np.abs(b - A1 * xbar)[rows].sum()) + 1e-20
    return r / nf


def solve_with_rows(m: Mesh, aP, aM, aPl, b, fixed, fixed_val):
    """Solve the assembled system; rows where `fixed` hold x = fixed_val
    (direct matrix manipulation, Sec. 2.3)."""
    A = to_sparse(m, aP, aM, aPl)
    f = fixed.ravel().astype(np.float64)
    keep = sp.diags(1.0 - f)
    A = keep @ A + sp.diags(f)
    rhs = (1.0 - f) * b.ravel() + f * np.broadcast_to(fixed_val, m.shape).ravel()
    x = spla.spsolve(A.tocsc(), rhs)
    return x.reshape(m.shape)


# ==========================================================================
# the solver
# ==========================================================================
class Oracle:
    """FP64 SIMPLE/HFDIB solver on a uniform grid.  `case` as produced by
    paper_2606_06135_gb300.geometry; `opts` overrides relaxation factors."""

    def __init__(self, case, opts=None):
        self.case = case
        self.opts = dict(DEFAULT_OPTS)
        if opts:
            self.opts.update(opts)
        m = self.m = Mesh(case["grid"])
        self.lam = np.ascontiguousarray(case["lam"], dtype=np.float64).reshape(m.shape)
        self.model = case["model"]
        self.nu = case["u_ref"] * case["l_ref"] / case["Re"]
        self.u_s = np.array(case["u_s"], dtype=np.float64)
        self.bnd = Boundaries(m, case, self.lam)
        self.ywall = np.ascontiguousarray(case["ywall"], dtype=np.float64).reshape(m.shape)
        # a0
        self.tag = classify(m, self.lam)
        self.geo = ib_geometry(m, self.lam, self.tag)
        self.ic = self.tag == TAG_IC
        self.bcm = self.tag == TAG_BC
        self.mask_m = self.lam < 1.0     # continuity enforced where lambda < 1 (reading A)
        # inlet turbulence (Eq. bcspkoein), literal C_nu k^1.5 / l_t
        U = float(np.linalg.norm(case["u_in"]))
        self.k_in = 1.5 * (U * case["I_in"]) ** 2
        self.eps_in = C_MU * self.k_in ** 1.5 / case["lt_in"]
        self.omega_in = self.eps_in / (C_MU * self.k_in)
        self.init_state()
        self.iteration = 0
        self.history = []

    def continuity_mask(self, lam=None):
        """m of the pressure source m div(phiHbyA), the discrete form of the
        (1 - lambda) factor of Eq. hfdibrans_2.  Reading A (default): m = 1
        where lambda < 1, else 0 -- continuity everywhere but in the fully
        solid cells, whose rows stay nonsingular.  Reading B: m = 1 - lambda,
        the factor itself, smooth in lambda."""
        lam = self.lam if lam is None else lam
        if self.opts.get("continuity_mask", "A") == "B":
            return 1.0 - lam
        return np.where(lam < 1.0, 1.0, 0.0)

    # ---------------------------------------------------------------- state
    def init_state(self):
        m = self.m
        self.u = [np.where(self.ic, self.u_s[c], self.bnd.u_in[c]) for c in range(m.dims)]
        self.p = np.zeros(m.shape)
        turb = self.model != "laminar"
        self.k = np.where(self.ic, 0.0, self.k_in) if turb else np.zeros(m.shape)
        self.eps = np.full(m.shape, self.eps_in) if turb else np.zeros(m.shape)
        self.omega = np.full(m.shape, self.omega_in) if turb else np.zeros(m.shape)
        if turb:
            self.nut = np.where(self.ic, 0.0, C_MU * self.k ** 2 / self.eps)
        else:
            self.nut = np.zeros(m.shape)
        self.phi = self._flux_of(self.u)

    def _flux_of(self, u):
        """Face fluxes of a velocity field (linear interpolation)."""
        m = self.m
        phi = []
        for d in range(m.dims):
            Fs = face_values(m, u[d], self.bnd.velocity_spec(d))[d]
            phi.append(Fs * m.S[d])
        for d in range(m.dims):
            ax = 2 - d
            n = m.n[d]
            for hi in (0, 1):
                kind = self.bnd.kind[(d, hi)]
                fs = _sl(ax, n, n + 1) if hi else _sl(ax, 0, 1)
                cl = self.bnd.closed[(d, hi)]
                if kind in ("wall", "slip"):
                    phi[d][fs] = 0.0
                phi[d][fs] = np.where(cl, 0.0, phi[d][fs])
        return phi

    def velocity_grad(self, u):
        """G[a][b] = d u_b / d x_a (Gauss, linear)."""
        m = self.m
        G = [[np.zeros(m.shape) for _ in range(3)] for _ in range(3)]
        for c in range(m.dims):
            g = gauss_grad(m, u[c], self.bnd.velocity_spec(c))
            for a in range(m.dims):
                G[a][c] = g[a]
        return G

    # ---------------------------------------------------------------- a1/a2
    def imposed_fields(self):
        """a1 + a2: masks and imposed values from the fields at sweep start."""
        m = self.m
        geo = self.geo
        cells = geo["cell"]
        turb = self.model != "laminar"
        notic = ~self.ic
        # Eq. imval: omega_ib = max over bc u fc of omega_old (eps for k-eps)
        self.omega_max = float(self.omega[notic].max()) if (turb and notic.any()) else 0.0
        self.eps_max = float(self.eps[notic].max()) if (turb and notic.any()) else 0.0
        alpha_u = self.ic.astype(np.float64)
        u_ib = [np.where(self.ic, self.u_s[c], 0.0) for c in range(m.dims)]
        k_ib = np.zeros(m.shape)
        w_ib = np.where(self.ic, self.omega_max, 0.0)
        e_ib = np.where(self.ic, self.eps_max, 0.0)
        kf = self.k.ravel()
        kP = kf[cells]
        # Eq. frictionvel, Eq. yplus
        ut = C_MU ** 0.25 * np.sqrt(kP)
        # Eq. yplus uses y_eff; App. A compares it with y_perp
        ywf = geo["y_perp"] if self.opts.get("wall_distance", "y_eff") == "y_perp" else geo["y_eff"]
        yplus = ywf * ut / self.nu
        lamb = (yplus <= YPLUS_LAM) if turb else np.ones(len(cells), bool)
        # reading (opt-in, not in the paper): from sweep `freeze_switch` on, a
        # bc cell may leave the laminar branch but never re-enter it.  The
        # laminar branch feeds k_P back through k_ib ~ k_vis(y+) C_mu^1/2 k_P,
        # a gain above 1 for y+ above ~5, so cells between ~5 and y+_lam
        # cycle between the branches; the one-way rule ends such cycles.
        fz = self.opts.get("freeze_switch", 0)
        if turb and fz > 0 and self.iteration >= fz and getattr(self, "lam_branch", None) is not None:
            lamb = self.lam_branch & lamb
        self.yplus_bc = yplus
        self.lam_branch = lamb
        af = alpha_u.ravel()
        af[cells] = np.where(lamb, 1.0, 0.0)
        alpha_u = af.reshape(m.shape)
        # quadratic interpolation along n from the previous iteration
        for c in range(m.dims):
            v1 = interp_at(m, self.u[c], geo["base1"], geo["t1"])
            v2 = interp_at(m, self.u[c], geo["base2"], geo["t2"])
            val = geo["wS"] * self.u_s[c] + geo["w1"] * v1 + geo["w2"] * v2
            uf = u_ib[c].ravel()
            uf[cells] = np.where(lamb, val, 0.0)
            u_ib[c] = uf.reshape(m.shape)
        if turb:
            # Eq. kws: surface k = k_vis(y+) u_tau^2
            Cf = (1.0 / (yplus + C_WF) ** 2 + 2.0 * yplus / C_WF ** 3 - 1.0 / C_WF ** 2)
            kvis = 2400.0 * Cf / C_EPS2 ** 2
            kS = kvis * ut ** 2
            self.k_surface = kS      # per bc cell, kept for inspection
            v1 = interp_at(m, self.k, geo["base1"], geo["t1"])
            v2 = interp_at(m, self.k, geo["base2"], geo["t2"])
            kval = geo["wS"] * kS + geo["w1"] * v1 + geo["w2"] * v2
            # reading: the quadratic profile may undershoot; k_ib >= 0
            kval = np.maximum(kval, 0.0)
            kfl = k_ib.ravel()
            kfl[cells] = np.where(lamb, kval, 0.0)
            k_ib = kfl.reshape(m.shape)
            # Eq. omegaws, written with y+ = y_eff u_tau / nu substituted:
            # lam: (u_tau^2/nu) 6/(beta1 y+^2) = 6 nu/(beta1 y_eff^2)
            # log: (u_tau^2/nu) /(kappa sqrt(C_nu) y+) = u_tau/(kappa sqrt(C_nu) y_eff)
            ye = ywf
            wl = 6.0 * self.nu / (BETA1_WF * ye ** 2)
            wg = ut / (KAPPA * math.sqrt(C_MU) * ye)
            wv = np.where(lamb, wl, wg)
            wf = w_ib.ravel()
            wf[cells] = wv
            w_ib = wf.reshape(m.shape)
            ef = e_ib.ravel()
            # eps = C_mu k omega with the k this cell takes this sweep: k_ib
            # where k is imposed (laminar branch), the old k_P where it is solved
            ef[cells] = C_MU * np.where(lamb, kval, kP) * wv
            e_ib = ef.reshape(m.shape)
        self.alpha_u = alpha_u
        self.u_ib = u_ib
        self.k_ib = k_ib
        self.omega_ib = w_ib
        self.eps_ib = e_ib

    # ---------------------------------------------------------------- sweep
    def sweep(self, frozen_turbulence=False):
        """One extended SIMPLE iteration (Fig. simplehfdibrans).  With
        frozen_turbulence the turbulence steps a9-a12 are skipped: nu_t, k and
        eps/omega keep their values (the frozen-turbulence flow problem whose
        adjoint the gradient checks differentiate)."""
        m = self.m
        o = self.opts
        au, ap = o["urf_u"], o["urf_p"]
        res = {}
        # ---- a1/a2: set alpha_u, compute u_ib
        self.imposed_fields()
        fixed_u = self.alpha_u > 0.5
        free_u = ~fixed_u
        # ---- a3: momentum assembly
        nu_eff = self.nu + self.nut
        G = self.velocity_grad(self.u)
        gradp = gauss_grad(m, self.p, self.bnd.pressure_spec())
        aPc, b0c = [], []
        for c in range(m.dims):
            aP, aM, aPl, b = assemble_transport(m, self.phi, nu_eff, self.bnd.velocity_spec(c))
            b = b + self.transpose_source(G, nu_eff, c) + self.momentum_convection_correction(G, c)
            aPc.append(aP)
            b0c.append(b)
        # ---- a4: momentum predictor (relaxed), rows u = u_ib where alpha_u = 1
        ustar = []
        for c in range(m.dims):
            res["U%d" % c] = scaled_residual(m, aPc[c], aM, aPl, b0c[c] - gradp[c] * m.V,
                                             self.u[c], free_u, self.u_ib[c])
            aPr = aPc[c] / au
            br = b0c[c] + (1.0 - au) / au * aPc[c] * self.u[c]
            x = solve_with_rows(m, aPr, aM, aPl, br - gradp[c] * m.V, fixed_u, self.u_ib[c])
            # ---- a5: correction, Eq. corru
            x = x + self.alpha_u * (self.u_ib[c] - x)
            ustar.append(x)
        # ---- a6: rAU, HbyA, phiHbyA (component-averaged diagonal)
        aPr = [aPc[c] / au for c in range(m.dims)]
        aavg = sum(aPr) / m.dims
        rAU = m.V / aavg
        HbyA = []
        for c in range(m.dims):
            br = b0c[c] + (1.0 - au) / au * aPc[c] * self.u[c]
            H = br - apply_offdiag(m, aM, aPl, ustar[c]) - (aPr[c] - aavg) * ustar[c]
            HbyA.append(H / aavg)
        phiH = self._flux_of(HbyA)
        # outlet faces carry the extrapolated HbyA (zero gradient)
        # ---- a7: pressure equation
        coef, pA_P, pA_M, pA_Pl, prhs_b = self.pressure_operator(rAU)
        div = self.divergence(phiH)
        cm = self.continuity_mask()
        rhs = -(cm * div) + prhs_b
        res["p"] = scaled_residual(m, pA_P, pA_M, pA_Pl, rhs, self.p, np.ones(m.shape, bool))
        pnew = solve_with_rows(m, pA_P, pA_M, pA_Pl, rhs, np.zeros(m.shape, bool), 0.0)
        # ---- a8: flux, pressure relaxation, velocity update
        self.phi = self.correct_flux(phiH, coef, pnew)
        self.p = self.p + ap * (pnew - self.p)
        gradp = gauss_grad(m, self.p, self.bnd.pressure_spec())
        self.u = [HbyA[c] - rAU * gradp[c] for c in range(m.dims)]
        divphi = self.divergence(self.phi)
        res["cont"] = float(np.abs(cm * divphi).sum())
        # ---- a9-a12: turbulence
        if frozen_turbulence:
            pass
        elif self.model == "kepsilon":
            self.kepsilon(res)
        elif self.model == "komegasst":
            self.komegasst(res)
        elif self.model == "komega":
            self.komega(res)
        elif self.model == "realizableke":
            self.realizable_ke(res)
        self.iteration += 1
        self.history.append(res)
        return res

    def momentum_convection_correction(self, G, c):
        """Deferred correction of the convection of u_c for the scheme of
        opts["convection"] (App. B), from u and grad u at sweep start."""
        m = self.m
        scheme = self.opts.get("convection", "upwind")
        return convection_correction(m, self.phi, self.u[c], [G[d][c] for d in range(m.dims)], scheme)

    def transpose_source(self, G, nu_eff, c):
        """Explicit div(nu_eff (grad u)^T) for component c: face flux
        nu_f (d u_a / d x_c)_f S_a through the a-faces."""
        m = self.m
        T = _zeros(m.shape, nu_eff, *[G[c][a] for a in range(m.dims)])
        for a in range(m.dims):
            ax = 2 - a
            n = m.n[a]
            val = G[c][a]                 # d u_a / d x_c
            Fv = _zeros([n + 1 if q == ax else s for q, s in enumerate(m.shape)], val)
            Fn = _zeros(Fv.shape, nu_eff)
            Fv[_sl(ax, 1, n)] = 0.5 * (val[_sl(ax, 0, n - 1)] + val[_sl(ax, 1, n)])
            Fn[_sl(ax, 1, n)] = 0.5 * (nu_eff[_sl(ax, 0, n - 1)] + nu_eff[_sl(ax, 1, n)])
            Fv[_sl(ax, 0, 1)] = m.slab(val, a, 0)
            Fv[_sl(ax, n, n + 1)] = m.slab(val, a, 1)
            Fn[_sl(ax, 0, 1)] = m.slab(nu_eff, a, 0)
            Fn[_sl(ax, n, n + 1)] = m.slab(nu_eff, a, 1)
            flux = Fn * Fv * m.S[a]
            T += flux[_sl(ax, 1, n + 1)] - flux[_sl(ax, 0, n)]
        return T

    def pressure_operator(self, rAU):
        """laplacian(rAU_f, p): face coefficients rAU_f S/Delta inside,
        rAU_P S/(Delta/2) on outlet faces (p = p_out).  Returned as the SPD
        matrix of -laplacian plus the outlet right-hand side."""
        m = self.m
        coef = []
        aP = _zeros(m.shape, rAU)
        aM = [_zeros(m.shape, rAU) for _ in range(3)]
        aPl = [_zeros(m.shape, rAU) for _ in range(3)]
        rhs = _zeros(m.shape, rAU)
        for d in range(m.dims):
            ax = 2 - d
            n = m.n[d]
            shp = list(m.shape)
            shp[ax] = n + 1
            C = _zeros(shp, rAU)
            C[_sl(ax, 1, n)] = 0.5 * (rAU[_sl(ax, 0, n - 1)] + rAU[_sl(ax, 1, n)]) * m.S[d] / m.D[d]
            for hi in (0, 1):
                if self.bnd.kind[(d, hi)] == "outlet":
                    fs = _sl(ax, n, n + 1) if hi else _sl(ax, 0, 1)
                    C[fs] = m.slab(rAU, d, hi) * m.S[d] / (0.5 * m.D[d])
            coef.append(C)
            lo = _sl(ax, 0, n - 1)
            up = _sl(ax, 1, n)
            ci = C[_sl(ax, 1, n)]
            aPl[d][lo] = -ci
            aP[lo] += ci
            aM[d][up] = -ci
            aP[up] += ci
            for hi in (0, 1):
                if self.bnd.kind[(d, hi)] == "outlet":
                    cb = C[_sl(ax, n, n + 1)] if hi else C[_sl(ax, 0, 1)]
                    cs = _sl(ax, n - 1, n) if hi else _sl(ax, 0, 1)
                    aP[cs] += cb
                    rhs[cs] += cb * self.bnd.p_out
        return coef, aP, aM, aPl, rhs

    def divergence(self, phi):
        m = self.m
        div = _zeros(m.shape, *phi[:m.dims])
        for d in range(m.dims):
            ax = 2 - d
            n = m.n[d]
            div += phi[d][_sl(ax, 1, n + 1)] - phi[d][_sl(ax, 0, n)]
        return div

    def correct_flux(self, phiH, coef, p):
        """phi = phiHbyA - rAU_f (p_N - p_P)/Delta S on interior and outlet
        faces (the pressure-equation flux)."""
        m = self.m
        out = []
        for d in range(m.dims):
            ax = 2 - d
            n = m.n[d]
            F = phiH[d].copy()
            F[_sl(ax, 1, n)] -= coef[d][_sl(ax, 1, n)] * (p[_sl(ax, 1, n)] - p[_sl(ax, 0, n - 1)])
            for hi in (0, 1):
                if self.bnd.kind[(d, hi)] == "outlet":
                    pb = self.bnd.p_out
                    if hi:
                        F[_sl(ax, n, n + 1)] -= coef[d][_sl(ax, n, n + 1)] * (pb - m.slab(p, d, 1))
                    else:
                        F[_sl(ax, 0, 1)] -= coef[d][_sl(ax, 0, 1)] * (m.slab(p, d, 0) - pb)
            out.append(F)
        return out

    # ---------------------------------------------------------------- turbulence
    def _production(self):
        """G = nu_t 2 S:S with S = sym(grad u) of the updated velocity; P_ib
        (Eq. omegaws) assigned in alpha_omega cells: P_k (laminar branch) or
        kappa nu y+ |n.grad u|^2 / ln^2(E y+) (log branch) in bc, 0 in ic."""
        m = self.m
        G = self.velocity_grad(self.u)
        S2 = np.zeros(m.shape)
        for a in range(m.dims):
            for b in range(m.dims):
                s = 0.5 * (G[a][b] + G[b][a])
                S2 += s * s
        S2 = 2.0 * S2
        Gk = self.nut * S2
        geo = self.geo
        cells = geo["cell"]
        nvec = geo["n"]
        dudn2 = np.zeros(len(cells))
        for b in range(m.dims):
            comp = np.zeros(len(cells))
            for a in range(m.dims):
                comp += nvec[:, a] * G[a][b].ravel()[cells]
            dudn2 += comp * comp
        # log branch of Eq. omegaws; y+ > y+_lam there, so max(y+, y+_lam) only
        # matters for cells kept in the log branch by the one-way switch
        yp = np.maximum(self.yplus_bc, YPLUS_LAM)
        with np.errstate(divide="ignore", invalid="ignore"):
            plog = KAPPA * self.nu * yp * dudn2 / np.log(E_WF * yp) ** 2
        Gf = Gk.ravel().copy()
        Gf[cells] = np.where(self.lam_branch, Gf[cells], plog)
        Gf[self.ic.ravel()] = 0.0
        return G, S2, Gk, Gf.reshape(m.shape)

    def _turb_solve(self, aP, aM, aPl, b, x_old, fixed, fixed_val, urf, name, res):
        m = self.m
        res[name] = scaled_residual(m, aP, aM, aPl, b, x_old, ~fixed, fixed_val)
        aPr = aP / urf
        br = b + (1.0 - urf) / urf * aP * x_old
        return solve_with_rows(m, aPr, aM, aPl, br, fixed, fixed_val)

    def kepsilon(self, res):
        """Standard k-epsilon with the HFDIB treatment (Fig. simplehfdibrans)."""
        m = self.m
        V = m.V
        urf = self.opts["urf_turb"]
        G, S2, Gk, Gmod = self._production()
        alpha_w = self.ic | self.bcm
        k_old = self.k
        e_old = self.eps
        # epsilon: rows eps = eps_ib in alpha_omega cells
        gam = self.nu + self.nut / KE_SIGE
        aP, aM, aPl, b = assemble_transport(m, self.phi, gam, self.bnd.scalar_spec(self.eps_in))
        ratio = e_old / np.maximum(k_old, K_MIN)
        aP = aP + KE_C2 * ratio * V
        b = b + KE_C1 * Gmod * ratio * V
        eps = self._turb_solve(aP, aM, aPl, b, e_old, alpha_w, self.eps_ib, urf, "eps", res)
        eps = np.maximum(eps, EPS_MIN)
        # k: rows k = k_ib in alpha_k (= alpha_u) cells
        gam = self.nu + self.nut / KE_SIGK
        aP, aM, aPl, b = assemble_transport(m, self.phi, gam, self.bnd.scalar_spec(self.k_in))
        aP = aP + eps / np.maximum(k_old, K_MIN) * V
        b = b + Gmod * V
        fixed_k = self.alpha_u > 0.5
        k = self._turb_solve(aP, aM, aPl, b, k_old, fixed_k, self.k_ib, urf, "k", res)
        k = np.maximum(k, K_MIN)
        k = k + self.alpha_u * (self.k_ib - k)        # k correction
        self.k = k
        self.eps = eps
        self.omega = eps / (C_MU * np.maximum(k, K_MIN))
        self.nut = C_MU * k * k / eps

    def _sst_blend(self, k, w, S2, gradk, gradw):
        """Menter's blending functions (SST, cited in Sec. 2.1): the
        cross-diffusion CD_kw = 2 sigma_w2 grad(k).grad(omega)/omega, F1 =
        tanh(arg1^4) with arg1 = min(max(sqrt(k)/(beta* omega y),
        500 nu/(y^2 omega)), 4 sigma_w2 k/(CD_kw+ y^2)), CD_kw+ = max(CD_kw,
        1e-10), and F2 = tanh(arg2^2) with arg2 = min(max(2 sqrt(k)/(beta*
        omega y), 500 nu/(y^2 omega)), 100).  y is the wall distance input,
        clipped below at 1e-3 h.  Returns (CD_kw, F1, F2)."""
        m = self.m
        c = SST
        y = np.maximum(self.ywall, 1e-3 * m.h)
        dot = sum(gradk[d] * gradw[d] for d in range(m.dims))
        CDkw = 2.0 * c["aw2"] * dot / w
        CDp = np.maximum(CDkw, 1e-10)
        sk = np.sqrt(k)
        arg1 = np.minimum(np.maximum(sk / (c["bstar"] * w * y), 500.0 * self.nu / (y * y * w)),
                          4.0 * c["aw2"] * k / (CDp * y * y))
        F1 = np.tanh(arg1 ** 4)
        arg2 = np.minimum(np.maximum(2.0 * sk / (c["bstar"] * w * y), 500.0 * self.nu / (y * y * w)),
                          100.0)
        F2 = np.tanh(arg2 * arg2)
        return CDkw, F1, F2

    @staticmethod
    def sst_nut(k, w, S2, F2):
        """SST eddy viscosity with Menter's limiter: nu_t = a1 k / max(a1
        omega, b1 F2 sqrt(2 S:S)) (S2 = 2 S:S)."""
        c = SST
        return c["a1"] * k / np.maximum(c["a1"] * w, c["bb1"] * F2 * np.sqrt(S2))

    @staticmethod
    def sst_k_production(G, k, w):
        """Production in the SST k equation with Menter's limiter:
        min(G, c1 beta* k omega)."""
        c = SST
        return np.minimum(G, c["c1"] * c["bstar"] * k * w)

    @staticmethod
    def sst_gbynu(S2, w, F2):
        """G/nu_t of the SST omega source, limited consistently with
        sst_nut and sst_k_production: min(2 S:S, (c1/a1) beta* omega
        max(a1 omega, b1 F2 sqrt(2 S:S)))."""
        c = SST
        return np.minimum(S2, (c["c1"] / c["a1"]) * c["bstar"] * w
                          * np.maximum(c["a1"] * w, c["bb1"] * F2 * np.sqrt(S2)))

    def komegasst(self, res):
        """k-omega SST (Menter) with the HFDIB treatment."""
        m = self.m
        V = m.V
        c = SST
        urf = self.opts["urf_turb"]
        G, S2, Gk, Gmod = self._production()
        alpha_w = self.ic | self.bcm
        k_old = self.k
        w_old = self.omega
        sspec = self.bnd.scalar_spec
        gradk = gauss_grad(m, k_old, sspec(self.k_in))
        gradw = gauss_grad(m, w_old, sspec(self.omega_in))
        CDkw, F1, F2 = self._sst_blend(np.maximum(k_old, K_MIN), w_old, S2, gradk, gradw)
        blend = lambda a1, a2: F1 * a1 + (1.0 - F1) * a2
        # omega equation
        gamma = blend(c["g1"], c["g2"])
        beta = blend(c["b1"], c["b2"])
        GbyNu = self.sst_gbynu(S2, w_old, F2)
        gam = self.nu + blend(c["aw1"], c["aw2"]) * self.nut
        aP, aM, aPl, b = assemble_transport(m, self.phi, gam, sspec(self.omega_in))
        aP = aP + beta * w_old * V
        b = b + gamma * GbyNu * V
        cdc = (F1 - 1.0) * CDkw / w_old
        aP = aP + np.where(cdc > 0.0, cdc, 0.0) * V
        b = b - np.where(cdc > 0.0, 0.0, cdc) * w_old * V
        w = self._turb_solve(aP, aM, aPl, b, w_old, alpha_w, self.omega_ib, urf, "omega", res)
        w = np.maximum(w, OMEGA_MIN)
        # k equation
        gam = self.nu + blend(c["ak1"], c["ak2"]) * self.nut
        aP, aM, aPl, b = assemble_transport(m, self.phi, gam, sspec(self.k_in))
        aP = aP + c["bstar"] * w * V
        b = b + self.sst_k_production(Gmod, k_old, w) * V
        fixed_k = self.alpha_u > 0.5
        k = self._turb_solve(aP, aM, aPl, b, k_old, fixed_k, self.k_ib, urf, "k", res)
        k = np.maximum(k, K_MIN)
        k = k + self.alpha_u * (self.k_ib - k)
        self.k = k
        self.omega = w
        self.eps = C_MU * k * w
        # nu_t = a1 k / max(a1 omega, b1 F2 sqrt(S2)) with the new k, omega
        _, _, F2n = self._sst_blend(np.maximum(k, K_MIN), w, S2, gradk, gradw)
        self.nut = self.sst_nut(k, w, S2, F2n)

    def komega(self, res):
        """k-omega (Wilcox) of Eq. hfdibkomega with the HFDIB treatment (the
        same imposed rows and P_ib as SST)."""
        m = self.m
        V = m.V
        c = KW
        urf = self.opts["urf_turb"]
        G, S2, Gk, Gmod = self._production()
        alpha_w = self.ic | self.bcm
        k_old = self.k
        w_old = self.omega
        sspec = self.bnd.scalar_spec
        # omega: C_alpha1 (omega/k) P_k - C_beta1 omega^2, nu + nu_t/sigma_omega1
        gam = self.nu + c["aw"] * self.nut
        aP, aM, aPl, b = assemble_transport(m, self.phi, gam, sspec(self.omega_in))
        aP = aP + c["beta"] * w_old * V
        b = b + c["gamma"] * w_old / np.maximum(k_old, K_MIN) * Gk * V
        w = self._turb_solve(aP, aM, aPl, b, w_old, alpha_w, self.omega_ib, urf, "omega", res)
        w = np.maximum(w, OMEGA_MIN)
        # k: P_k (P_ib in bc cells) - beta* k omega, nu + nu_t/sigma_k1
        gam = self.nu + c["ak"] * self.nut
        aP, aM, aPl, b = assemble_transport(m, self.phi, gam, sspec(self.k_in))
        aP = aP + c["bstar"] * w * V
        b = b + Gmod * V
        fixed_k = self.alpha_u > 0.5
        k = self._turb_solve(aP, aM, aPl, b, k_old, fixed_k, self.k_ib, urf, "k", res)
        k = np.maximum(k, K_MIN)
        k = k + self.alpha_u * (self.k_ib - k)
        self.k = k
        self.omega = w
        self.eps = C_MU * k * w
        self.nut = k / w

    def rke_coefficients(self, G):
        """Realizable k-eps: (A_s U*, S) per cell from the velocity gradient
        G[a][b] = d u_b / d x_a.  S_ij = sym(grad u), Omega_ij = skew(grad
        u), S~ = sqrt(S_ij S_ij), W = S_ij S_jk S_ki / S~^3 (0 where S~ = 0),
        phi = arccos(sqrt(6) W)/3 (argument clipped to [-1, 1]), A_s =
        sqrt(6) cos(phi), U* = sqrt(S_ij S_ij + Omega_ij Omega_ij), S =
        sqrt(2 S_ij S_ij)."""
        m = self.m
        d = m.dims
        Sm = [[0.5 * (G[a][b] + G[b][a]) for b in range(d)] for a in range(d)]
        Om = [[0.5 * (G[a][b] - G[b][a]) for b in range(d)] for a in range(d)]
        SS = sum(Sm[a][b] * Sm[a][b] for a in range(d) for b in range(d))
        OO = sum(Om[a][b] * Om[a][b] for a in range(d) for b in range(d))
        SSS = sum(Sm[a][b] * Sm[b][c] * Sm[c][a] for a in range(d) for b in range(d) for c in range(d))
        St = np.sqrt(SS)
        with np.errstate(divide="ignore", invalid="ignore"):
            W = np.where(St > 0.0, SSS / (St * St * St), 0.0)
        phi = np.arccos(np.clip(math.sqrt(6.0) * W, -1.0, 1.0)) / 3.0
        As = math.sqrt(6.0) * np.cos(phi)
        Us = np.sqrt(SS + OO)
        return As * Us, np.sqrt(2.0 * SS)

    def realizable_ke(self, res):
        """Realizable k-epsilon with the HFDIB treatment (the imposed rows and
        P_ib of standard k-epsilon)."""
        m = self.m
        V = m.V
        c = RKE
        urf = self.opts["urf_turb"]
        G, S2, Gk, Gmod = self._production()
        AsUs, S = self.rke_coefficients(G)
        alpha_w = self.ic | self.bcm
        k_old = self.k
        e_old = self.eps
        # eps: C1 S eps - C2 eps^2 / (k + sqrt(nu eps)), nu + nu_t/sigma_eps
        kk = np.maximum(k_old, K_MIN)
        eta = S * kk / e_old
        C1 = np.maximum(0.43, eta / (eta + 5.0))
        gam = self.nu + self.nut / c["sige"]
        aP, aM, aPl, b = assemble_transport(m, self.phi, gam, self.bnd.scalar_spec(self.eps_in))
        aP = aP + c["C2"] * e_old / (kk + np.sqrt(self.nu * e_old)) * V
        b = b + C1 * S * e_old * V
        eps = self._turb_solve(aP, aM, aPl, b, e_old, alpha_w, self.eps_ib, urf, "eps", res)
        eps = np.maximum(eps, EPS_MIN)
        # k: P_k (P_ib in bc cells) - eps, nu + nu_t/sigma_k
        gam = self.nu + self.nut / c["sigk"]
        aP, aM, aPl, b = assemble_transport(m, self.phi, gam, self.bnd.scalar_spec(self.k_in))
        aP = aP + eps / kk * V
        b = b + Gmod * V
        fixed_k = self.alpha_u > 0.5
        k = self._turb_solve(aP, aM, aPl, b, k_old, fixed_k, self.k_ib, urf, "k", res)
        k = np.maximum(k, K_MIN)
        k = k + self.alpha_u * (self.k_ib - k)
        self.k = k
        self.eps = eps
        self.omega = eps / (C_MU * np.maximum(k, K_MIN))
        # nu_t = C_mu k^2/eps = k^2 / (A0 eps + A_s U* k)
        self.nut = k * k / (c["A0"] * eps + AsUs * k)

    # ---------------------------------------------------------------- driver
    def max_residual(self, res):
        return max(v for key, v in res.items() if key != "cont")

    def solve(self, tol=1e-6, max_iter=1000, min_iter=1):
        for it in range(max_iter):
            res = self.sweep()
            if it + 1 >= min_iter and self.max_residual(res) <= tol:
                return it + 1, res
        return max_iter, res

    def fields(self):
        m = self.m
        f = dict(p=self.p.copy(), k=self.k.copy(), eps=self.eps.copy(),
                 omega=self.omega.copy(), nut=self.nut.copy())
        for c, nm in zip(range(m.dims), ("ux", "uy", "uz")):
            f[nm] = self.u[c].copy()
        return f
