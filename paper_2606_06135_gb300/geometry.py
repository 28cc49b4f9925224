"""Seeded synthetic inputs for the HFDIB steady-RANS SIMPLE path.

This module builds the *inputs* of the solver and nothing else: uniform
Cartesian grids, signed distances sigma_perp of analytic bodies (positive in
fluid, negative in solid, Sec. 2.3), the lambda indicator of Eq. (lambda)
made from them, the wall distance the k-omega SST blending functions need,
and the boundary/flow description of the benchmark-shaped workloads
(cylinder, backward-facing step, NACA 0012, Ahmed-like body, random
obstacles, a rectangle misaligned with the mesh).  No step of the SIMPLE sweep lives here; both the CUDA path and
the CPU oracle take these dictionaries as plain inputs.

A case is a dict with keys
    grid   : dict(nx, ny, nz, x0, y0, z0, dx, dy, dz)   (nz == 1 -> 2D,
             one cell thick, dz := sqrt(dx*dy) so that V^(1/3) = sqrt(dx*dy))
    lam    : float64 [nz, ny, nx]  lambda in [0, 1]
    ywall  : float64 [nz, ny, nx]  distance to the nearest no-slip wall
    model  : 'laminar' | 'kepsilon' | 'komegasst' | 'komega' | 'realizableke'
    Re, u_ref, l_ref           nu = u_ref * l_ref / Re
    bc     : dict side -> 'inlet' | 'outlet' | 'slip' | 'wall' | 'empty'
             for sides xmin, xmax, ymin, ymax, zmin, zmax
    u_in   : inlet velocity (3,), I_in : turbulence intensity,
    lt_in  : turbulent length scale, p_out : outlet pressure,
    u_s    : velocity of the solid (3,)
"""
from __future__ import annotations

import math

import numpy as np

SIDES = ("xmin", "xmax", "ymin", "ymax", "zmin", "zmax")


# --------------------------------------------------------------------------
# grids
# --------------------------------------------------------------------------
def make_grid(nx, ny, nz, x0, y0, lx, ly, z0=0.0, lz=None):
    dx = lx / nx
    dy = ly / ny
    if nz == 1:
        dz = math.sqrt(dx * dy)
    else:
        dz = lz / nz
    return dict(nx=int(nx), ny=int(ny), nz=int(nz), x0=float(x0), y0=float(y0),
                z0=float(z0), dx=float(dx), dy=float(dy), dz=float(dz))


def cell_size(grid):
    """V^(1/3) of a cell; sqrt(dx*dy) for one-cell-thick 2D grids."""
    if grid["nz"] == 1:
        return math.sqrt(grid["dx"] * grid["dy"])
    return math.pow(grid["dx"] * grid["dy"] * grid["dz"], 1.0 / 3.0)


def cell_centres(grid):
    nx, ny, nz = grid["nx"], grid["ny"], grid["nz"]
    i = np.arange(nx, dtype=np.float64)
    j = np.arange(ny, dtype=np.float64)
    k = np.arange(nz, dtype=np.float64)
    xc = grid["x0"] + (i + 0.5) * grid["dx"]
    yc = grid["y0"] + (j + 0.5) * grid["dy"]
    zc = grid["z0"] + (k + 0.5) * grid["dz"]
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    return X, Y, Z


def lambda_from_sigma(sigma, h_c, half_width=0.75):
    """lambda = 0 (fluid) / 0.5[1 - tanh(sigma/h_c)] (cut band) / 1 (solid).

    The band of intersected cells is |sigma| < half_width*h_c, i.e. a
    smoothed interface 1.5 cells wide (Eq. lambda with V^(1/3) = h_c).
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    lam = np.where(sigma >= half_width * h_c, 0.0,
                   np.where(sigma <= -half_width * h_c, 1.0,
                            0.5 * (1.0 - np.tanh(sigma / h_c))))
    return np.ascontiguousarray(lam, dtype=np.float64)


def _base_case(name, grid, sigma, ywall, model, Re, bc, u_in=(1.0, 0.0, 0.0),
               I_in=0.02, lt_in=0.1, u_ref=1.0, l_ref=1.0):
    h = cell_size(grid)
    lam = lambda_from_sigma(sigma, h)
    return dict(name=name, grid=grid, lam=lam,
                ywall=np.ascontiguousarray(np.maximum(ywall, 0.0), dtype=np.float64),
                sigma=np.ascontiguousarray(sigma, dtype=np.float64),
                model=model, Re=float(Re), u_ref=float(u_ref), l_ref=float(l_ref),
                bc=dict(bc), u_in=tuple(float(v) for v in u_in), I_in=float(I_in),
                lt_in=float(lt_in), p_out=0.0, u_s=(0.0, 0.0, 0.0))


def bc2d(xmin="inlet", xmax="outlet", ymin="slip", ymax="slip"):
    return dict(xmin=xmin, xmax=xmax, ymin=ymin, ymax=ymax, zmin="empty", zmax="empty")


# --------------------------------------------------------------------------
# workloads shaped like the paper's benchmarks
# --------------------------------------------------------------------------
def case_uniform(nx=32, ny=16, model="kepsilon", Re=100.0, I_in=0.05):
    """lambda == 0 everywhere: uniform inflow between slip walls."""
    g = make_grid(nx, ny, 1, 0.0, 0.0, 2.0, 1.0)
    X, Y, _ = cell_centres(g)
    sigma = np.full(X.shape, 1e3)
    return _base_case("uniform", g, sigma, np.full(X.shape, 1e3), model, Re,
                      bc2d(), I_in=I_in, lt_in=0.1)


def case_cylinder(nx=128, ny=64, model="kepsilon", Re=40.0, D=1.0):
    """Circular cylinder D=1 at (4D, 4D) in a 16D x 8D channel (Sec. 3.4)."""
    g = make_grid(nx, ny, 1, 0.0, 0.0, 16.0 * D, 8.0 * D)
    X, Y, _ = cell_centres(g)
    sigma = np.sqrt((X - 4.0 * D) ** 2 + (Y - 4.0 * D) ** 2) - 0.5 * D
    return _base_case("cylinder", g, sigma, sigma, model, Re, bc2d(),
                      I_in=0.02, lt_in=0.8 * D, l_ref=D)


def case_channel(ny_in=16, nx=24, model="laminar", Re=10.0, wall_offset=0.0,
                 pad_cells=3):
    """Plane channel of height 1 between two immersed walls (Sec. 3.1 shape).

    The fluid gap y in [0, 1] is resolved by ny_in cells; pad_cells solid
    cells sit outside each wall.  wall_offset shifts both walls by a fraction
    of a cell (interface-position study, Sec. 3.1).
    """
    dy = 1.0 / ny_in
    ny = ny_in + 2 * pad_cells
    y0 = -pad_cells * dy + wall_offset * dy
    g = make_grid(nx, ny, 1, 0.0, y0, nx * dy * 1.0, ny * dy)
    X, Y, _ = cell_centres(g)
    sigma = np.minimum(Y, 1.0 - Y)
    return _base_case("channel", g, sigma, sigma, model, Re,
                      bc2d(ymin="wall", ymax="wall"), I_in=0.02, lt_in=0.1)


def case_bfs(nx=1024, ny=256, model="komegasst", Re=36000.0, I_in=0.05):
    """Backward-facing step (Sec. 3.3): step height h=1, expansion 9/8.

    Domain [-4h, 26h] x [0, 9h]; the step is the solid x < 0, y < h.  Inlet
    plug U=1 with I=5 %, l_t = 0.1 x inlet width (8h).  The bottom boundary
    is a no-slip wall (inside the step it is closed by the solid), the top a
    slip boundary.
    """
    g = make_grid(nx, ny, 1, -4.0, 0.0, 30.0, 9.0)
    X, Y, _ = cell_centres(g)
    outside = np.sqrt(np.maximum(X, 0.0) ** 2 + np.maximum(Y - 1.0, 0.0) ** 2)
    inside = -np.minimum(-X, 1.0 - Y)
    in_solid = (X < 0.0) & (Y < 1.0)
    sigma = np.where(in_solid, inside, outside)
    ywall = np.where(in_solid, 0.0, np.minimum(outside, np.where(X > 0.0, Y, 1e30)))
    return _base_case("bfs", g, sigma, ywall, model, Re,
                      bc2d(ymin="wall", ymax="slip"), I_in=I_in, lt_in=0.8)


def naca4_thickness(xc, t=0.12):
    """NACA 4-digit half thickness, closed trailing edge coefficient."""
    xc = np.clip(xc, 0.0, 1.0)
    return 5.0 * t * (0.2969 * np.sqrt(xc) - 0.1260 * xc - 0.3516 * xc ** 2
                      + 0.2843 * xc ** 3 - 0.1036 * xc ** 4)


def _naca_polyline(npts=4096, t=0.12):
    beta = np.linspace(0.0, math.pi, npts)
    xc = 0.5 * (1.0 - np.cos(beta))
    yt = naca4_thickness(xc, t)
    upper = np.stack([xc, yt], 1)
    lower = np.stack([xc[::-1], -yt[::-1]], 1)
    return np.concatenate([upper, lower[1:]], 0)


def case_naca(nx=2048, ny=1024, aoa_deg=0.0, model="komegasst", Re=1e6):
    """NACA 0012, chord 1, leading edge at (5c, 5c), domain 20c x 10c.

    The body is rotated about the quarter chord by the angle of attack.
    sigma_perp is the distance to a 4096-point polyline of the surface,
    signed by the analytic inside test.
    """
    from scipy.spatial import cKDTree
    g = make_grid(nx, ny, 1, 0.0, 0.0, 20.0, 10.0)
    X, Y, _ = cell_centres(g)
    a = math.radians(aoa_deg)
    xq, yq = 5.25, 5.0
    # body frame: rotate by +aoa about the quarter chord (nose up for a>0)
    xr = (X - xq) * math.cos(a) - (Y - yq) * math.sin(a) + 0.25
    yr = (X - xq) * math.sin(a) + (Y - yq) * math.cos(a)
    poly = _naca_polyline()
    tree = cKDTree(poly)
    pts = np.stack([xr.ravel(), yr.ravel()], 1)
    dist, idx = tree.query(pts)
    # refine with the two segments adjacent to the nearest vertex
    best = dist.copy()
    for off in (-1, 0):
        i0 = np.clip(idx + off, 0, len(poly) - 2)
        p0 = poly[i0]
        p1 = poly[i0 + 1]
        seg = p1 - p0
        L2 = np.maximum((seg ** 2).sum(1), 1e-300)
        tpar = np.clip(((pts - p0) * seg).sum(1) / L2, 0.0, 1.0)
        proj = p0 + tpar[:, None] * seg
        best = np.minimum(best, np.sqrt(((pts - proj) ** 2).sum(1)))
    dist = best.reshape(X.shape)
    inside = (xr > 0.0) & (xr < 1.0) & (np.abs(yr) < naca4_thickness(xr))
    sigma = np.where(inside, -dist, dist)
    c = dict(_base_case("naca0012", g, sigma, np.where(inside, 0.0, dist), model, Re,
                        bc2d(), I_in=0.001, lt_in=0.1))
    c["aoa_deg"] = float(aoa_deg)
    return c


def _ahmed_sdf(X, Y, Z):
    """Approximate signed distance of an Ahmed-like body (metres)."""
    L, W, H, r = 1.044, 0.389, 0.288, 0.1
    xn, yc, zb = 2.0, 1.44, 0.05
    # box centred frame
    cx, cy, cz = xn + 0.5 * L, yc, zb + 0.5 * H
    qx = np.abs(X - cx) - 0.5 * L
    qy = np.abs(Y - cy) - 0.5 * W
    qz = np.abs(Z - cz) - 0.5 * H
    # rounded front: round the edges in the front part only
    rr = np.where(X < xn + r, r, 0.0)
    qx2, qy2, qz2 = qx + rr, qy + rr, qz + rr
    out = np.sqrt(np.maximum(qx2, 0) ** 2 + np.maximum(qy2, 0) ** 2 + np.maximum(qz2, 0) ** 2)
    inn = np.minimum(np.maximum(np.maximum(qx2, qy2), qz2), 0.0)
    box = out + inn - rr
    # 25 degree rear slant over the last 0.222 m of the roof
    s = math.radians(25.0)
    x_s = xn + L - 0.222
    z_top = zb + H
    nxs, nzs = math.sin(s), math.cos(s)
    plane = (X - x_s) * nxs + (Z - z_top) * nzs
    return np.maximum(box, plane)


def case_ahmed(nx=256, ny=96, nz=96, model="kepsilon", Re=2.8e6):
    """3D Ahmed-like bluff body on cubic cells h = 0.03 (Sec. 3.6 shape)."""
    h = 0.03
    g = make_grid(nx, ny, nz, 0.0, 0.0, nx * h, ny * h, z0=0.0, lz=nz * h)
    X, Y, Z = cell_centres(g)
    sigma = _ahmed_sdf(X, Y, Z)
    ywall = np.minimum(np.maximum(sigma, 0.0), Z)
    bc = dict(xmin="inlet", xmax="outlet", ymin="slip", ymax="slip", zmin="wall", zmax="slip")
    return _base_case("ahmed", g, sigma, ywall, model, Re, bc, I_in=0.02,
                      lt_in=0.1 * ny * h, l_ref=1.044)


def grf_design_size(b):
    nxb = 256 + 8 * ((32 * b) // 31)
    return nxb, nxb // 2


def case_grf(nx=64, ny=32, seed=0, model="kepsilon", Re=1000.0, corr_cells=None):
    """Channel [0,2]x[0,1] with a random smooth obstacle.

    g is unit-variance filtered white noise from numpy.random.default_rng(seed)
    (Gaussian filter, std = corr_cells, default nx/16 cells); the solid is g > 1
    inside x in [0.5, 1.5]; sigma_perp ~ (1 - g)/|grad g|.
    """
    from scipy.ndimage import gaussian_filter
    g = make_grid(nx, ny, 1, 0.0, 0.0, 2.0, 1.0)
    X, Y, _ = cell_centres(g)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((ny, nx))
    s = corr_cells if corr_cells is not None else max(nx / 16.0, 2.0)
    f = gaussian_filter(w, s, mode="wrap")
    f = f / f.std()
    gy, gx = np.gradient(f, g["dy"], g["dx"])
    gn = np.maximum(np.sqrt(gx ** 2 + gy ** 2), 1e-12)
    window = (X[0] > 0.5) & (X[0] < 1.5)
    sig = np.where(window, (1.0 - f) / gn, 1e3)
    sig = sig[None]
    ywall = np.maximum(sig, 0.0)
    return _base_case("grf", g, sig, ywall, model, Re, bc2d(), I_in=0.02, lt_in=0.1)


def case_rotated_box(beta_deg=15.0, n=64, model="kepsilon", Re=1e4):
    """Rectangle 1 x 0.25 at the domain centre rotated by beta (App. C)."""
    g = make_grid(2 * n, n, 1, 0.0, 0.0, 4.0, 2.0)
    X, Y, _ = cell_centres(g)
    b = math.radians(beta_deg)
    xr = (X - 2.0) * math.cos(b) + (Y - 1.0) * math.sin(b)
    yr = -(X - 2.0) * math.sin(b) + (Y - 1.0) * math.cos(b)
    qx = np.abs(xr) - 0.5
    qy = np.abs(yr) - 0.125
    out = np.sqrt(np.maximum(qx, 0) ** 2 + np.maximum(qy, 0) ** 2)
    inn = np.minimum(np.maximum(qx, qy), 0.0)
    sigma = out + inn
    return _base_case("rotated_box", g, sigma, np.maximum(sigma, 0.0), model, Re, bc2d(),
                      I_in=0.02, lt_in=0.2)


def case_misaligned_box(beta_deg=15.0, n=64, L=8.0, model="kepsilon", Re=1e5, I_in=0.02):
    """Rectangle 1 x 0.25 at the centre of a square L x L domain, rotated by
    beta in [0, 90] degrees, with the inflow rotated with it (App. C: zero
    angle of attack, misaligned with the mesh faces).

    The paper's domain is a circle whose inlet arc turns with the body. A
    square grid cannot rotate its sides, so the flow (cos beta, sin beta)
    enters through x- and y- and leaves through x+ and y+ (at beta = 0 the
    y- side carries the free stream tangentially). Mirroring about the
    diagonal maps this problem at beta onto the problem at 90 - beta, and
    at 45 degrees onto itself: the invariance the tests check. Inlet
    turbulence as in the paper's pipe flows: I = 2 %, l_t a tenth of the
    inlet width."""
    g = make_grid(n, n, 1, 0.0, 0.0, L, L)
    X, Y, _ = cell_centres(g)
    b = math.radians(beta_deg)
    cb, sb = math.cos(b), math.sin(b)
    c = 0.5 * L
    xr = (X - c) * cb + (Y - c) * sb
    yr = -(X - c) * sb + (Y - c) * cb
    qx = np.abs(xr) - 0.5
    qy = np.abs(yr) - 0.125
    out = np.sqrt(np.maximum(qx, 0) ** 2 + np.maximum(qy, 0) ** 2)
    inn = np.minimum(np.maximum(qx, qy), 0.0)
    sigma = out + inn
    bc = bc2d(xmin="inlet", xmax="outlet", ymin="inlet", ymax="outlet")
    return _base_case("misaligned_box", g, sigma, np.maximum(sigma, 0.0), model, Re, bc,
                      u_in=(cb, sb, 0.0), I_in=I_in, lt_in=0.1 * L)


def case_sphere(nx=32, ny=16, nz=16, model="kepsilon", Re=40.0, D=1.0):
    """Sphere D = 1 at (4D, 4D, 4D) in a 16D x 8D x 8D box (3D cylinder
    analogue): inlet x-, outlet x+, slip on the four other sides."""
    g = make_grid(nx, ny, nz, 0.0, 0.0, 16.0 * D, 8.0 * D, z0=0.0, lz=8.0 * D)
    X, Y, Z = cell_centres(g)
    sigma = np.sqrt((X - 4.0 * D) ** 2 + (Y - 4.0 * D) ** 2 + (Z - 4.0 * D) ** 2) - 0.5 * D
    bc = dict(xmin="inlet", xmax="outlet", ymin="slip", ymax="slip", zmin="slip", zmax="slip")
    return _base_case("sphere", g, sigma, sigma, model, Re, bc, I_in=0.02, lt_in=0.8 * D, l_ref=D)


def nu_of(case):
    return case["u_ref"] * case["l_ref"] / case["Re"]
