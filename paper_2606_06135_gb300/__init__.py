"""GB300 (sm_103a) implementation of the HFDIB steady-RANS SIMPLE sweep.

Submodules:
    geometry  seeded synthetic inputs (grids, lambda, wall distance, cases)
    hfdib     ctypes binding of the C-ABI library libhfdib.so
    autograd  torch.autograd.Function around the steady solve and its adjoint
    build     nvcc build of libhfdib.so (in-tree)

Typical use (all compute runs in the library's CUDA kernels):

    from paper_2606_06135_gb300 import geometry as G
    from paper_2606_06135_gb300.hfdib import Solver, BatchSolver

    case = G.case_bfs(1024, 256)                 # lambda, wall distance, BCs
    s = Solver(case, precision=1, freeze_switch=300, p_reltol=0.2)
    rc, sweeps, res = s.solve(tol=1e-6, max_iter=20000)
    fields = s.fields()                          # ux, uy, p, k, omega, nut
    tau = s.wall_shear("ymin")                   # wall shear (Sec. 3.3)
    Fn, Ft = s.force()                           # force on the body (Eq. dragcoeff)
    Cd, Cl = s.force_coefficients()
    L, V, n = s.recirculation(x_rear=0.0)        # recirculation behind x_rear

    # many designs in one persistent launch per phase
    b = BatchSolver([G.case_grf(256, 128, seed=i) for i in range(8)], precision=1)
    b.solve(tol=1e-6, max_iter=20000)

    # dJ/dlambda of the converged state (frozen-turbulence adjoint)
    J, dJ, iters, change, status = s.adjoint_grad(tol=1e-10, objective="drag")

Options are the fields of hfdib_options (include/hfdib.h): the turbulence
model comes with the case ("laminar", "kepsilon", "komegasst", "komega",
"realizableke"); precision (0 FP64, 1 mixed), convection (0 upwind,
1 linearUpwind, 2 vanLeer, 3 limited linearUpwind), continuity_mask (0
reading A, 1 reading B), wall_distance (0 y_eff, 1 y_perp) and the solver
controls (relaxation, inner sweeps, pressure tolerance and multigrid).
"""
