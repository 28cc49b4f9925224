/*
 * hfdib.h -- C ABI of the GB300 (sm_103a) HFDIB steady-RANS SIMPLE solver.
 *
 * The library solves the steady RANS equations with the hybrid fictitious
 * domain-immersed boundary (HFDIB) treatment on a uniform Cartesian grid:
 * momentum with the immersed-boundary source f_ib and the lambda-masked
 * continuity equation (Sec. 2.1, Eq. hfdibrans), k-epsilon or k-omega SST
 * transport with wall-function values imposed at immersed-boundary cells
 * (Sec. 2.5, Eqs. imval, kws, frictionvel, omegaws), iterated with the
 * extended SIMPLE loop of Sec. 2.5.1 (Fig. simplehfdibrans).
 *
 * Conventions
 *   - Cell arrays are [nz][ny][nx] with x fastest, FP64, on the device.
 *     nz == 1 is a one-cell-thick 2D grid (dz is then taken as sqrt(dx*dy),
 *     so that the cell size V^(1/3) is sqrt(dx*dy)).
 *   - Every call returns an int status: HFDIB_OK (0) or a negative
 *     hfdib_status.  No call aborts, traps or exits.  After an error the
 *     handle stays valid (HFDIB_ERR_CUDA after a sticky CUDA error excepted).
 *   - Device pointers passed in are read on the handle's stream; the caller
 *     keeps ownership of every buffer it passes.  The handle owns its fields
 *     and scratch (allocated at create from the allocator set by
 *     hfdib_set_allocator -- cudaMalloc by default -- and freed at destroy).
 *   - All work is issued on the handle's stream (see hfdib_create); calls
 *     that return data to host memory synchronise that stream.
 */
#ifndef HFDIB_H
#define HFDIB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HFDIB_OK = 0,
    HFDIB_ERR_INVALID_ARG = -1,   /* bad sizes, NaN / out-of-range lambda, bad enum */
    HFDIB_ERR_CUDA = -2,          /* a CUDA runtime call failed                     */
    HFDIB_ERR_OOM = -3,           /* device allocation failed                       */
    HFDIB_ERR_NOT_CONVERGED = -4, /* max_iter reached above tol                     */
    HFDIB_ERR_DIVERGED = -5,      /* NaN / Inf in a residual                        */
    HFDIB_ERR_STATE_MISMATCH = -6,/* checkpoint from another grid / model           */
    HFDIB_ERR_TOO_LARGE = -7,     /* problem exceeds a fixed capacity (see below)   */
    HFDIB_ERR_TIMEOUT = -8        /* a device-wide barrier wait gave up (see below)  */
} hfdib_status;

/* Turbulence closures (Sec. 2.1 names four, each with the same HFDIB
 * treatment: imposed eps/omega rows in ic and bc cells, imposed k rows where
 * alpha_k = 1, P_ib in bc cells):
 *   KEPSILON     : standard k-epsilon (Launder-Spalding coefficients)
 *   KOMEGA_SST   : Menter's SST (needs ywall)
 *   KOMEGA       : the k-omega model of Eq. hfdibkomega as printed (no
 *                  cross-diffusion, no stress limiter), nu_t = k/omega,
 *                  beta* 0.09, C_beta1 0.072, C_alpha1 0.52, 1/sigma 0.5
 *   REALIZABLE_KE: Shih et al.'s realizable k-epsilon: C_mu = 1/(A0 + A_s U*
 *                  k/eps) (A0 = 4), eps source C1 S eps, sink C2 eps^2/(k +
 *                  sqrt(nu eps)), C2 1.9, sigma_k 1.0, sigma_eps 1.2 */
typedef enum { HFDIB_LAMINAR = 0, HFDIB_KEPSILON = 1, HFDIB_KOMEGA_SST = 2, HFDIB_KOMEGA = 3,
               HFDIB_REALIZABLE_KE = 4 } hfdib_model;

/* Domain boundary kinds (Sec. 3.1 "Boundary conditions"):
 *  INLET  : Dirichlet u = u_in, k, eps/omega from Eq. (bcspkoein); zero-gradient p
 *  OUTLET : p = p_out; zero-gradient u, k, eps/omega
 *  SLIP   : zero normal velocity, zero-gradient tangential velocity and scalars
 *  WALL   : no-slip u = 0; zero-gradient p and turbulence (Sec. 3.6)
 *  EMPTY  : the two z sides of a 2D grid
 * A wall or slip face whose cell has lambda > 0, and an inlet face whose cell
 * has lambda >= 0.5, is closed: zero gradient for all variables, no flux
 * (walls inside the solid phase, Sec. 3.1). */
typedef enum {
    HFDIB_BC_INLET = 0, HFDIB_BC_OUTLET = 1, HFDIB_BC_SLIP = 2, HFDIB_BC_WALL = 3,
    HFDIB_BC_EMPTY = 4
} hfdib_bc_kind;

typedef struct {
    int32_t nx, ny, nz;          /* cells; nz == 1 -> 2D                         */
    double x0, y0, z0;           /* lower corner                                 */
    double dx, dy, dz;           /* uniform spacings (2D: dz = sqrt(dx*dy))      */
} hfdib_grid;

typedef struct {
    int32_t face[6];             /* hfdib_bc_kind for xmin,xmax,ymin,ymax,zmin,zmax */
    double u_in[3];              /* inlet velocity                                */
    double I_in;                 /* inlet turbulence intensity (Eq. bcspkoein)    */
    double lt_in;                /* inlet turbulent length scale l_t              */
    double p_out;                /* outlet kinematic pressure                     */
    double u_ref, l_ref;         /* nu = u_ref * l_ref / Re                       */
    double u_s[3];               /* velocity of the solid (Eq. imval)             */
} hfdib_bc;

typedef struct {
    double urf_u;                /* momentum under-relaxation (default 0.7)       */
    double urf_p;                /* pressure under-relaxation (default 0.3)       */
    double urf_turb;             /* k, eps/omega under-relaxation (default 0.85)  */
    int32_t n_u;                 /* red-black Gauss-Seidel sweeps, momentum (2)   */
    int32_t n_turb;              /* red-black Gauss-Seidel sweeps, k and eps/omega (2) */
    double p_reltol;             /* pressure solve: |r| <= p_reltol |r0| (0.1)    */
    int32_t p_maxiter;           /* pressure solve iteration cap (50)             */
    int32_t precision;           /* 0: FP64 throughout (default).  1: mixed -- FP64
                                    state, assembly and defects (residuals); the
                                    red-black inner sweeps of the momentum and
                                    turbulence equations and the pressure
                                    correction solve (CG vectors and product, the
                                    multigrid V-cycle) run in FP32 on FP32
                                    corrections, with FP64 CG scalars and FP64 sums
                                    across warps and blocks; the correction solve
                                    stops at max(p_reltol, 1e-6) (needs
                                    p_persistent = 1, precond = 1); the steady state
                                    solves the FP64 equations                      */
    int32_t precond;             /* pressure preconditioner: 0 Jacobi (one launch per
                                    CG step), 1 GMG V-cycle (1)                    */
    int32_t p_check;             /* host-driven solve: read the convergence flag every
                                    p_check CG iterations; 0 = no host reads: the loop
                                    stops on the device (0) */
    int32_t mg_coarse_sweeps;    /* red-black sweeps (each way) on the coarsest level (4) */
    int32_t graph;               /* 1: run each sweep as one CUDA graph, the pressure
                                    iterations in a device-controlled while node (1);
                                    needs p_check == 0 */
    int32_t p_persistent;        /* 1: the whole pressure solve is one persistent
                                    cooperative kernel (1); 0: one launch per step */
    int32_t freeze_switch;       /* 0: the y+ <= y+_lam branch of every bc cell is
                                    re-evaluated each sweep (Eq. alphauk, default);
                                    n > 0: from sweep n on a bc cell may leave the
                                    laminar branch but not re-enter it, which ends
                                    limit cycles of the discrete switch (not part
                                    of the paper)                                  */
    int32_t frozen_turbulence;   /* 1: sweeps skip the turbulence steps (a9-a12):
                                    nu_t, k and eps/omega keep their values; the
                                    flow problem whose adjoint hfdib_adjoint_grad
                                    differentiates (0)                             */
    int32_t wall_distance;       /* distance in y+ (Eq. yplus) and omega_ib (Eq.
                                    omegaws): 0 y_eff = (y_perp + h/2)/2 (default),
                                    1 y_perp (the comparison of App. A)           */
    int32_t continuity_mask;     /* the (1 - lambda) factor of Eq. hfdibrans_2 as the
                                    pressure source m div(phiHbyA): 0 reading A,
                                    m = 1 where lambda < 1, else 0 (default);
                                    1 reading B, m = 1 - lambda (smooth in lambda:
                                    hfdib_adjoint_grad then differentiates it)     */
    int32_t convection;          /* momentum convection scheme (App. B): 0 upwind
                                    (Sec. 3.1, default); 1 linearUpwind, 2 vanLeer,
                                    3 linearUpwind with each cell's gradient
                                    scaled by its Barth-Jespersen limiter, all
                                    as a deferred correction of the bounded
                                    upwind rows from the sweep-start velocity and
                                    its Gauss-linear gradient (hfdib_adjoint_grad
                                    needs 0)                                       */
    int32_t mg_tail_cells;       /* persistent pressure solve: multigrid levels of at
                                    most this many cells run inside one thread block
                                    (in shared memory when they fit), the others
                                    as grid-wide phases (0: the library default)   */
    int32_t p_cg32;              /* precision = 1 only, kept for compatibility: the
                                    mixed pressure correction solve always runs its
                                    CG product and vectors in FP32 now, so 0 and 1
                                    behave the same.  Single problems only
                                    (hfdib_create_batch rejects 1)                */
} hfdib_options;

typedef struct hfdib_ctx* hfdib_handle;

/* Field identifiers for hfdib_get_field / hfdib_set_field. */
enum {
    HFDIB_FIELD_UX = 0, HFDIB_FIELD_UY = 1, HFDIB_FIELD_UZ = 2, HFDIB_FIELD_P = 3,
    HFDIB_FIELD_K = 4, HFDIB_FIELD_EPS = 5, HFDIB_FIELD_OMEGA = 6, HFDIB_FIELD_NUT = 7,
    HFDIB_FIELD_PHIX = 8, HFDIB_FIELD_PHIY = 9, HFDIB_FIELD_PHIZ = 10
};

/* Residual slots of the per-sweep residual vector (HFDIB_NRES doubles):
 * scaled residuals sum|b-Ax| / (sum|Ax - xbar A1| + sum|b - xbar A1|) of the
 * momentum components, pressure, eps or omega and k, evaluated at the start
 * of each solve (App. D), then the continuity error sum over lambda<1 cells
 * of |div phi| (App. D), the number of pressure iterations, the number of
 * bc cells in the laminar branch y+ <= y+_lam (Eq. alphauk) and the number
 * of bc cells whose branch changed since the previous sweep -- a non-zero
 * count late in a solve marks a limit cycle of the discrete switch. */
enum { HFDIB_RES_UX = 0, HFDIB_RES_UY = 1, HFDIB_RES_UZ = 2, HFDIB_RES_P = 3,
       HFDIB_RES_EPSW = 4, HFDIB_RES_K = 5, HFDIB_RES_CONT = 6, HFDIB_RES_PITER = 7,
       HFDIB_RES_NLAM = 8, HFDIB_RES_NSWITCH = 9, HFDIB_NRES = 10 };

/* Device memory.  By default handles and batches allocate with cudaMalloc
 * and free with cudaFree.  hfdib_set_allocator installs the caller's
 * allocator instead, process-wide, for every handle and batch created
 * afterwards; each handle and batch keeps the allocator it was created with
 * until it is destroyed (changing the setting later does not move it).
 *   alloc(bytes, stream, ctx)  : return device memory of at least `bytes`
 *                                bytes, 256-byte aligned, usable on `stream`
 *                                (the handle's stream), or NULL when there is
 *                                none (the calling entry point then returns
 *                                HFDIB_ERR_OOM).  Memory that is not 256-byte
 *                                aligned is given back and the call fails
 *                                with HFDIB_ERR_INVALID_ARG.
 *   release(ptr, bytes, stream, ctx) : take back a block from alloc; called
 *                                from hfdib_destroy / hfdib_destroy_batch (or
 *                                a failing create) after the stream has been
 *                                synchronised, so no work on the block is
 *                                pending.
 *   ctx                        : passed through unchanged.
 * Both NULL restores cudaMalloc / cudaFree; exactly one NULL is
 * INVALID_ARG.  Pinned host staging buffers are not affected.  The Python
 * binding installs PyTorch's caching allocator. */
typedef void* (*hfdib_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*hfdib_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
int hfdib_set_allocator(hfdib_alloc_fn alloc, hfdib_free_fn release, void* ctx);

/* Fill *opt with the defaults listed in hfdib_options. */
void hfdib_default_options(hfdib_options* opt);

/* hfdib_create -- set up a solver for one lambda field.
 *   grid     : sizes and spacings; nx, ny >= 2; nz >= 1.
 *   lambda   : device pointer, nx*ny*nz doubles in [0, 1] (Eq. lambda); copied.
 *   ywall    : device pointer to the wall distance used by the SST blending
 *              functions (nullable; required for HFDIB_KOMEGA_SST); copied.
 *   model    : hfdib_model.
 *   Re       : Reynolds number; nu = bc->u_ref * bc->l_ref / Re.
 *   bc       : boundary description (not NULL).
 *   opt      : options (NULL -> defaults).
 *   stream   : cudaStream_t used for every call on the handle.  NULL: the
 *              handle creates and owns a non-blocking stream (the legacy
 *              default stream cannot be captured into a CUDA graph).
 *   out      : receives the handle.
 * At create the library classifies cells into ic/bc/fc (Sec. 2.3), builds
 * the boundary-cell geometry -- normal, in-solid neighbour, y_perp, y_eff,
 * interpolation stencils (Sec. 2.4-2.5) -- and sets the initial state: u_in
 * outside the solid and u_s in it, p = 0, k and eps/omega at their inlet
 * values (k = 0 in the solid).  Errors: INVALID_ARG for bad sizes / enums or
 * lambda outside [0, 1] or NaN; OOM; CUDA. */
int hfdib_create(const hfdib_grid* grid, const double* lambda, const double* ywall,
                 int model, double Re, const hfdib_bc* bc, const hfdib_options* opt,
                 void* stream, hfdib_handle* out);

/* hfdib_simple_sweep -- run n_sweeps iterations of the extended SIMPLE loop
 * (Fig. simplehfdibrans, Sec. 2.5.1): set alpha_u and compute u_ib, momentum
 * predictor, correction u += alpha_u (u_ib - u) (Eq. corru), pressure
 * corrector with the lambda-masked continuity, velocity/flux update, omega_ib
 * (eps_ib) and P_ib, the eps/omega equation with its imposed rows, k_ib, the
 * k equation and the k correction.
 *   residuals : host pointer to HFDIB_NRES doubles receiving the residuals of
 *               the last sweep (nullable: then nothing is copied back and the
 *               call returns without waiting for the GPU). */
int hfdib_simple_sweep(hfdib_handle h, int n_sweeps, double* residuals);

/* hfdib_pressure_trace -- runs ONE sweep (host-driven, like
 * hfdib_simple_sweep with graph capture off for that sweep; the solution
 * advances) and records the phases of its persistent pressure kernel: after
 * every device-wide barrier, block 0 appends a (phase, time) pair, the time
 * from %globaltimer in ns.  Phases: 0 start, 1 level-0 operator built, 2 a
 * coarse level built, 3 initial residual, 4 first black half sweep of
 * level 0, 5 a restriction, 6 a black half sweep of a coarse level, 7 the
 * one-block coarse tail, 8 a prolongation with its black half sweep, 9 a red
 * half sweep going up, 10 the final red half sweep of level 0 (r.z), 11 the
 * CG product (d, q, d.q), 12 the CG update (p, r, r.r), 13 end; and, within
 * block 0 without a barrier, 14 its share of the initial residual done, 15
 * its tail table set up, 16 a tail level built, 17 the tail input copied
 * in, 18 the tail computed, and inside the tail 19 a level down (block
 * wide), 20 the coarsest levels, 21 a level up (block wide), 22 the cell
 * loop of a CG product or update done, 23 its block partial written.  A
 * measurement aid for the pressure solve (it allocates a small device
 * buffer for the call).
 *   out      : HOST, 2 * capacity int64: tag, ns, tag, ns, ...
 *   capacity : pairs (1 .. 2^20); later phases are dropped
 *   n_out    : host, pairs written (nullable)
 * Errors: INVALID_ARG (NULL, bad capacity, a handle without the persistent
 * pressure kernel), OOM, CUDA, and the sweep's own statuses. */
int hfdib_pressure_trace(hfdib_handle h, int64_t* out, int capacity, int* n_out);

/* Barrier timeouts.  The persistent pressure kernels (one cooperative launch
 * per pressure solve, single problem or batch) separate their phases by
 * device-wide barriers.  Every wait at such a barrier polls at most a fixed
 * number of times (default 2^26, about 0.1-1 s); a wait that runs out sets
 * the kernel's error word, every block that then finds the word set leaves
 * the kernel at its next barrier, and the rest of the sweep runs on the
 * partial pressure solution.  The next call that reads residuals back
 * (hfdib_simple_sweep with a residual buffer, hfdib_solve_steady,
 * hfdib_batch_sweep / hfdib_batch_solve_steady) returns HFDIB_ERR_TIMEOUT
 * once and clears the flag; the handle stays usable (restore a checkpoint
 * with hfdib_set_state to discard the incomplete sweep).  No kernel waits
 * without a bound and none traps.
 * hfdib_set_barrier_polls sets the poll budget of each wait (polls > 0) or
 * restores the default (polls == 0); a budget of 1 makes every wait that is
 * not already complete give up, which is how a timeout is exercised. */
int hfdib_set_barrier_polls(hfdib_handle h, int64_t polls);

/* hfdib_solve_steady -- sweep until the largest scaled residual (momentum,
 * pressure, turbulence) is <= tol, or max_iter sweeps.  Residuals are read
 * back every check_every sweeps (<= 0 -> 10).  Returns HFDIB_OK,
 * HFDIB_ERR_NOT_CONVERGED or HFDIB_ERR_DIVERGED.  iters_out and final_res
 * (HFDIB_NRES doubles) are host pointers and nullable. */
int hfdib_solve_steady(hfdib_handle h, double tol, int max_iter, int check_every,
                       int* iters_out, double* final_res);

/* Objectives of hfdib_adjoint_grad, and the largest GMRES restart length. */
enum { HFDIB_OBJ_PRESSURE_DROP = 0, HFDIB_OBJ_DRAG = 1 };
enum { HFDIB_GMRES_MAX_RESTART = 200 };

/* hfdib_adjoint_grad -- frozen-turbulence discrete adjoint of the converged
 * state: the gradient of an objective J with respect to the indicator lambda.
 * The paper has no adjoint; this entry point differentiates its discrete
 * method.  Hold fixed nu_t, k, eps/omega, the cell groups (Sec. 2.3), the
 * wall-function branch of each bc cell (Eq. alphauk), the closed faces and,
 * under reading A, the continuity mask.  Then the converged state is a fixed
 * point of the sweep's momentum-pressure part (steps a2-a8 of Fig.
 * simplehfdibrans), and lambda moves it through the imposed velocity u_ib of
 * the laminar-branch bc cells: the normal n = -grad(lambda)/|grad(lambda)|
 * (Eq. yorthoaux), y_perp (Eq. yortho) and the interpolation of Sec. 2.5;
 * under reading B (options.continuity_mask = 1) also through the pressure
 * source (1 - lambda) div(phiHbyA), which reaches every cell.
 * The adjoint psi of that fixed point solves (I - G_x^T) psi = J_x^T.  G_x^T
 * is one transposed sweep: reverse accumulation through the same red-black
 * momentum passes, with exact pressure solves, run as one CUDA graph.
 * Then dJ/dlambda = psi^T dG/dlambda.
 *   objective  : HFDIB_OBJ_PRESSURE_DROP, J = mean p over the cells of the open
 *                inlet faces minus mean p over the cells of the outlet faces;
 *                HFDIB_OBJ_DRAG, J = the x force of the fluid on the body:
 *                minus the sum over the imposed rows (in-solid cells and
 *                laminar-branch bc cells) of the x-momentum row residual
 *                aP u~ + sum a_N u~_N - b0 + V dp/dx, the forcing of Eq.
 *                hfdibrans_1 applied there (u~: u_s, u_ib or u).  The drag
 *                also depends on lambda directly through u_ib, which the
 *                gradient includes.
 *   gmres_restart : 0 (recommended): the reverse fixed point
 *                psi <- G_x^T psi + J_x^T; stop when max|psi_new - psi| <=
 *                tol max|psi| (checked every 10 iterations).  m > 0:
 *                GMRES(m) on (I - G_x^T) psi = J_x^T; stop when the residual
 *                2-norm is <= tol |J_x^T| (restarted GMRES can stagnate on
 *                these operators).  At most HFDIB_GMRES_MAX_RESTART.  Either
 *                way each adjoint pressure solve is warm-started from the
 *                previous one and accurate to 1e-12 of its right-hand side.
 *   tol, max_iter : tolerance as above; max_iter caps the transposed sweeps;
 *                max_iter = 0 only evaluates J (dJ_dlambda may then be NULL)
 *   dJ_dlambda : DEVICE pointer, N doubles (cell order of lambda), caller-owned
 *   J_out, iters_out (transposed sweeps run), change_out (final relative
 *                residual or change) : host pointers, nullable
 * Call it on a converged state (hfdib_solve_steady to a tight tolerance): the
 * gradient is that of the fixed point, and its error follows the residual.
 * 2D and 3D grids; the upwind convection scheme only (INVALID_ARG
 * otherwise).  The state is left unchanged.
 * Returns HFDIB_OK, HFDIB_ERR_NOT_CONVERGED (gradient of the last iterate
 * still written), HFDIB_ERR_DIVERGED, HFDIB_ERR_INVALID_ARG, or CUDA/OOM errors.
 * The first call allocates about 90 doubles per cell of work arrays (plus
 * (m + 2) flat state vectors for GMRES), which live until hfdib_destroy. */
int hfdib_adjoint_grad(hfdib_handle h, int objective, double tol, int max_iter, int gmres_restart,
                       double* dJ_dlambda, double* J_out, int* iters_out, double* change_out);

/* hfdib_ib_force -- force of the fluid on the immersed body at the current
 * state (Eq. dragcoeff, Eq. dlcoeffs: the integrand f_tot = f_n + f_t).  The
 * surface integral over the fluid-solid interface is taken through the
 * momentum balance of the imposed rows (in-solid cells and laminar-branch bc
 * cells): the force is minus the sum over those rows of the momentum row
 * residual aP u~ + sum a_N u~_N - b0 + V grad p, the forcing of Eq.
 * hfdibrans_1 applied there, with the imposed values u~ and grad u of the
 * current state (the rows of the next sweep).
 *   force : HOST pointer, 6 doubles: [0..2] the pressure part -sum V grad p
 *           (f_n), [3..5] the rest, viscous and convective (f_t); components
 *           beyond the grid's dimensions are 0.  Kinematic units (pressure /
 *           rho times area).  C_d = 2 F.v_d / (A_ref |u_in|^2) with
 *           F = force[0..2] + force[3..5].
 * Waits for the handle's stream.  Leaves the state unchanged (it refreshes
 * the imposed fields and grad u, which the next sweep recomputes from the
 * same state).  Errors: INVALID_ARG (NULL), CUDA. */
int hfdib_ib_force(hfdib_handle h, double* force);

/* hfdib_force_coefficients -- drag and lift coefficients of the force of
 * hfdib_ib_force: C_d = 2 F.v_d / (A_ref |u_in|^2) with v_d = (1, 0, 0)
 * (Eq. dragcoeff) and C_l = 2 F.v_l / (A_ref |u_in|^2) with v_l =
 * (-sin gamma, cos gamma, 0) (Eq. dlcoeffs), F = f_n + f_t.
 *   A_ref  : reference area; 0 selects the paper's l_ref dz, the reference
 *            length times the cell depth (one-cell-thick 2D grids only)
 *   gamma  : angle of attack in radians (the lift direction)
 *   coeffs : HOST pointer, 2 doubles: C_d, C_l
 * Waits for the handle's stream; leaves the state unchanged (as
 * hfdib_ib_force).  Errors: INVALID_ARG (NULL, A_ref < 0, A_ref = 0 on a 3D
 * grid, zero inlet velocity, non-finite gamma), CUDA. */
int hfdib_force_coefficients(hfdib_handle h, double A_ref, double gamma, double* coeffs);

/* hfdib_wall_shear -- wall shear stress along one no-slip domain side
 * (Sec. 3.3, tau_w = nu du/dn at the wall): the shear of the discrete wall
 * flux, (nu + nu_t,P) u_P / (Delta/2) per tangential component, u_P the
 * velocity of the wall cell as its row sees it.  Zero on closed faces (a
 * wall inside the solid) and for the normal component.  C_f = 2 tau_w /
 * |u_in|^2.
 *   side  : 0..5 = x-, x+, y-, y+, z-, z+; must be an HFDIB_BC_WALL side of
 *           the grid's dimensions (INVALID_ARG otherwise)
 *   tau   : DEVICE pointer, 3 * n_faces doubles, caller-owned: component q of
 *           face f at tau[q * n_faces + f]; faces in the order of the wall's
 *           cells (the two tangential indices, the lower direction fastest).
 *           n_faces = the product of the other two cell counts.  NULL with
 *           n_faces_out set only reports the size.
 *   n_faces_out : host pointer, nullable
 * Asynchronous on the handle's stream. */
int hfdib_wall_shear(hfdib_handle h, int side, double* tau, int64_t* n_faces_out);

/* hfdib_recirculation -- size of the recirculation region behind a body
 * (Sec. 3.6): the cells outside the solid (not in-solid cells) whose centre
 * lies downstream of x_rear (x_c > x_rear) and whose u_x is negative.
 *   x_rear : x of the body's rear end (finite)
 *   out    : HOST pointer, 3 doubles: [0] length = the largest x_c - x_rear
 *            over those cells (0 when there is none), [1] volume = their
 *            number times the cell volume, [2] their number.
 * Waits for the handle's stream.  Errors: INVALID_ARG (NULL, NaN), CUDA. */
int hfdib_recirculation(hfdib_handle h, double x_rear, double* out);

/* Copy a field (HFDIB_FIELD_*) device-to-device into dst (caller-owned, sized
 * like the field: cells, or faces (nx+1)*ny*nz / nx*(ny+1)*nz / nx*ny*(nz+1)). */
int hfdib_get_field(hfdib_handle h, int field, double* dst);
/* Overwrite a field from a caller device buffer (used to restart or to set a
 * test state).  nu_t is recomputed by the next sweep. */
int hfdib_set_field(hfdib_handle h, int field, const double* src);

/* Cell groups and boundary-cell list (Sec. 2.3-2.4).
 *   tags     : device, N bytes: 0 fc, 1 bc, 2 ic (nullable)
 *   n_bc     : host, receives the number of bc cells (nullable)
 * hfdib_get_bc_list copies, for the n_bc boundary cells in increasing cell
 * order, device arrays (each nullable):
 *   ints     : int64 [n_bc][8] = cell, in-solid neighbour (-1 none), y_perp
 *              case (0,1,2), clamped flag, X1 base cell (i,j,k), and the
 *              wall-function branch of the last sweep (1: laminar, y+ <=
 *              y+_lam, Eq. alphauk; 0: log) -- X2 base (i,j,k) is in ints2 ;
 *   ints2    : int64 [n_bc][3] = X2 base (i,j,k)
 *   reals    : double [n_bc][14] = n (3), y_perp, y_eff, wS, w1, w2,
 *              t1 (3), t2 (3). */
int hfdib_get_tags(hfdib_handle h, uint8_t* tags, int64_t* n_bc);
int hfdib_get_bc_list(hfdib_handle h, int64_t* ints, int64_t* ints2, double* reals);

/* Residual history: copies the residual vectors of the last `count` sweeps
 * (at most 1024 are kept) into host memory, oldest first; *n_out = rows. */
int hfdib_get_history(hfdib_handle h, int count, double* host, int* n_out);

/* Checkpoint: the complete FP64 state (u, p, phi, k, eps, omega, nu_t and the
 * sweep counter).  hfdib_get_state with buf == NULL returns the size in
 * *bytes.  Buffers are host memory, caller-owned; both calls wait for the
 * handle's stream.  Resuming from a saved state reproduces the uninterrupted
 * run bit for bit.  Layout: eight int64 header words (magic, nx, ny, nz,
 * model, sweep counter, total bytes, 0), then the arrays in the order above.
 * Errors: INVALID_ARG (NULL; get_state with *bytes below the size),
 * STATE_MISMATCH (set_state with a size, magic word, grid or model other
 * than the handle's; the size is checked before the header is read), CUDA. */
int hfdib_get_state(hfdib_handle h, void* buf, size_t* bytes);
int hfdib_set_state(hfdib_handle h, const void* buf, size_t bytes);

/* Kernel launches of one sweep outside the pressure iterations, and of one
 * pressure (CG + V-cycle) iteration. */
int hfdib_get_launch_counts(hfdib_handle h, int64_t* per_sweep, int64_t* per_pcg_iteration);

/* Number of sweeps run so far and of kernel launches issued by the last
 * hfdib_simple_sweep / hfdib_solve_steady call. */
int hfdib_get_counters(hfdib_handle h, int64_t* sweeps, int64_t* launches);

/* Kernel classes timed by hfdib_profile_sweeps. */
enum { HFDIB_K_IMPOSED = 0,   /* a1, a2 and the residual means                */
       HFDIB_K_GRAD_U = 1,    /* velocity gradient (a3, a9)                   */
       HFDIB_K_MOM_ASM = 2,   /* a3 momentum assembly + momentum residual      */
       HFDIB_K_MOM_SMOOTH = 3,/* a4 red-black sweeps of the predictor         */
       HFDIB_K_HBYA = 4,      /* a6 rAU, HbyA, phiHbyA                        */
       HFDIB_K_P_COEF = 5,    /* a7 pressure operator on all levels           */
       HFDIB_K_PCG = 6,       /* a7 CG kernels (init, products, updates)      */
       HFDIB_K_VCYCLE = 7,    /* a7 initial multigrid V-cycle                 */
       HFDIB_K_UPDATE = 8,    /* a8 flux / pressure / velocity update         */
       HFDIB_K_TURB_PREP = 9, /* a9 production, P_ib, blending, k sources     */
       HFDIB_K_SCAL_ASM = 10, /* a10/a11 assembly + residuals                 */
       HFDIB_K_SCAL_SMOOTH = 11, /* a10/a11 red-black sweeps                  */
       HFDIB_K_TURB_FINAL = 12,  /* a11 k bound + correction, a12 nu_t         */
       HFDIB_K_SWEEP_END = 13,   /* a12 residual record                       */
       HFDIB_K_COUNT = 14 };

/* Run n_sweeps host-driven sweeps with a CUDA event pair around every
 * launch group and return, per kernel class, the summed device time in
 * microseconds (total_us) and the number of timed launch groups (calls).
 * Arrays are host memory of n_classes >= HFDIB_K_COUNT entries.  The sweeps
 * advance the solution exactly like hfdib_simple_sweep. */
int hfdib_profile_sweeps(hfdib_handle h, int n_sweeps, double* total_us, int64_t* calls, int n_classes);

/* hfdib_classify_noalloc -- cell groups and the ordered boundary-cell list
 * for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is the allocation-free form of the classification step
 * of hfdib_create, for callers whose device memory belongs to another
 * framework's pool, that run under a fixed memory budget, or that must not
 * enter the driver's allocator.  It allocates nothing: the compaction's
 * per-block counts live in a fixed array inside the library (room for
 * 2^24 cells; every GPU that loads the library keeps it until exit).
 *   grid      : sizes (spacings are not used).
 *   lambda    : device, nx*ny*nz doubles in [0, 1].
 *   tags      : device, nx*ny*nz bytes out: 0 fc, 1 bc, 2 ic (Sec. 2.3),
 *               identical to hfdib_get_tags of a handle made from lambda.
 *   bc_cells  : device, bc_capacity int32 out: the bc cells in increasing
 *               cell order, identical to the cell column of hfdib_get_bc_list.
 *   n_bc      : host, receives the number of bc cells.
 *   stream    : cudaStream_t of the current device; the call synchronises
 *               it before returning.
 * Errors: INVALID_ARG (NULL pointers, bad sizes, a stream of another device,
 * or a lambda value outside [0, 1] or NaN -- *n_bc is then 0 -- as
 * hfdib_create rejects such a field); TOO_LARGE when nx*ny*nz > 2^24, or when
 * n_bc > bc_capacity (*n_bc is then set and the list is truncated); CUDA
 * (checked right after the launches, which also consumes a launch error an
 * earlier, unrelated call may have left pending).
 * The first call on a device looks up the fixed array's device address and
 * should not be made inside a stream capture.  Calls share the array: two
 * calls that overlap on the GPU (unordered streams) race. */
int hfdib_classify_noalloc(const hfdib_grid* grid, const double* lambda, uint8_t* tags, int32_t* bc_cells,
                           int64_t bc_capacity, int64_t* n_bc, void* stream);

/* ---------------------------------------------------------------------------
 * Batches: B independent problems (design candidates, angles of attack; grid
 * sizes may differ) advanced together.  Each sweep runs parts A and B of the
 * extended SIMPLE loop of all problems concurrently and solves all their
 * pressure equations in ONE persistent cooperative launch (shared grid
 * barriers, per-problem convergence); the batched sweep is one CUDA graph.
 * All problems share the options (precond must be 1).  B <= 64.
 *   grids, bcs, Re : host arrays of B entries.
 *   lambdas, ywalls: host arrays of B device pointers (ywalls nullable, or
 *                    entries nullable unless the model is SST).
 * The handles returned by hfdib_batch_handle give field access to problem i;
 * do not sweep them individually. */
typedef struct hfdib_batch_ctx* hfdib_batch;

/* hfdib_create_batch -- B problems created as hfdib_create would create
 * them, on one stream (stream NULL: the batch creates and owns a
 * non-blocking stream).  *out is NULL on failure.  Errors: INVALID_ARG (NULL
 * out, grids, lambdas, Re or bcs; B < 1 or B > 64; precond != 1; p_cg32 != 0;
 * 2D and 3D grids mixed; or an error of hfdib_create for one problem, whose
 * status is returned), TOO_LARGE (B above the GPU's SM count: problem b's
 * coarse tail runs on block b), OOM, CUDA. */
int hfdib_create_batch(int B, const hfdib_grid* grids, const double* const* lambdas, const double* const* ywalls,
                       int model, const double* Re, const hfdib_bc* bcs, const hfdib_options* opt, void* stream,
                       hfdib_batch* out);
/* residuals: host, B * HFDIB_NRES doubles (nullable).  Errors: INVALID_ARG
 * (NULL, n_sweeps < 0), DIVERGED (a non-finite residual), TIMEOUT, CUDA. */
int hfdib_batch_sweep(hfdib_batch b, int n_sweeps, double* residuals);
/* Sweep until every problem's largest scaled residual is <= tol (or
 * max_iter); iters_out (host, B ints) receives the sweep at which each
 * problem first met tol; final_res host B * HFDIB_NRES (both nullable). */
int hfdib_batch_solve_steady(hfdib_batch b, double tol, int max_iter, int check_every, int* iters_out,
                             double* final_res);
/* The handle of problem i (0 <= i < B, else INVALID_ARG).  It belongs to
 * the batch and lives until hfdib_destroy_batch: do not destroy it. */
int hfdib_batch_handle(hfdib_batch b, int i, hfdib_handle* out);

/* Autotuner of the batched pressure kernel: threads per block {512, 1024},
 * coarse-tail threshold {256, 1024, 4096 cells} (the tail runs in one block,
 * in shared memory when it fits) and coarsest-level sweeps {2, 4, 8}.  Every
 * candidate is timed over trial_sweeps real sweeps (the solution advances),
 * the fastest is kept for the batch and cached for later batches of the same
 * shape in this process.  Changing the block size changes the summation
 * order of the reductions (round-off level). */
typedef struct {
    int32_t threads, tail_cells, coarse_sweeps;
    double us_per_sweep;
    int32_t candidates;
} hfdib_tune;
int hfdib_batch_autotune(hfdib_batch b, int trial_sweeps, hfdib_tune* best);
/* the batch's barrier poll budget, as hfdib_set_barrier_polls */
int hfdib_batch_set_barrier_polls(hfdib_batch b, int64_t polls);
/* Waits for the batch's stream, destroys its problem handles and releases
 * every block through the allocator the batch was created with; NULL is a
 * no-op. */
void hfdib_destroy_batch(hfdib_batch b);

/* A static description of a status code ("unknown error" for any other
 * value); never NULL. */
const char* hfdib_error_string(int code);
/* Waits for the handle's stream and releases all its device memory through
 * the allocator it was created with; NULL is a no-op. */
void hfdib_destroy(hfdib_handle h);

#ifdef __cplusplus
}
#endif
#endif /* HFDIB_H */
