// kernels.cuh -- device data structures and kernel launchers of the sweep.
#pragma once
#include "common.cuh"

namespace hf {

// compacted boundary-cell list (bc cells in increasing cell order)
struct BcList {
    int nbc;
    int* cell;      // cell index
    int* nbr;       // in-solid neighbour (-1: none)
    int* cas;       // y_perp case 0 (a), 1 (b), 2 (c)
    int* clamped;   // y_perp clamped at 1e-3 h
    int* b1;        // [3*nbc] base cell of the X1 stencil
    int* b2;        // [3*nbc] base cell of the X2 stencil
    int* lamb;      // per sweep: 1 if y+ <= y+_lam (laminar branch)
    double* n;      // [3*nbc] outer unit normal
    double* yp;     // y_perp
    double* ye;     // y_eff
    const double* ywf;  // the distance the wall functions use: ye (Eq. yplus) or yp (App. A)
    double *wS, *w1, *w2;  // quadratic weights
    double* t1;     // [3*nbc]
    double* t2;     // [3*nbc]
    double* yplus;  // per sweep
};

// device scalar slots
enum {
    SC_WMAX = 0,                 // max over bc u fc of omega_old / eps_old
    SC_SUM_U = 1,                // sums of substituted u_x, u_y, u_z, p, k, eps|omega (6)
    SC_SUM_P = 4, SC_SUM_K = 5, SC_SUM_W = 6,
    SC_RES_U = 8,                // 9: |r|, |Ax-A1 xbar|, |b-A1 xbar| per component
    SC_RES_W = 20,               // 3
    SC_RES_K = 23,               // 3
    SC_CONT = 26,
    SC_PCG_RZ = 28,              // r.z of the current iterate
    SC_PCG_RZP = 29,             // previous r.z
    SC_PCG_RZN = 30,             // r.z of the new residual   (RZN, RR adjacent)
    SC_PCG_RR = 31,              // r.r of the new residual
    SC_PCG_DQ = 32,
    SC_PCG_IT = 33,              // iteration counter
    SC_PCG_DONE = 34,            // 1: converged or capped
    SC_PCG_TOL2 = 35,            // p_reltol^2 |r0|^2
    SC_PCG_ITERS = 36,           // iterations of the last solve
    SC_NSWEEP = 37,              // sweeps run (history slot)
    SC_NLAM = 38,                // bc cells in the laminar branch this sweep
    SC_NSWITCH = 39,             // bc cells whose branch changed
    SC_TIMEOUT = 46,             // 1 once a persistent kernel's grid barrier gave up
    SC_PCG_INIT = 40,            // r0.z0, r0.r0, b.b, then the 3 scaled-residual sums of p
    SC_FORCE = 52,               // 6: force on the body, pressure part xyz then the rest xyz
    SC_RECIRC = 58,              // largest x - x_rear of a recirculating cell
    SC_COEF = 60,                // 2: drag and lift coefficients of the force
    // the stop test of a batch solve, checked on the device at every sweep end
    SC_STOP_TOL = 64,            // tolerance on the largest scaled residual
    SC_STOP_ON = 65,             // 1 while a batch solve runs
    SC_DONE = 66,                // 1 converged, 2 diverged (non-finite residual); the problem then skips
    SC_DONE_AT = 67,             // the sweep count at which it stopped
    SC_NSCAL = 72
};

struct Fields {
    double* u[3];
    double* us[3];     // predictor output u*
    double* p;
    double* pn;        // pressure-equation solution
    double* pr;        // relaxed pressure (swap buffer)
    double* phi[3];
    double* phiH[3];
    double* HbyA[3];
    double* rAU;
    double* bm[3];
    double* mrow;      // [9][N] momentum rows of the sweep, written by the
                       // assembly for HbyA: aP per component (3), a per side (6)
    double* k;
    double* w;         // eps (k-epsilon) or omega (SST)
    double* w2;        // the other one (omega for k-eps, eps for SST), diagnostic
    double* nut;
    double* uib[3];
    double* kib;
    double* wib;
    double* G;         // 9*N velocity gradient, G[(3a+b)N + c] = d u_b / d x_a
    double* Glim;      // 9*N its cell-limited copy (convection scheme 3 only)
    double* Pk;
    double* S2;
    double* gam;       // scalar equation diffusivity
    double* gamk;
    double* sp;        // extra implicit diagonal (integrated)
    double* src;       // explicit source (integrated)
    double* asus;      // realizable k-eps: A_s U* of the velocity gradient (for nu_t)
    const double* lam; // lambda (the continuity mask of reading B)
    double* bt;        // relaxed right-hand side
    double* diag;      // relaxed diagonal
    double* ywall;
    double* iyw;       // k-omega SST: 1 / max(ywall, 1e-3 h), set at create (ywall is fixed)
    uint16_t* flags;
    // pressure solver
    double* prhs;
    double* pdiag;
    double* r;
    double* r_alt;     // FP64 path: the second CG residual buffer of the persistent solve
    double* z;
    double* d[2];
    double* q;
    // FP32 mirrors and corrections of the mixed-precision path (precision = 1):
    // the inner red-black sweeps solve for corrections in FP32, the defects
    // (right-hand sides) come from the FP64 assembly
    float* phi32[3];
    float* nut32;
    float* gam32;
    float* gamk32;
    float* r32[3];     // FP64 defect of each momentum component / scalar, rounded
    float* d32[3];     // FP32 correction
    float* diag32;     // relaxed diagonal of the scalar equation
    float* z32;        // preconditioned residual of the CG (mixed path)
    float* pd32[2];    // FP32 CG search directions of the pressure correction solve
    float* pq32;       // FP32 A d of the pressure correction solve
    float* px32;       // FP32 pressure correction (pn = p + px32)
    float* pr32;       // the second FP32 CG residual buffer of the persistent solve
    int mixed;
    // scalars and reductions
    double* scal;
    double* partials;
    unsigned int* counters;
};

// one multigrid level of the pressure operator (level 0 = the fine grid),
// in FP64 (the plain path) or FP32 (the preconditioner of the mixed path)
template <typename T>
struct LevelT {
    int nx, ny, nz;
    long long N;
    T* cf[3];   // face coefficients, face layout of the level
    T* diag;
    T* idg;     // 1/diag (0 where diag is 0)
    T* x;       // correction (level 0: z)
    T* b;       // right-hand side (level 0: r)
};
using Level = LevelT<double>;
using Level32 = LevelT<float>;
constexpr int MAX_LEVELS = 16;
constexpr long long TAIL_CELLS = 4096;
// persistent pressure solve: default largest level run by block 0 alone (in
// shared memory when the levels fit; the V-cycle is the same either way)
constexpr long long PT_DEFAULT_TAIL_CELLS = 4096;
template <typename T>
struct MgLevelsT {
    int nl;
    LevelT<T> lv[MAX_LEVELS];
};
using MgLevels = MgLevelsT<double>;
using MgLevels32 = MgLevelsT<float>;

struct Params {
    int model;
    double urf_u, urf_p, urf_turb;
    double iurf_u, iurf_t;   // 1/urf
    double rlx_u, rlx_t;     // (1 - urf)/urf
    double k_in, w_in;   // inlet k and eps (k-eps) or omega (SST)
};

// ib.cu
void launch_classify(const Grid& g, const double* lam, uint16_t* flags, cudaStream_t s);
void launch_compact_bc(const Grid& g, const uint16_t* flags, int* counts, int* total, int* cells,
                       cudaStream_t s);
void launch_bc_geometry(const Grid& g, const double* lam, const uint16_t* flags, const BcList& bl,
                        cudaStream_t s);
void launch_max_not_ic(const Grid& g, const uint16_t* flags, const double* w, double* partials,
                       unsigned int* counter, double* out, cudaStream_t s);
void launch_imposed(const Grid& g, int model, int freeze, const BcList& bl, uint16_t* flags, double* scal, const double* ux,
                    const double* uy, const double* uz, const double* k, double* uibx, double* uiby,
                    double* uibz, double* kib, double* wib, cudaStream_t s);
void launch_export_bc(const BcList& bl, long long* ints, long long* ints2, double* reals, cudaStream_t s);

// flow.cu
void launch_init_flux(const Grid& g, const Fields& F, cudaStream_t s);
void launch_means(const Grid& g, const Params& P, const Fields& F, cudaStream_t s);
void launch_grad_u(const Grid& g, const Fields& F, cudaStream_t s);
void launch_mom_asm(const Grid& g, const Params& P, const Fields& F, cudaStream_t s);
void launch_conv_limit(const Grid& g, const Fields& F, cudaStream_t s);
void launch_ib_force(const Grid& g, const Fields& F, cudaStream_t s);
// C_d, C_l (Eqs. dragcoeff, dlcoeffs) from the force in scal[SC_FORCE..]: into scal[SC_COEF..]
void launch_force_coefficients(const Fields& F, double A_ref, double U2, double gamma, cudaStream_t s);
void launch_recirc(const Grid& g, const Fields& F, double x_rear, unsigned int* count, cudaStream_t s);
void launch_wall_shear(const Grid& g, const Fields& F, int side, long long nf, double* tau, cudaStream_t s);
void launch_mom_smooth(const Grid& g, const Params& P, const Fields& F, int colour, cudaStream_t s);
void launch_hbya(const Grid& g, const Params& P, const Fields& F, cudaStream_t s);
void launch_phiH(const Grid& g, const Fields& F, cudaStream_t s);
void launch_update(const Grid& g, const Params& P, const Fields& F, const Level& L0, cudaStream_t s);
// res_out: HFDIB_NRES residuals then one slot that is 1 once a persistent
// kernel's barrier wait gave up (err: that kernel's error word, nullable);
// the flag stays set in the scalars until the host clears it
void launch_sweep_end(const Params& P, const Fields& F, int dims, const int* err, double* res_out, double* hist,
                      int nhist, cudaStream_t s);

// pressure.cu
void launch_p_coef(const Grid& g, const MgLevels& M, const double* rAU, int ntail_from, cudaStream_t s);
void launch_vcycle(const Grid& g, const MgLevels& M, int ntail_from, const Fields& F, double* dot_out,
                   int coarse_sweeps, cudaStream_t s);
void launch_pcg_init(const Grid& g, const Fields& F, const MgLevels& M, int jacobi, cudaStream_t s);
void launch_pcg_start(const Fields& F, int jacobi, double reltol, int maxit, cudaGraphConditionalHandle h,
                      int use_cond, cudaStream_t s);
void launch_pcg_body(const Grid& g, const Fields& F, const MgLevels& M, int ntail_from, int jacobi,
                     int coarse_sweeps, int maxit, cudaGraphConditionalHandle h, int use_cond, cudaStream_t s);

// persistent pressure solve (pcgb.cu): default poll budget of one wait at its
// grid barrier (about 0.1-1 s); a wait that runs out sets the kernel's error word.
constexpr long long BARRIER_POLLS = 1ll << 26;
constexpr int PT_THREADS = 1024;                 // threads per block of a single problem's solve
constexpr size_t PT_SMEM_BUDGET = 160 * 1024;    // shared memory of one problem's tail levels
// Phase tags of the persistent pressure kernel's trace (see hfdib_pressure_trace)
enum { PH_START = 0, PH_BUILD0 = 1, PH_COARSEN = 2, PH_R0 = 3, PH_VC_SMOOTH0 = 4, PH_VC_RESTRICT = 5,
       PH_VC_SMOOTH = 6, PH_VC_TAIL = 7, PH_VC_PROLONG = 8, PH_VC_UPSMOOTH = 9, PH_VC_FINAL = 10,
       PH_CG_PRODUCT = 11, PH_CG_UPDATE = 12, PH_END = 13,
       // within block 0 (no barrier): its r0 share done, its tail table set
       // up, a tail level built, the tail input copied in, the tail computed
       PH_R0_SHARE = 14, PH_TB_TABLE = 15, PH_TB_LEVEL = 16, PH_TAIL_IN = 17, PH_TAIL_DONE = 18,
       // inside the tail (pcg_ops.cuh): a block-wide level down, the coarsest
       // part, a block-wide level up
       PH_TL_DOWN = 19, PH_TL_WARP = 20, PH_TL_UP = 21,
       // within block 0: the cell loop of a CG phase done, its block partial written
       PH_B0_LOOP = 22, PH_B0_PART = 23 };
void launch_p_coef32(const Grid& g, const MgLevels& M, const MgLevels32& M32, cudaStream_t s);
// mixed path: FP32 red-black pass on the momentum correction; finalize (the
// last pass of each colour) adds the correction to u* in FP64
void launch_mom_smooth32(const Grid& g, const Params& P, const Fields& F, int colour, int zero_init, int finalize,
                         cudaStream_t s);
void launch_scal_smooth32(const Grid& g, const Params& P, const Fields& F, int eq, int colour, int zero_init,
                          cudaStream_t s);

// pcgb.cu: the persistent pressure solve of a batch of B >= 1 problems
// (a single problem is a batch of one); descriptors as below, all problems of
// a launch 2D or all 3D
size_t pcgb_describe64(void* dst, const Grid& g, const Fields& F, const MgLevels& M, double* part,
                       long long tail_cells, size_t smem_budget);
size_t pcgb_describe32(void* dst, const Grid& g, const Fields& F, const MgLevels& M, const MgLevels32& M32,
                       double* part, long long tail_cells, size_t smem_budget);
size_t pcgb_desc_size(int mixed);
int pcgb_max_batch();
cudaError_t launch_pressure_batched(int mixed, int dims, const void* ddesc, int B, int maxlev, int coarse_sweeps,
                                    double reltol, int maxit, int nblk, int threads, size_t smem,
                                    unsigned int* bar, int* err, long long spin_limit, long long* trace,
                                    int trace_cap, int skip, cudaStream_t s);
size_t pcgb_fields_offset(int mixed);
void launch_pressure_reset(unsigned int* bar, int* err, cudaStream_t s);
int pcgb_fits(int mixed, int dims, int threads, size_t smem, int* blocks_per_sm);

// adjoint.cu: reverse pass of the frozen-turbulence sweep (reverse fixed
// point of Christianson type for d(pressure drop)/d(lambda))
struct Adj {
    int nu;              // red-black momentum sweep pairs of the differentiated sweep
    long long nvec;      // length of the flat adjoint state (u components, p, face fluxes)
    double* vpsi;        // flat psi; psu / psp / psf point into it
    double* vxb;         // flat x-bar; xbu / xbp / xbf point into it
    double* vb;          // flat J_x^T (right-hand side of the adjoint)
    double* vbu[3];      // its velocity, pressure and face-flux blocks
    double* vbp;
    double* vbf[3];
    double* fixs[3];     // drag: adjoint of u_ib from the objective itself (explicit J_lambda)
    double* snap;        // [2 nu][3][N] predictor iterates S_0 .. S_{2nu-1} (S_{2nu} = F.us)
    double* As;          // [6][N] neighbour coefficients of the momentum rows (0: no neighbour)
    double* AP;          // [3][N] unrelaxed diagonal per component
    double* aavg;        // [N] component-averaged relaxed diagonal
    double* jw;          // [N] objective weights on p
    double* psu[3];      // adjoint state: velocity, pressure, face flux (input of a pass)
    double* psp;
    double* psf[3];
    double* xbu[3];      // output of a pass
    double* xbp;
    double* xbf[3];
    double* pnb;         // right-hand side of the adjoint pressure solve
    double* ps;          // its solution (kept as the next warm start)
    double* Hb[3];       // adjoints of HbyA, rAU, b0, bm, aP, a_s
    double* rAUb;
    double* b0b[3];
    double* bmb[3];
    double* aPb[3];
    double* asb;         // [6][N]
    double* usb[2][3];   // ping-pong adjoint of the predictor iterates
    double* fixb[3];     // adjoint of the imposed velocity u_ib
    double* Gb;          // [9][N] adjoint of the velocity gradient, layout of F.G
    int* tptr;           // [N+1] interpolation transpose: entries per cell
    int* tent;           // entries: bc index * 16 + stencil * 8 + corner
    double* dlam;        // output dJ/dlambda [N]
};
void launch_adj_coef(const Grid& g, const Params& P, const Fields& F, const Adj& A, cudaStream_t s);
void launch_adj_update(const Grid& g, const Params& P, const Fields& F, const Level& L0, const Adj& A,
                       cudaStream_t s);
void launch_adj_pcg_init(const Grid& g, const Fields& Fa, const Level& L0, const double* rhs, int jacobi,
                         cudaStream_t s);
void launch_adj_pressure(const Grid& g, const Fields& F, const Level& L0, const Adj& A, cudaStream_t s);
void launch_adj_hbya(const Grid& g, const Params& P, const Fields& F, const Adj& A, cudaStream_t s);
void launch_adj_gs(const Grid& g, const Params& P, const Fields& F, const Adj& A, int colour, const double* Sin,
                   const double* Sout, int in_buf, cudaStream_t s);
void launch_adj_b0(const Grid& g, const Params& P, const Fields& F, const Adj& A, int buf, cudaStream_t s);
void launch_adj_transpose(const Grid& g, const Fields& F, const Adj& A, cudaStream_t s);
void launch_adj_gradu(const Grid& g, const Fields& F, const BcList& bl, const Adj& A, cudaStream_t s);
void launch_adj_phi(const Grid& g, const Fields& F, const Adj& A, cudaStream_t s);
void launch_adj_next(const Grid& g, const Fields& F, const Adj& A, int first, cudaStream_t s);
void launch_adj_objective(const Grid& g, const Fields& F, const Adj& A, cudaStream_t s);
void launch_adj_dlambda_mask(const Grid& g, const Fields& F, const Adj& A, cudaStream_t s);
void launch_adj_drag_value(const Grid& g, const Fields& F, const Adj& A, cudaStream_t s);
void launch_adj_drag_seed(const Grid& g, const Fields& F, const Adj& A, cudaStream_t s);
void launch_adj_dlambda(const Grid& g, const Fields& F, const BcList& bl, const double* lam, const Adj& A,
                        cudaStream_t s);
enum { SC_ADJ_DIFF = 48, SC_ADJ_NORM = 49, SC_ADJ_J = 50 };

// krylov.cu: GMRES(m) vector kernels and the Hessenberg bookkeeping
void launch_vsub(long long n, const double* a, const double* b, double* out, cudaStream_t s);
void launch_vsub_add(long long n, const double* a, const double* b, const double* c, double* out, cudaStream_t s);
int mdot_grid(long long n);
void launch_mdot(long long n, const double* w, const double* V, long long ldv, int k, double* partials,
                 unsigned int* counter, double* out, cudaStream_t s);
void launch_maxpy(long long n, double* w, const double* V, long long ldv, int k, const double* c, double sgn,
                  cudaStream_t s);
void launch_vnormalize(long long n, const double* src, double* dst, const double* nrm2, cudaStream_t s);
void launch_gmres_start(int m, const double* nrm2, double* gv, double* st, cudaStream_t s);
void launch_gmres_column(int j, int m, double* H, const double* h1, const double* h2, const double* nrm2, double* cs,
                         double* sn, double* gv, double* st, cudaStream_t s);
void launch_gmres_y(int k, int m, const double* H, const double* gv, double* y, cudaStream_t s);

// turb.cu
void launch_turb_prep(const Grid& g, const Params& P, const Fields& F, cudaStream_t s);
void launch_bc_prod(const Grid& g, const BcList& bl, const Fields& F, cudaStream_t s);
void launch_scal_asm(const Grid& g, const Params& P, const Fields& F, int eq, cudaStream_t s);
void launch_scal_smooth(const Grid& g, const Params& P, const Fields& F, int eq, int colour,
                        cudaStream_t s);
void launch_k_prep(const Grid& g, const Params& P, const Fields& F, cudaStream_t s);
void launch_turb_final(const Grid& g, const Params& P, const Fields& F, cudaStream_t s);
void launch_inv_wall_distance(const Grid& g, const Fields& F, cudaStream_t s);

}  // namespace hf
