// pcgp.cu -- the pressure corrector (a7) as one persistent cooperative
// kernel: PCG with one multigrid V-cycle per iteration (or Jacobi), the
// whole loop inside a single launch.
//
// Operator and preconditioner are those of pressure.cu (same face
// coefficients, same V-cycle: red-black Gauss-Seidel, piecewise-constant
// transfers, coarse coefficients half the covered fine faces); only the
// execution differs: phases separated by a grid barrier instead of kernel
// boundaries.  The launch is cooperative (all blocks resident).  Each wait
// at the grid barrier is bounded: a block whose poll budget runs out sets the
// error word, and every block that finds the error word set at a barrier
// leaves the kernel there (no further phase runs on incomplete data).  The
// host reads the word after the sweep and reports HFDIB_ERR_TIMEOUT.
// Reductions: every block writes its partial; after the barrier every block
// sums all partials in the same order, so all blocks hold the same
// bit-identical value (deterministic, no atomics on floating point).  Levels
// of at most tail_cells cells (an option) run inside block 0.
//
// Mixed precision (pattern "FP32 sweeps inside FP64 refinement"): the CG
// vectors, dot products, scalars and the defect r = rhs - A p stay FP64; the
// V-cycle that preconditions them runs in FP32 on an FP32 copy of the
// operator (level 0 rounded from the FP64 face coefficients, coarse levels
// coarsened in FP32).  The converged pressure solves the FP64 equation.
#include "common.cuh"
#include "kernels.cuh"
#include "pcg_ops.cuh"

namespace hf {

constexpr int PT_THREADS = 1024;

template <typename MT>
struct PcgpArgs {
    Grid g;
    Fields F;
    Level L0d;           // FP64 operator of the CG product (level 0)
    MgLevelsT<MT> M;     // preconditioner hierarchy (level 0 = the grid)
    MT* zp;              // preconditioned residual z (= M.lv[0].x)
    int lf;              // levels 0..lf-1 by the whole grid, lf..nl-1 by block 0
    int smem_tail;       // 1: block 0 keeps the tail levels in shared memory
    int coarse_sweeps;
    int jacobi;
    double reltol;
    int maxit;
    double* part;        // [8][gridDim.x] block partials
    unsigned int* bar;   // barrier arrival counter (zeroed before each launch)
    int* err;            // barrier timeout flag (zeroed before each launch)
    long long spin_limit;  // polls of one barrier wait before giving up
    long long tail_cells;  // largest level block 0 runs alone (shared memory when it fits)
    int cg32;              // FP32 preconditioner only: CG vectors and product in FP32
    float* cd32[2];        // FP32 search directions (cg32)
    float* cq32;           // FP32 A d (cg32)
    long long* trace;      // nullable: block 0 records (phase, %globaltimer) pairs here
    int trace_cap;         // pairs that fit after the count in trace[0]
};

// ---------------------------------------------------------------- barrier
// monotone arrival counter: barrier number m completes when the counter
// reaches m * gridDim.x; polled with acquire loads, bounded
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
    return *(const volatile int*)p;
}

// Phase trace: with A.trace set, thread 0 of block 0 appends (phase tag,
// %globaltimer in ns) after every barrier; trace[0] counts the pairs.
__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}
template <typename AT>
__device__ inline void trace_mark(const AT& A, int tag) {
    if (A.trace && blockIdx.x == 0 && threadIdx.x == 0) {
        long long n = A.trace[0];
        if (n < A.trace_cap) {
            A.trace[1 + 2 * n] = tag;
            A.trace[2 + 2 * n] = global_ns();
            A.trace[0] = n + 1;
        }
    }
}

// Grid barrier.  Thread 0 arrives and polls; a wait that runs out of polls
// sets the error word, and a wait that sees the error word set stops.  Then
// the whole block either continues or, on an error, leaves the kernel
// together (block-uniform, after the block barrier, so no thread is left
// waiting at a later __syncthreads).
template <typename AT>
__device__ inline void grid_sync(const AT& A, int tag) {
    __shared__ int s_abort;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int nb = gridDim.x;
        __threadfence();
        unsigned int old = atomicAdd(A.bar, 1u);
        unsigned int target = (old / nb + 1u) * nb;
        long long spins = 0;
        int abort = 0;
        while ((int)(ld_acquire_u32(A.bar) - target) < 0) {
            if (ld_volatile_i32(A.err)) { abort = 1; break; }
            if (++spins > A.spin_limit) { atomicExch(A.err, 1); abort = 1; break; }
        }
        if (!abort && ld_volatile_i32(A.err)) abort = 1;
        s_abort = abort;
    }
    __syncthreads();
    if (s_abort) asm volatile("exit;");
    trace_mark(A, tag);
}

// block partial of v into slot q; returns nothing (combined after a barrier)
template <typename AT>
__device__ inline void block_partial(const AT& A, int q, double v) {
    __shared__ double sm[PT_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = sm[0];
        for (int w = 1; w < PT_THREADS / 32; ++w) x += sm[w];
        A.part[(long long)q * gridDim.x + blockIdx.x] = x;
    }
}

// sum of slot q over all blocks, same order in every block
template <typename AT>
__device__ inline double grid_total(const AT& A, int q) {
    __shared__ double sm[PT_THREADS / 32];
    __shared__ double res;
    double x = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) x += __ldcg(&A.part[(long long)q * gridDim.x + b]);
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double y = sm[0];
        for (int w = 1; w < PT_THREADS / 32; ++w) y += sm[w];
        res = y;
    }
    __syncthreads();
    return res;
}

// block 0's copy of the level table whose tail levels point into dynamic
// shared memory (set up once per solve by pl_build_tail)
template <typename MT>
__device__ inline MgLevelsT<MT>* tail_levels() {
    __shared__ MgLevelsT<MT> table;
    return &table;
}

extern __shared__ __align__(16) unsigned char pt_dyn_smem[];

// block 0: the tail levels lf..nl-1 built directly in dynamic shared memory
// (level lf coarsened from the grid's level lf-1, each further level from the
// shared one above it); the grid never builds them in global memory
template <typename MT>
__device__ void pl_build_tail(const PcgpArgs<MT>& A) {
    MgLevelsT<MT>* S = tail_levels<MT>();
    const int dims = A.g.dims;
    if (threadIdx.x == 0) {
        *S = A.M;
        MT* p = (MT*)pt_dyn_smem;
        for (int l = A.lf; l < A.M.nl; ++l) {
            LevelT<MT>& L = S->lv[l];
            L.diag = p; p += L.N;
            L.idg = p; p += L.N;
            L.x = p; p += L.N;
            L.b = p; p += L.N;
            L.cf[0] = p; p += (long long)(L.nx + 1) * L.ny * L.nz;
            L.cf[1] = p; p += (long long)L.nx * (L.ny + 1) * L.nz;
            if (dims == 3) { L.cf[2] = p; p += (long long)L.nx * L.ny * (L.nz + 1); }
        }
    }
    __syncthreads();
    for (int l = A.lf; l < A.M.nl; ++l) {
        if (l == A.lf) pl_coarsen(A.M.lv[l - 1], S->lv[l], dims, threadIdx.x, blockDim.x);
        else pl_coarsen(S->lv[l - 1], S->lv[l], dims, threadIdx.x, blockDim.x);
        __syncthreads();
    }
}

// z = B r: the level-0 zero-start red half sweep has been done by the caller;
// the final red half sweep of level 0 accumulates r.z (r in FP64) into slot qdot
template <typename MT>
__device__ void pl_vcycle_rest(const PcgpArgs<MT>& A, int qdot) {
    const MgLevelsT<MT>& M = A.M;
    const int dims = A.g.dims;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long TT = (long long)gridDim.x * blockDim.x;
    const int lf = A.lf;
    pl_smooth(M.lv[0], dims, 1, t0, TT);
    grid_sync(A, PH_VC_SMOOTH0);
    for (int l = 0; l + 1 < lf; ++l) {
        pl_restrict(M.lv[l], M.lv[l + 1], dims, true, t0, TT);
        grid_sync(A, PH_VC_RESTRICT);
        pl_smooth(M.lv[l + 1], dims, 1, t0, TT);
        grid_sync(A, PH_VC_SMOOTH);
    }
    if (lf < M.nl) {
        pl_restrict(M.lv[lf - 1], M.lv[lf], dims, false, t0, TT);
        grid_sync(A, PH_VC_RESTRICT);
        if (blockIdx.x == 0) {
            if (A.smem_tail) {
                // the tail levels live in shared memory: bring b of level lf in,
                // cycle, send x of level lf back for the grid's prolongation
                const MgLevelsT<MT>& S = *tail_levels<MT>();
                for (long long c = threadIdx.x; c < M.lv[lf].N; c += blockDim.x) S.lv[lf].b[c] = M.lv[lf].b[c];
                __syncthreads();
                pl_tail(S, dims, lf, A.coarse_sweeps);
                for (long long c = threadIdx.x; c < M.lv[lf].N; c += blockDim.x) M.lv[lf].x[c] = S.lv[lf].x[c];
                __syncthreads();
            } else {
                pl_tail(M, dims, lf, A.coarse_sweeps);
            }
        }
        grid_sync(A, PH_VC_TAIL);
    }
    for (int l = lf - 1; l >= 0; --l) {
        const LevelT<MT>& L = M.lv[l];
        if (l + 1 < M.nl) pl_prolong_black(L, M.lv[l + 1], dims, t0, TT);
        else pl_smooth(L, dims, 1, t0, TT);
        grid_sync(A, PH_VC_PROLONG);
        if (l > 0) {
            pl_smooth(L, dims, 0, t0, TT);
            grid_sync(A, PH_VC_UPSMOOTH);
        }
    }
    // final red half sweep of level 0 with r.z (the CG residual: FP64, or
    // under cg32 the FP32 one held in level 0's right-hand side)
    const LevelT<MT>& L0 = M.lv[0];
    const double* r = A.F.r;
    const bool r32 = A.cg32 != 0;
    double rz = 0.0;
    const long long NP = pl_npairs(L0);
    for (long long p = t0; p < NP; p += TT) {
        int i0, j, k;
        long long c0;
        pl_pair(L0, p, i0, j, k, c0);
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            if (i0 + o >= L0.nx) break;
            long long c = c0 + o;
            if (((i0 + o + j + k) & 1) == 0)
                L0.x[c] = (L0.b[c] + pl_offsum(L0, dims, L0.x, c, i0 + o, j, k)) * L0.idg[c];
            rz += (r32 ? (double)L0.b[c] : r[c]) * (double)L0.x[c];
        }
    }
    block_partial(A, qdot, rz);
    grid_sync(A, PH_VC_FINAL);
}

// level-0 operator from rAU (FP64, also used by the flux correction), its
// copy in the preconditioner precision, then the coarse levels
template <typename MT>
__device__ void pl_build_operator(const PcgpArgs<MT>& A) {
    const Grid& g = A.g;
    const Level& L = A.L0d;
    const LevelT<MT>& P0 = A.M.lv[0];
    const double* rAU = A.F.rAU;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long TT = (long long)gridDim.x * blockDim.x;
    const bool copy = (void*)P0.diag != (void*)L.diag;
    for (long long c = t0; c < g.N; c += TT) {
        int i, j, k;
        cell_ijk(g, c, i, j, k);
        const int idx[3] = {i, j, k};
        double diag = 0.0;
        #pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d >= g.dims) break;
            long long fl = pl_face(L, d, i, j, k);
            long long fs = pl_fstride(L, d);
            double clo, chi;
            if (idx[d] > 0) clo = 0.5 * (rAU[c] + rAU[c - g.stride[d]]) * g.SoD[d];
            else clo = p_fixed(g, 2 * d) ? rAU[c] * g.SoHD[d] : 0.0;
            if (idx[d] < g.n[d] - 1) chi = 0.5 * (rAU[c] + rAU[c + g.stride[d]]) * g.SoD[d];
            else chi = p_fixed(g, 2 * d + 1) ? rAU[c] * g.SoHD[d] : 0.0;
            L.cf[d][fl] = clo;
            if (copy) P0.cf[d][fl] = (MT)clo;
            if (idx[d] == g.n[d] - 1) {
                L.cf[d][fl + fs] = chi;
                if (copy) P0.cf[d][fl + fs] = (MT)chi;
            }
            diag += clo + chi;
        }
        double idg = diag > 0.0 ? 1.0 / diag : 0.0;
        L.diag[c] = diag;
        L.idg[c] = idg;
        if (copy) { P0.diag[c] = (MT)diag; P0.idg[c] = (MT)idg; }
    }
    grid_sync(A, PH_BUILD0);
    // the shared-memory tail levels are built by block 0 (pl_build_tail)
    const int lend = (A.smem_tail && A.lf < A.M.nl) ? A.lf : A.M.nl;
    for (int l = 1; l < lend; ++l) {
        pl_coarsen(A.M.lv[l - 1], A.M.lv[l], g.dims, t0, TT);
        grid_sync(A, PH_COARSEN);
    }
}

// ---------------------------------------------------------------- the solver
enum { Q_RZ = 0, Q_RR = 1, Q_BB = 2, Q_R1 = 3, Q_R2 = 4, Q_R3 = 5, Q_DQ = 6 };

template <typename MT>
__global__ void __launch_bounds__(PT_THREADS) k_pressure_persistent(PcgpArgs<MT> A) {
    const Grid& g = A.g;
    const Fields& F = A.F;
    const Level& L0 = A.L0d;             // FP64 operator
    const LevelT<MT>& P0 = A.M.lv[0];    // preconditioner level 0 (z, b)
    MT* z = A.zp;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long T = (long long)gridDim.x * blockDim.x;
    const bool jac = A.jacobi != 0;
    trace_mark(A, PH_START);
    // ---- operator hierarchy for this sweep's rAU (tail levels to shared memory)
    pl_build_operator(A);
    // ---- block 0 builds the shared-memory tail while the other blocks form
    // r = rhs - A p, the residual sums and z0 (Jacobi, or the level-0 red start)
    const bool tail_b0 = A.smem_tail && A.lf < A.M.nl;
    if (tail_b0 && blockIdx.x == 0) pl_build_tail(A);
    long long rc0 = t0, RT = T;
    if (tail_b0 && gridDim.x > 1) {
        RT = T - blockDim.x;
        rc0 = blockIdx.x == 0 ? g.N : t0 - blockDim.x;
    }
    double s_rz = 0, s_rr = 0, s_bb = 0, s1 = 0, s2 = 0, s3 = 0;
    double pbar = F.scal[SC_SUM_P] * g.iN;
    for (long long c = rc0; c < g.N; c += RT) {
        int i, j, k;
        cell_ijk(g, c, i, j, k);
        uint16_t f = F.flags[c];
        const int idx[3] = {i, j, k};
        double div = 0.0, bout = 0.0, A1 = 0.0;
        #pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d >= g.dims) break;
            long long fl = face_lo(g, d, i, j, k);
            long long fs = face_stride(g, d);
            div += F.phiH[d][fl + fs] - F.phiH[d][fl];
            if (idx[d] == 0 && p_fixed(g, 2 * d)) { bout += L0.cf[d][fl] * g.p_out; A1 += L0.cf[d][fl]; }
            if (idx[d] == g.n[d] - 1 && p_fixed(g, 2 * d + 1)) {
                bout += L0.cf[d][fl + fs] * g.p_out;
                A1 += L0.cf[d][fl + fs];
            }
        }
        double rhs = -masked_div(g, F.lam, f, c, div) + bout;
        double Ap = L0.diag[c] * F.p[c] - pl_offsum(L0, g.dims, F.p, c, i, j, k);
        double r = rhs - Ap;
        F.r[c] = r;
        F.d[0][c] = 0.0;
        if constexpr (sizeof(MT) == 4) {
            if (A.cg32) A.cd32[0][c] = 0.0f;
        }
        F.pn[c] = F.p[c];
        if (jac) {
            double zz = r * L0.idg[c];
            z[c] = (MT)zz;
            s_rz += r * zz;
        } else {
            MT rb = (MT)r;
            if ((void*)P0.b != (void*)F.r) P0.b[c] = rb;
            if (((i + j + k) & 1) == 0) z[c] = rb * P0.idg[c];
        }
        s_rr += r * r;
        s_bb += rhs * rhs;
        s1 += fabs(r);
        s2 += fabs(Ap - A1 * pbar);
        s3 += fabs(rhs - A1 * pbar);
    }
    block_partial(A, Q_RZ, s_rz);
    block_partial(A, Q_RR, s_rr);
    block_partial(A, Q_BB, s_bb);
    block_partial(A, Q_R1, s1);
    block_partial(A, Q_R2, s2);
    block_partial(A, Q_R3, s3);
    grid_sync(A, PH_R0);
    double rr0 = grid_total(A, Q_RR);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        F.scal[SC_PCG_INIT + 1] = rr0;
        F.scal[SC_PCG_INIT + 3] = 0.0;
    }
    double r1 = grid_total(A, Q_R1), r2 = grid_total(A, Q_R2), r3 = grid_total(A, Q_R3);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        F.scal[SC_PCG_INIT + 3] = r1;
        F.scal[SC_PCG_INIT + 4] = r2;
        F.scal[SC_PCG_INIT + 5] = r3;
    }
    double tol2 = A.reltol * A.reltol * rr0;
    int it = 0;
    if (rr0 > 0.0 && isfinite(rr0) && A.maxit > 0) {
        double rz;
        if (jac) {
            rz = grid_total(A, Q_RZ);
        } else {
            pl_vcycle_rest(A, Q_RZ);
            rz = grid_total(A, Q_RZ);
        }
        double rz_prev = 1.0;
        while (it < A.maxit) {
            double beta = it == 0 ? 0.0 : rz / rz_prev;
            if constexpr (sizeof(MT) == 4) {
                if (A.cg32) {
                    // the correction solve in FP32 (P1): the product with the FP32
                    // copy of the operator, FP32 vectors, dots accumulated in FP64;
                    // the start defect (r0 above) and p stay FP64
                    const float* dold = A.cd32[it & 1];
                    float* dnew = A.cd32[(it + 1) & 1];
                    const float fb = (float)beta;
                    double s_dq = 0.0;
                    for (long long c = t0; c < g.N; c += T) {
                        int i, j, k;
                        cell_ijk(g, c, i, j, k);
                        const int idx[3] = {i, j, k};
                        float zc = (float)z[c];
                        float acc = (float)P0.diag[c] * zc;
                        #pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            if (d >= g.dims) break;
                            long long fl = face_lo(g, d, i, j, k);
                            if (idx[d] > 0) acc -= (float)P0.cf[d][fl] * (float)z[c - g.stride[d]];
                            if (idx[d] < g.n[d] - 1) acc -= (float)P0.cf[d][fl + face_stride(g, d)] * (float)z[c + g.stride[d]];
                        }
                        float dP = zc + fb * dold[c];
                        float qv = it == 0 ? acc : acc + fb * A.cq32[c];
                        dnew[c] = dP;
                        A.cq32[c] = qv;
                        s_dq += (double)dP * (double)qv;
                    }
                    block_partial(A, Q_DQ, s_dq);
                    grid_sync(A, PH_CG_PRODUCT);
                    double dq = grid_total(A, Q_DQ);
                    double alpha = dq != 0.0 ? rz / dq : 0.0;
                    const float fa = (float)alpha;
                    double s_r2 = 0.0;
                    for (long long c = t0; c < g.N; c += T) {
                        F.pn[c] += alpha * (double)dnew[c];
                        float r = (float)P0.b[c] - fa * A.cq32[c];
                        P0.b[c] = (MT)r;
                        s_r2 += (double)r * (double)r;
                        int i, j, k;
                        cell_ijk(g, c, i, j, k);
                        if (((i + j + k) & 1) == 0) z[c] = (MT)(r * (float)P0.idg[c]);
                    }
                    block_partial(A, Q_RR, s_r2);
                    grid_sync(A, PH_CG_UPDATE);
                    double rr = grid_total(A, Q_RR);
                    rz_prev = rz;
                    pl_vcycle_rest(A, Q_RZ);
                    rz = grid_total(A, Q_RZ);
                    ++it;
                    if (!(rr > tol2)) break;
                    continue;
                }
            }
            const double* dold = F.d[it & 1];
            double* dnew = F.d[(it + 1) & 1];
            // d = z + beta d_old; q = A d = A z + beta q_old (linearity: the
            // neighbours' d need not be rebuilt); d.q
            double s_dq = 0.0;
            for (long long c = t0; c < g.N; c += T) {
                int i, j, k;
                cell_ijk(g, c, i, j, k);
                const int idx[3] = {i, j, k};
                double zc = (double)z[c];
                double acc = L0.diag[c] * zc;
                #pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (d >= g.dims) break;
                    long long fl = face_lo(g, d, i, j, k);
                    if (idx[d] > 0) acc -= L0.cf[d][fl] * (double)z[c - g.stride[d]];
                    if (idx[d] < g.n[d] - 1) acc -= L0.cf[d][fl + face_stride(g, d)] * (double)z[c + g.stride[d]];
                }
                double dP = zc + beta * dold[c];
                double qv = it == 0 ? acc : acc + beta * F.q[c];
                dnew[c] = dP;
                F.q[c] = qv;
                s_dq += dP * qv;
            }
            block_partial(A, Q_DQ, s_dq);
            grid_sync(A, PH_CG_PRODUCT);
            double dq = grid_total(A, Q_DQ);
            double alpha = dq != 0.0 ? rz / dq : 0.0;
            // p += alpha d; r -= alpha q; r.r; z start
            double s_r2 = 0.0, s_z = 0.0;
            for (long long c = t0; c < g.N; c += T) {
                F.pn[c] += alpha * dnew[c];
                double r = F.r[c] - alpha * F.q[c];
                F.r[c] = r;
                s_r2 += r * r;
                if (jac) {
                    double zz = r * L0.idg[c];
                    z[c] = (MT)zz;
                    s_z += r * zz;
                } else {
                    MT rb = (MT)r;
                    if ((void*)P0.b != (void*)F.r) P0.b[c] = rb;
                    int i, j, k;
                    cell_ijk(g, c, i, j, k);
                    if (((i + j + k) & 1) == 0) z[c] = rb * P0.idg[c];
                }
            }
            block_partial(A, Q_RR, s_r2);
            if (jac) block_partial(A, Q_RZ, s_z);
            grid_sync(A, PH_CG_UPDATE);
            double rr = grid_total(A, Q_RR);
            rz_prev = rz;
            if (jac) {
                rz = grid_total(A, Q_RZ);
            } else {
                pl_vcycle_rest(A, Q_RZ);
                rz = grid_total(A, Q_RZ);
            }
            ++it;
            if (!(rr > tol2)) break;
            // no barrier here: every partial slot read above is written again
            // only after the next iteration's product and update barriers
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        F.scal[SC_PCG_ITERS] = (double)it;
        F.scal[SC_PCG_DONE] = 1.0;
    }
    trace_mark(A, PH_END);
}

// ---------------------------------------------------------------- launcher
int pcgp_blocks(int* out) {
    int dev = 0, sms = 0, occ = 0, occ32 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pressure_persistent<double>, PT_THREADS, 0) !=
        cudaSuccess)
        return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ32, k_pressure_persistent<float>, PT_THREADS, 0) !=
        cudaSuccess)
        return -1;
    if (occ < 1 || occ32 < 1) return -1;
    *out = sms;   // one block per SM: fewer arrivals per grid barrier
    return 0;
}

// shared-memory bytes of the tail levels l0..nl-1
template <typename MT>
static size_t tail_bytes(const MgLevelsT<MT>& M, int dims, int l0) {
    size_t n = 0;
    for (int l = l0; l < M.nl; ++l) {
        const LevelT<MT>& L = M.lv[l];
        n += 4 * (size_t)L.N + (size_t)(L.nx + 1) * L.ny * L.nz + (size_t)L.nx * (L.ny + 1) * L.nz;
        if (dims == 3) n += (size_t)L.nx * L.ny * (L.nz + 1);
    }
    return n * sizeof(MT);
}

constexpr size_t PT_SMEM_BUDGET = 160 * 1024;

template <typename MT>
static cudaError_t launch_pp(PcgpArgs<MT>& A, int nblk, cudaStream_t s) {
    // tail = the coarsest levels whose operator fits the shared-memory
    // budget (at most PT_SMEM_TAIL_CELLS cells on its finest level)
    A.lf = A.M.nl;
    A.smem_tail = 0;
    size_t bytes = 0;
    for (int l = 1; l < A.M.nl; ++l) {
        if (A.M.lv[l].N > A.tail_cells) continue;
        size_t b = tail_bytes(A.M, A.g.dims, l);
        if (b <= PT_SMEM_BUDGET) { A.lf = l; A.smem_tail = 1; bytes = b; break; }
    }
    if (!A.smem_tail) {
        for (int l = 1; l < A.M.nl; ++l)
            if (A.M.lv[l].N <= A.tail_cells) { A.lf = l; break; }
    }
    if (bytes > 0) {
        cudaError_t e = cudaFuncSetAttribute(k_pressure_persistent<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)bytes);
        if (e != cudaSuccess) return e;
    }
    void* args[] = {&A};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblk);
    cfg.blockDim = dim3(PT_THREADS);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (const void*)k_pressure_persistent<MT>, args);
}

cudaError_t launch_pressure_persistent(const Grid& g, const Fields& F, const MgLevels& M, int jacobi,
                                       int coarse_sweeps, double reltol, int maxit, int nblk, double* part,
                                       unsigned int* bar, int* err, long long spin_limit, long long tail_cells,
                                       long long* trace, int trace_cap, cudaStream_t s) {
    PcgpArgs<double> A;
    A.g = g; A.F = F; A.L0d = M.lv[0]; A.M = M; A.zp = M.lv[0].x;
    A.coarse_sweeps = coarse_sweeps; A.jacobi = jacobi; A.reltol = reltol; A.maxit = maxit;
    A.part = part; A.bar = bar; A.err = err; A.spin_limit = spin_limit; A.tail_cells = tail_cells;
    A.cg32 = 0; A.cd32[0] = A.cd32[1] = nullptr; A.cq32 = nullptr;
    A.trace = trace; A.trace_cap = trace_cap;
    return launch_pp(A, nblk, s);
}

cudaError_t launch_pressure_persistent32(const Grid& g, const Fields& F, const MgLevels& M, const MgLevels32& M32,
                                         int coarse_sweeps, double reltol, int maxit, int nblk, double* part,
                                         unsigned int* bar, int* err, long long spin_limit, long long tail_cells,
                                         int cg32, long long* trace, int trace_cap, cudaStream_t s) {
    PcgpArgs<float> A;
    A.g = g; A.F = F; A.L0d = M.lv[0]; A.M = M32; A.zp = M32.lv[0].x;
    A.coarse_sweeps = coarse_sweeps; A.jacobi = 0; A.reltol = reltol; A.maxit = maxit;
    A.part = part; A.bar = bar; A.err = err; A.spin_limit = spin_limit; A.tail_cells = tail_cells;
    A.cg32 = cg32; A.cd32[0] = F.pd32[0]; A.cd32[1] = F.pd32[1]; A.cq32 = F.pq32;
    A.trace = trace; A.trace_cap = trace_cap;
    return launch_pp(A, nblk, s);
}

}  // namespace hf
