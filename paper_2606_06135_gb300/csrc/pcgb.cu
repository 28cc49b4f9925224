// pcgb.cu -- the pressure corrector (a7) of a batch of independent problems
// (one lambda field each; grid sizes may differ) in ONE persistent
// cooperative launch.
//
// Every problem runs the same algorithm as pcgp.cu (PCG, one multigrid
// V-cycle per iteration, FP64 CG with an FP64 or FP32 preconditioner), and
// the problems advance in lockstep: each phase loops over the problems
// before the grid barrier, so the barrier cost is shared by the whole batch
// and small problems fill the GPU together.  Each problem keeps its own
// reductions, iteration count and convergence test (a converged problem
// skips its work); the coarse tail of problem b runs on block b (in parallel
// across problems), in that block's shared memory when it fits.
#include "common.cuh"
#include "kernels.cuh"
#include "pcg_ops.cuh"

namespace hf {

constexpr int PB_MAXB = 64;

template <typename MT>
struct PcgbDesign {
    Grid g;
    Fields F;
    Level L0d;          // FP64 operator (level 0)
    MgLevelsT<MT> M;    // preconditioner hierarchy
    MT* zp;             // z (= M.lv[0].x)
    int lf;             // levels 0..lf-1 by the grid, lf..nl-1 by one block
    int smem_tail;      // the tail fits the tail block's shared memory
    double* part;       // [8][gridDim.x] partial sums of this problem
};

template <typename MT>
struct PcgbArgs {
    const PcgbDesign<MT>* D;   // device array of B descriptors
    int B;
    int maxlev;
    int coarse_sweeps;
    double reltol;
    int maxit;
    unsigned int* bar;
    int* err;              // zeroed before each launch
    long long spin_limit;  // polls of one barrier wait before giving up
};

// ---------------------------------------------------------------- sync and sums
__device__ __forceinline__ unsigned int pb_ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// grid barrier: monotone arrival counter, bounded acquire polling.  A wait
// that runs out of polls sets the error word; a wait that finds it set
// stops, and the whole block then leaves the kernel together (the host
// reports HFDIB_ERR_TIMEOUT).
__device__ inline void pb_sync(unsigned int* bar, int* err, long long spin_limit) {
    __shared__ int s_abort;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int nb = gridDim.x;
        __threadfence();
        unsigned int old = atomicAdd(bar, 1u);
        unsigned int target = (old / nb + 1u) * nb;
        long long spins = 0;
        int abort = 0;
        while ((int)(pb_ld_acquire(bar) - target) < 0) {
            if (*(const volatile int*)err) { abort = 1; break; }
            if (++spins > spin_limit) { atomicExch(err, 1); abort = 1; break; }
        }
        if (!abort && *(const volatile int*)err) abort = 1;
        s_abort = abort;
    }
    __syncthreads();
    if (s_abort) asm volatile("exit;");
}

__device__ inline void pb_partial(double* part, int q, double v) {
    __shared__ double sm[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += sm[w];
        part[(long long)q * gridDim.x + blockIdx.x] = x;
    }
}

// same value in every block (fixed summation order)
__device__ inline double pb_total(const double* part, int q) {
    __shared__ double sm[32];
    __shared__ double res;
    double x = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) x += __ldcg(&part[(long long)q * gridDim.x + b]);
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double y = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) y += sm[w];
        res = y;
    }
    __syncthreads();
    return res;
}

enum { QB_RZ = 0, QB_RR = 1, QB_R1 = 2, QB_R2 = 3, QB_R3 = 4, QB_DQ = 5 };

// per-problem loop state, identical in every block
struct PbState {
    double rz[PB_MAXB], rzp[PB_MAXB], tol2[PB_MAXB], dq[PB_MAXB], rr[PB_MAXB];
    int it[PB_MAXB], done[PB_MAXB];
};

extern __shared__ __align__(16) unsigned char pb_dyn_smem[];

// ---------------------------------------------------------------- phases
template <typename MT>
__device__ void pb_build(const PcgbArgs<MT>& A, long long t0, long long TT) {
    for (int b = 0; b < A.B; ++b) {
        const PcgbDesign<MT>& D = A.D[b];
        const Grid& g = D.g;
        const Level& L = D.L0d;
        const LevelT<MT>& P0 = D.M.lv[0];
        const double* rAU = D.F.rAU;
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
    }
    pb_sync(A.bar, A.err, A.spin_limit);
    for (int l = 1; l < A.maxlev; ++l) {
        for (int b = 0; b < A.B; ++b) {
            const PcgbDesign<MT>& D = A.D[b];
            if (l < D.M.nl) pl_coarsen(D.M.lv[l - 1], D.M.lv[l], D.g.dims, t0, TT);
        }
        pb_sync(A.bar, A.err, A.spin_limit);
    }
}

// this block's tail table (its problem's coarse levels in shared memory)
template <typename MT>
__device__ inline MgLevelsT<MT>* pb_table() {
    __shared__ MgLevelsT<MT> table;
    return &table;
}

template <typename MT>
__device__ void pb_load_tail(const PcgbDesign<MT>& D) {
    MgLevelsT<MT>* S = pb_table<MT>();
    const int dims = D.g.dims;
    if (threadIdx.x == 0) {
        *S = D.M;
        MT* p = (MT*)pb_dyn_smem;
        for (int l = D.lf; l < D.M.nl; ++l) {
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
    for (int l = D.lf; l < D.M.nl; ++l) {
        const LevelT<MT>& G = D.M.lv[l];
        const LevelT<MT>& L = S->lv[l];
        for (long long c = threadIdx.x; c < G.N; c += blockDim.x) { L.diag[c] = G.diag[c]; L.idg[c] = G.idg[c]; }
        long long nf[3] = {(long long)(G.nx + 1) * G.ny * G.nz, (long long)G.nx * (G.ny + 1) * G.nz,
                           (long long)G.nx * G.ny * (G.nz + 1)};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d >= dims) break;
            for (long long f = threadIdx.x; f < nf[d]; f += blockDim.x) L.cf[d][f] = G.cf[d][f];
        }
    }
    __syncthreads();
}

// one V-cycle for every active problem (the level-0 red start is done)
template <typename MT>
__device__ void pb_vcycle(const PcgbArgs<MT>& A, const PbState& S, long long t0, long long TT) {
    const int B = A.B;
    for (int b = 0; b < B; ++b)
        if (!S.done[b]) pl_smooth(A.D[b].M.lv[0], A.D[b].g.dims, 1, t0, TT);
    pb_sync(A.bar, A.err, A.spin_limit);
    for (int l = 0; l + 1 < A.maxlev; ++l) {
        bool any = false;
        for (int b = 0; b < B; ++b) {
            const PcgbDesign<MT>& D = A.D[b];
            if (S.done[b]) continue;
            if (l + 1 < D.lf) { pl_restrict(D.M.lv[l], D.M.lv[l + 1], D.g.dims, true, t0, TT); any = true; }
            else if (l + 1 == D.lf && D.lf < D.M.nl) { pl_restrict(D.M.lv[l], D.M.lv[l + 1], D.g.dims, false, t0, TT); any = true; }
        }
        if (!any) break;
        pb_sync(A.bar, A.err, A.spin_limit);
        for (int b = 0; b < B; ++b) {
            const PcgbDesign<MT>& D = A.D[b];
            if (!S.done[b] && l + 1 < D.lf) pl_smooth(D.M.lv[l + 1], D.g.dims, 1, t0, TT);
        }
        pb_sync(A.bar, A.err, A.spin_limit);
    }
    // coarse tails, problem b on block b % gridDim.x
    for (int b = 0; b < B; ++b) {
        const PcgbDesign<MT>& D = A.D[b];
        if (S.done[b] || D.lf >= D.M.nl || (int)(b % gridDim.x) != (int)blockIdx.x) continue;
        if (D.smem_tail && b < (int)gridDim.x) {
            const MgLevelsT<MT>& T = *pb_table<MT>();
            for (long long c = threadIdx.x; c < D.M.lv[D.lf].N; c += blockDim.x) T.lv[D.lf].b[c] = D.M.lv[D.lf].b[c];
            __syncthreads();
            pl_tail(T, D.g.dims, D.lf, A.coarse_sweeps);
            for (long long c = threadIdx.x; c < D.M.lv[D.lf].N; c += blockDim.x) D.M.lv[D.lf].x[c] = T.lv[D.lf].x[c];
            __syncthreads();
        } else {
            pl_tail(D.M, D.g.dims, D.lf, A.coarse_sweeps);
        }
    }
    pb_sync(A.bar, A.err, A.spin_limit);
    for (int l = A.maxlev - 1; l >= 0; --l) {
        bool any = false;
        for (int b = 0; b < B; ++b) {
            const PcgbDesign<MT>& D = A.D[b];
            if (S.done[b] || l >= D.lf) continue;
            any = true;
            if (l + 1 < D.M.nl) pl_prolong_black(D.M.lv[l], D.M.lv[l + 1], D.g.dims, t0, TT);
            else pl_smooth(D.M.lv[l], D.g.dims, 1, t0, TT);
        }
        if (!any) continue;
        pb_sync(A.bar, A.err, A.spin_limit);
        if (l > 0) {
            for (int b = 0; b < B; ++b) {
                const PcgbDesign<MT>& D = A.D[b];
                if (!S.done[b] && l < D.lf) pl_smooth(D.M.lv[l], D.g.dims, 0, t0, TT);
            }
            pb_sync(A.bar, A.err, A.spin_limit);
        }
    }
    // last red half sweep of level 0 with r.z
    for (int b = 0; b < B; ++b) {
        if (S.done[b]) continue;
        const PcgbDesign<MT>& D = A.D[b];
        const LevelT<MT>& L0 = D.M.lv[0];
        const double* r = D.F.r;
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
                    L0.x[c] = (L0.b[c] + pl_offsum(L0, D.g.dims, L0.x, c, i0 + o, j, k)) * L0.idg[c];
                rz += r[c] * (double)L0.x[c];
            }
        }
        pb_partial(D.part, QB_RZ, rz);
    }
    pb_sync(A.bar, A.err, A.spin_limit);
}

template <typename MT>
__global__ void __launch_bounds__(1024) k_pressure_batched(PcgbArgs<MT> A) {
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long TT = (long long)gridDim.x * blockDim.x;
    const int B = A.B;
    __shared__ PbState S;
    // ---- operators of all problems, this block's tail to shared memory
    pb_build(A, t0, TT);
    if ((int)blockIdx.x < B) {
        const PcgbDesign<MT>& D = A.D[blockIdx.x];
        if (D.smem_tail && D.lf < D.M.nl) pb_load_tail(D);
    }
    // ---- r = rhs - A p, residual sums, red start of z
    for (int b = 0; b < B; ++b) {
        const PcgbDesign<MT>& D = A.D[b];
        const Grid& g = D.g;
        const Fields& F = D.F;
        const Level& L0 = D.L0d;
        const LevelT<MT>& P0 = D.M.lv[0];
        MT* z = D.zp;
        double s_rr = 0, s1 = 0, s2 = 0, s3 = 0;
        double pbar = F.scal[SC_SUM_P] * g.iN;
        for (long long c = t0; c < g.N; c += TT) {
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
            F.pn[c] = F.p[c];
            MT rb = (MT)r;
            if ((void*)P0.b != (void*)F.r) P0.b[c] = rb;
            if (((i + j + k) & 1) == 0) z[c] = rb * P0.idg[c];
            s_rr += r * r;
            s1 += fabs(r);
            s2 += fabs(Ap - A1 * pbar);
            s3 += fabs(rhs - A1 * pbar);
        }
        pb_partial(D.part, QB_RR, s_rr);
        pb_partial(D.part, QB_R1, s1);
        pb_partial(D.part, QB_R2, s2);
        pb_partial(D.part, QB_R3, s3);
    }
    pb_sync(A.bar, A.err, A.spin_limit);
    for (int b = 0; b < B; ++b) {
        const PcgbDesign<MT>& D = A.D[b];
        double rr0 = pb_total(D.part, QB_RR);
        double r1 = pb_total(D.part, QB_R1), r2 = pb_total(D.part, QB_R2), r3 = pb_total(D.part, QB_R3);
        if (threadIdx.x == 0) {
            S.tol2[b] = A.reltol * A.reltol * rr0;
            S.done[b] = (rr0 > 0.0 && isfinite(rr0) && A.maxit > 0) ? 0 : 1;
            S.it[b] = 0;
            S.rzp[b] = 1.0;
            if (blockIdx.x == 0) {
                D.F.scal[SC_PCG_INIT + 1] = rr0;
                D.F.scal[SC_PCG_INIT + 3] = r1;
                D.F.scal[SC_PCG_INIT + 4] = r2;
                D.F.scal[SC_PCG_INIT + 5] = r3;
            }
        }
    }
    __syncthreads();
    pb_vcycle(A, S, t0, TT);
    for (int b = 0; b < B; ++b) {
        double rz = pb_total(A.D[b].part, QB_RZ);
        if (threadIdx.x == 0) S.rz[b] = rz;
    }
    __syncthreads();
    for (int iter = 0; iter < A.maxit; ++iter) {
        bool all = true;
        for (int b = 0; b < B; ++b) all = all && S.done[b];
        if (all) break;
        // d = z + beta d_old; q = A d = A z + beta q_old (linearity: the
        // neighbours' d need not be rebuilt); d.q
        for (int b = 0; b < B; ++b) {
            if (S.done[b]) continue;
            const PcgbDesign<MT>& D = A.D[b];
            const Grid& g = D.g;
            const Fields& F = D.F;
            const Level& L0 = D.L0d;
            const MT* z = D.zp;
            int it = S.it[b];
            double beta = it == 0 ? 0.0 : S.rz[b] / S.rzp[b];
            const double* dold = F.d[it & 1];
            double* dnew = F.d[(it + 1) & 1];
            double s_dq = 0.0;
            for (long long c = t0; c < g.N; c += TT) {
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
            pb_partial(D.part, QB_DQ, s_dq);
        }
        pb_sync(A.bar, A.err, A.spin_limit);
        for (int b = 0; b < B; ++b) {
            if (S.done[b]) continue;
            double dq = pb_total(A.D[b].part, QB_DQ);
            if (threadIdx.x == 0) S.dq[b] = dq;
        }
        __syncthreads();
        // p += alpha d; r -= alpha q; r.r; red start of z
        for (int b = 0; b < B; ++b) {
            if (S.done[b]) continue;
            const PcgbDesign<MT>& D = A.D[b];
            const Grid& g = D.g;
            const Fields& F = D.F;
            const LevelT<MT>& P0 = D.M.lv[0];
            MT* z = D.zp;
            double alpha = S.dq[b] != 0.0 ? S.rz[b] / S.dq[b] : 0.0;
            const double* dn = F.d[(S.it[b] + 1) & 1];
            double s_r2 = 0.0;
            for (long long c = t0; c < g.N; c += TT) {
                F.pn[c] += alpha * dn[c];
                double r = F.r[c] - alpha * F.q[c];
                F.r[c] = r;
                s_r2 += r * r;
                MT rb = (MT)r;
                if ((void*)P0.b != (void*)F.r) P0.b[c] = rb;
                int i, j, k;
                cell_ijk(g, c, i, j, k);
                if (((i + j + k) & 1) == 0) z[c] = rb * P0.idg[c];
            }
            pb_partial(D.part, QB_RR, s_r2);
        }
        pb_sync(A.bar, A.err, A.spin_limit);
        for (int b = 0; b < B; ++b) {
            if (S.done[b]) continue;
            double rr = pb_total(A.D[b].part, QB_RR);
            if (threadIdx.x == 0) S.rr[b] = rr;
        }
        __syncthreads();
        pb_vcycle(A, S, t0, TT);
        for (int b = 0; b < B; ++b) {
            if (S.done[b]) continue;
            double rz = pb_total(A.D[b].part, QB_RZ);
            if (threadIdx.x == 0) {
                S.rzp[b] = S.rz[b];
                S.rz[b] = rz;
                S.it[b] += 1;
                if (!(S.rr[b] > S.tol2[b]) || S.it[b] >= A.maxit) S.done[b] = 1;
            }
        }
        __syncthreads();
        // no grid barrier here: every partial slot read above is written again
        // only after the next iteration's product and update barriers
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int b = 0; b < B; ++b) {
            const Fields& F = A.D[b].F;
            F.scal[SC_PCG_ITERS] = (double)S.it[b];
            F.scal[SC_PCG_DONE] = 1.0;
        }
    }
}

// ---------------------------------------------------------------- host side
template <typename MT>
static size_t pb_tail_bytes(const MgLevelsT<MT>& M, int dims, int l0) {
    size_t n = 0;
    for (int l = l0; l < M.nl; ++l) {
        const LevelT<MT>& L = M.lv[l];
        n += 4 * (size_t)L.N + (size_t)(L.nx + 1) * L.ny * L.nz + (size_t)L.nx * (L.ny + 1) * L.nz;
        if (dims == 3) n += (size_t)L.nx * L.ny * (L.nz + 1);
    }
    return n * sizeof(MT);
}

// Fill the descriptor (host copy) of one problem; returns its tail bytes.
template <typename MT>
static size_t pb_describe(PcgbDesign<MT>& D, const Grid& g, const Fields& F, const MgLevels& M64,
                          const MgLevelsT<MT>& M, double* part, long long tail_cells, size_t smem_budget) {
    D.g = g;
    D.F = F;
    D.L0d = M64.lv[0];
    D.M = M;
    D.zp = M.lv[0].x;
    D.part = part;
    D.lf = M.nl;
    D.smem_tail = 0;
    size_t bytes = 0;
    for (int l = 1; l < M.nl; ++l) {
        if (M.lv[l].N > tail_cells) continue;
        D.lf = l;
        bytes = pb_tail_bytes(M, g.dims, l);
        D.smem_tail = bytes <= smem_budget ? 1 : 0;
        if (!D.smem_tail) bytes = 0;
        break;
    }
    return bytes;
}

size_t pcgb_describe64(void* dst, const Grid& g, const Fields& F, const MgLevels& M, double* part,
                       long long tail_cells, size_t smem_budget) {
    return pb_describe(*(PcgbDesign<double>*)dst, g, F, M, M, part, tail_cells, smem_budget);
}
size_t pcgb_describe32(void* dst, const Grid& g, const Fields& F, const MgLevels& M, const MgLevels32& M32,
                       double* part, long long tail_cells, size_t smem_budget) {
    return pb_describe(*(PcgbDesign<float>*)dst, g, F, M, M32, part, tail_cells, smem_budget);
}
size_t pcgb_desc_size(int mixed) { return mixed ? sizeof(PcgbDesign<float>) : sizeof(PcgbDesign<double>); }
int pcgb_max_batch() { return PB_MAXB; }

cudaError_t launch_pressure_batched(int mixed, const void* ddesc, int B, int maxlev, int coarse_sweeps,
                                    double reltol, int maxit, int nblk, int threads, size_t smem,
                                    unsigned int* bar, int* err, long long spin_limit, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblk);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (mixed) {
        PcgbArgs<float> A{(const PcgbDesign<float>*)ddesc, B, maxlev, coarse_sweeps, reltol, maxit, bar, err,
                          spin_limit};
        cudaError_t e = cudaFuncSetAttribute(k_pressure_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        void* args[] = {&A};
        return cudaLaunchKernelExC(&cfg, (const void*)k_pressure_batched<float>, args);
    }
    PcgbArgs<double> A{(const PcgbDesign<double>*)ddesc, B, maxlev, coarse_sweeps, reltol, maxit, bar, err,
                       spin_limit};
    cudaError_t e = cudaFuncSetAttribute(k_pressure_batched<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    void* args[] = {&A};
    return cudaLaunchKernelExC(&cfg, (const void*)k_pressure_batched<double>, args);
}

int pcgb_fits(int mixed, int threads, size_t smem, int* blocks_per_sm) {
    int occ = 0;
    cudaError_t e = mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pressure_batched<float>, threads, smem)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pressure_batched<double>, threads, smem);
    if (e != cudaSuccess) return -1;
    *blocks_per_sm = occ;
    return 0;
}

}  // namespace hf
