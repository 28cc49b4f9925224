// pcgb.cu -- the pressure corrector (a7) as ONE persistent cooperative
// launch for a batch of B >= 1 independent problems (one lambda field each;
// grid sizes may differ, all problems of a batch are 2D or all 3D).  A
// single problem is a batch of one, so a problem gives the same bits alone
// and inside a batch.
//
// Per problem: conjugate gradients on the pressure equation (Eq. hfdibrans_2
// with the face coefficients rAU_f S/Delta, outlet faces Dirichlet),
// preconditioned by one geometric-multigrid V-cycle: red-black Gauss-Seidel,
// piecewise-constant transfers (restriction = the transpose), coarse
// coefficients half the covered fine faces.  Grid levels run as phases of
// the whole launch separated by device-wide barriers; the levels of at most
// tail_cells cells (the "tail") run inside one thread block -- block b for
// problem b -- in its shared memory when they fit.  The problems advance in
// lockstep: each phase loops over the problems before the barrier, so the
// barrier cost is shared and small problems fill the GPU together; each
// problem keeps its own reductions, iteration count and stop test (a
// converged problem skips its work).
//
// Precision.  FP64 (MT = double): the CG vectors, products, dots and the
// V-cycle in FP64.  Mixed (MT = float), "FP32 sweeps inside FP64
// refinement": the defect r0 = rhs - A p of the FP64 pressure equation is
// formed in FP64, then the correction equation A x = r0 is solved to the
// relative tolerance by CG in FP32 (FP32 operator copy, vectors and
// V-cycle); the dot products are summed in FP32 per thread and warp and in
// FP64 across warps and blocks, and the CG scalars are FP64; at the end
// pn = p + x in FP64.  Every sweep starts from a fresh FP64 defect, so the
// steady state solves the FP64 equations.  FP32 cannot resolve a correction
// much below 1e-6 of its right-hand side, so the mixed solve stops at a
// relative tolerance of max(reltol, 1e-6).
//
// Reductions: every block writes its partial; after the barrier every block
// sums all partials in the same order, so every block holds the same value
// (deterministic, no atomics on floating point).
//
// Barriers: a monotone arrival counter; every wait is bounded by a poll
// budget.  A wait that runs out sets the error word, and every block that
// finds the word set at a barrier leaves the kernel there; the host reads
// the word after the sweep (HFDIB_ERR_TIMEOUT).
#include <stddef.h>
#include <string.h>

#include "common.cuh"
#include "kernels.cuh"
#include "pcg_ops.cuh"

namespace hf {

constexpr int PB_MAXB = 64;
constexpr double PB_FP32_RELTOL = 1e-6;

template <typename MT>
struct PcgbDesign {
    Grid g;
    Fields F;
    Level L0d;          // FP64 level-0 operator (the defect r0, the flux correction of a8)
    MgLevelsT<MT> M;    // preconditioner hierarchy; level 0: x = z, b = the CG residual
    int lf;             // levels 0..lf-1 by the grid, lf..nl-1 by this problem's tail block
    int smem_tail;      // the tail levels live in that block's shared memory
    double* part;       // [8][gridDim.x] partial sums of this problem
    float* d32[2];      // mixed: FP32 search directions
    float* q32;         // mixed: FP32 A d
    float* x32;         // mixed: FP32 correction
    MT* rbuf[2];        // the CG residual, double-buffered: rbuf[0] is level 0's b (the
                        // initial residual); iteration it reads rbuf[it & 1] and writes
                        // rbuf[(it + 1) & 1], the b of that iteration's V-cycle
};

template <typename MT>
struct PcgbArgs {
    const PcgbDesign<MT>* D;   // device array of B descriptors
    int B;
    int maxlev;
    int coarse_sweeps;
    double reltol;
    int maxit;
    unsigned int* bar;     // arrival counter (zeroed before each launch)
    int* err;              // error word (zeroed before each launch)
    long long spin_limit;  // polls of one barrier wait before giving up
    long long* trace;      // nullable: block 0 records (phase, ns) pairs
    int trace_cap;
    int skip;              // 1: problems whose stop flag (scal[SC_DONE]) is set do nothing
};

// ---------------------------------------------------------------- barrier
__device__ __forceinline__ unsigned int pb_ld_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long pb_global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

// trace entries written so far (block 0, thread 0; kept on chip so that a
// mark costs two posted stores and no read)
__device__ inline int& pb_tn() {
    __shared__ int n;
    return n;
}

template <typename MT>
__device__ inline void pb_mark(const PcgbArgs<MT>& A, int tag) {
    if (A.trace && blockIdx.x == 0 && threadIdx.x == 0) {
        const int n = pb_tn();
        if (n < A.trace_cap) {
            A.trace[1 + 2 * n] = tag;
            A.trace[2 + 2 * n] = pb_global_ns();
            A.trace[0] = n + 1;
            pb_tn() = n + 1;
        }
    }
}

// trace marks inside the coarse tail (pl_tail calls it with every thread)
template <typename MT>
struct PbMark {
    const PcgbArgs<MT>* A;
    __device__ void operator()(int tag) const { pb_mark(*A, tag); }
};

// barriers this block has passed (every block passes the same sequence, so
// the n-th barrier is complete when the arrival counter reaches n * blocks)
__device__ inline unsigned int& pb_gen() {
    __shared__ unsigned int gen;
    return gen;
}

// Grid barrier: thread 0 posts its arrival (a release add that returns
// nothing, so the poll starts at once) and polls the counter until it
// reaches this barrier's target.  A wait that runs out of polls sets the
// error word; the word is polled every 64 polls (a rare, slow path), so a
// wait that finds it set stops.  The whole block then continues or, on an
// error, leaves the kernel together (block-uniform, after the block
// barrier, so no thread is left at a later __syncthreads).
template <typename MT>
__device__ inline void pb_sync(const PcgbArgs<MT>& A, int tag) {
    __shared__ int s_abort;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int gen = pb_gen() + 1u;
        pb_gen() = gen;
        const unsigned int target = gen * gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(A.bar) : "memory");
        long long spins = 0;
        int abort = 0;
        while ((int)(pb_ld_acquire(A.bar) - target) < 0) {
            ++spins;
            if (spins > A.spin_limit) { atomicExch(A.err, 1); abort = 1; break; }
            if ((spins & 63) == 0 && *(const volatile int*)A.err) { abort = 1; break; }
        }
        s_abort = abort;
    }
    __syncthreads();
    if (s_abort) asm volatile("exit;");
    pb_mark(A, tag);
}

// sm[0 .. n-1] (n <= 32) summed by one warp in a fixed shuffle tree; the sum
// is valid in lane 0 (a serial sum by one thread would chain 32 FP64 adds,
// each waiting for the last)
__device__ __forceinline__ double pb_warp_sum(const double* sm, int n) {
    const int lane = threadIdx.x & 31;
    double y = lane < n ? sm[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
    return y;
}

// Block partial of v into slot q: summed in the type of v per thread and
// across the lanes of a warp, in FP64 across the warps of the block.
template <typename AT>
__device__ inline void pb_partial(double* part, int q, AT v) {
    __shared__ double sm[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[warp] = (double)v;
    __syncthreads();
    if (warp == 0) {
        const double x = pb_warp_sum(sm, (int)(blockDim.x >> 5));
        if (lane == 0) part[(long long)q * gridDim.x + blockIdx.x] = x;
    }
}

// slots q0 .. q0 + NV - 1 summed over all blocks with one round of loads,
// each in the same order as pb_total
template <int NV>
__device__ inline void pb_totals(const double* part, int q0, double (&out)[NV]) {
    __shared__ double sm[NV][32];
    __shared__ double res[NV];
    double x[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
        for (int v = 0; v < NV; ++v) x[v] += __ldcg(&part[(long long)(q0 + v) * gridDim.x + b]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v)
        for (int o = 16; o > 0; o >>= 1) x[v] += __shfl_down_sync(0xffffffffu, x[v], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int v = 0; v < NV; ++v) sm[v][warp] = x[v];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const double y = pb_warp_sum(sm[v], (int)(blockDim.x >> 5));
            if (lane == 0) res[v] = y;
        }
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = res[v];
}

// slot q summed over all blocks, the same value in every block (fixed order)
__device__ inline double pb_total(const double* part, int q) {
    __shared__ double sm[32];
    __shared__ double res;
    double x = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) x += __ldcg(&part[(long long)q * gridDim.x + b]);
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const double y = pb_warp_sum(sm, (int)(blockDim.x >> 5));
        if (lane == 0) res = y;
    }
    __syncthreads();
    return res;
}

enum { QB_RZ = 0, QB_RR = 1, QB_R1 = 2, QB_R2 = 3, QB_R3 = 4, QB_DQ = 5 };

// per-problem loop state, identical in every block; off: the problem sits
// this launch out (its batch solve has stopped)
struct PbState {
    double rz[PB_MAXB], rzp[PB_MAXB], tol2[PB_MAXB], dq[PB_MAXB], rr[PB_MAXB];
    // the CG step scalars, formed once by thread 0: an FP64 division by every
    // thread of a block costs microseconds on this GPU
    double alpha[PB_MAXB], beta[PB_MAXB];
    int it[PB_MAXB], done[PB_MAXB], off[PB_MAXB];
};

extern __shared__ __align__(16) unsigned char pb_dyn_smem[];

// this block's tail table: its problem's levels, the tail ones in shared memory
template <typename MT>
__device__ inline MgLevelsT<MT>* pb_table() {
    __shared__ MgLevelsT<MT> table;
    return &table;
}

// first cell of x-pair p: i0 = 2 * (pair column), j, k and its index
template <int D, typename T>
__device__ __forceinline__ void pb_pair(const LevelT<T>& L, int p, int& i0, int& j, int& k, int& c0) {
    const int npx = (L.nx + 1) >> 1;
    const int r = p / npx;
    i0 = 2 * (p - r * npx);
    if (D == 2) {
        j = r;
        k = 0;
    } else {
        k = r / L.ny;
        j = r - k * L.ny;
    }
    c0 = r * L.nx + i0;
}

// ---------------------------------------------------------------- set-up
// FP64 level-0 operator from rAU (face coefficients and diagonal; the FP64
// path also its inverse diagonal) and, on the mixed path, its FP32 copy
template <int D, typename MT>
__device__ void pb_build0(const PcgbDesign<MT>& Dz, int t0, int TT) {
    constexpr bool fp32 = sizeof(MT) == 4;
    const Grid& g = Dz.g;
    const Level L = Dz.L0d;
    const LevelT<MT> P0 = Dz.M.lv[0];
    const double* __restrict__ rAU = Dz.F.rAU;
    const int N = (int)g.N;
    const int sy = g.nx, sz = g.nx * g.ny;
    for (int c = t0; c < N; c += TT) {
        int i, j, k;
        pl_ijk<D>(L, c, i, j, k);
        const int idx[3] = {i, j, k};
        const double rP = rAU[c];
        double diag = 0.0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int fl = d == 0 ? pl_fx(L, i, j, k) : (d == 1 ? pl_fy(L, i, j, k) : c);
            const int fs = d == 0 ? 1 : (d == 1 ? L.nx : sz);
            const int cs = d == 0 ? 1 : (d == 1 ? sy : sz);
            double clo, chi;
            if (idx[d] > 0) clo = 0.5 * (rP + rAU[c - cs]) * g.SoD[d];
            else clo = p_fixed(g, 2 * d) ? rP * g.SoHD[d] : 0.0;
            if (idx[d] < g.n[d] - 1) chi = 0.5 * (rP + rAU[c + cs]) * g.SoD[d];
            else chi = p_fixed(g, 2 * d + 1) ? rP * g.SoHD[d] : 0.0;
            L.cf[d][fl] = clo;
            if (fp32) P0.cf[d][fl] = (MT)clo;
            if (idx[d] == g.n[d] - 1) {
                L.cf[d][fl + fs] = chi;
                if (fp32) P0.cf[d][fl + fs] = (MT)chi;
            }
            diag += clo + chi;
        }
        L.diag[c] = diag;
        if constexpr (fp32) {
            const float df = (float)diag;
            P0.diag[c] = df;
            P0.idg[c] = df > 0.0f ? 1.0f / df : 0.0f;
        } else {
            L.idg[c] = diag > 0.0 ? 1.0 / diag : 0.0;
        }
    }
}

// block b: its problem's tail levels lf..nl-1 built directly in dynamic
// shared memory (level lf coarsened from the grid's level lf-1, each further
// level from the shared one above it)
template <int D, typename MT>
__device__ void pb_build_tail(const PcgbArgs<MT>& A, const PcgbDesign<MT>& Dz) {
    MgLevelsT<MT>* S = pb_table<MT>();
    if (threadIdx.x == 0) {
        *S = Dz.M;
        MT* p = (MT*)pb_dyn_smem;
        for (int l = Dz.lf; l < Dz.M.nl; ++l) {
            LevelT<MT>& L = S->lv[l];
            L.diag = p; p += L.N;
            L.idg = p; p += L.N;
            L.x = p; p += L.N;
            L.b = p; p += L.N;
            L.cf[0] = p; p += (long long)(L.nx + 1) * L.ny * L.nz;
            L.cf[1] = p; p += (long long)L.nx * (L.ny + 1) * L.nz;
            if (D == 3) { L.cf[2] = p; p += (long long)L.nx * L.ny * (L.nz + 1); }
        }
    }
    __syncthreads();
    pb_mark(A, PH_TB_TABLE);
    for (int l = Dz.lf; l < Dz.M.nl; ++l) {
        if (l == Dz.lf) pl_coarsen<D>(Dz.M.lv[l - 1], S->lv[l], threadIdx.x, blockDim.x);
        else pl_coarsen<D>(S->lv[l - 1], S->lv[l], threadIdx.x, blockDim.x);
        __syncthreads();
        pb_mark(A, PH_TB_LEVEL);
    }
}

// ---------------------------------------------------------------- CG update
// sum over the neighbours of cf * z_red with z_red = (rold - a q) / diag:
// the zero-start red values of the next V-cycle at the (red) neighbours of a
// black cell, recomputed from the old residual buffer, in pl_offsum's order
// and branch-free like it (a missing neighbour's term dropped by a select)
template <int D, typename T>
__device__ __forceinline__ T pb_red_offsum(const LevelT<T>& L, const T* __restrict__ rold,
                                           const T* __restrict__ q, T a, int c, int i, int j, int k) {
    const int fx = pl_fx(L, i, j, k), fy = pl_fy(L, i, j, k);
    const bool xm = i > 0, xp = i < L.nx - 1, ym = j > 0, yp = j < L.ny - 1;
    const int nxm = xm ? c - 1 : c, nxp = xp ? c + 1 : c, nym = ym ? c - L.nx : c, nyp = yp ? c + L.nx : c;
    const T cxm = L.cf[0][fx], cxp = L.cf[0][fx + 1], cym = L.cf[1][fy], cyp = L.cf[1][fy + L.nx];
    const T zxm = (rold[nxm] - a * q[nxm]) * L.idg[nxm];
    const T zxp = (rold[nxp] - a * q[nxp]) * L.idg[nxp];
    const T zym = (rold[nym] - a * q[nym]) * L.idg[nym];
    const T zyp = (rold[nyp] - a * q[nyp]) * L.idg[nyp];
    T acc = T(0);
    acc = xm ? pl_fma(cxm, zxm, acc) : acc;
    acc = xp ? pl_fma(cxp, zxp, acc) : acc;
    acc = ym ? pl_fma(cym, zym, acc) : acc;
    acc = yp ? pl_fma(cyp, zyp, acc) : acc;
    if (D == 3) {
        const int s = L.nx * L.ny;
        const bool zm = k > 0, zp = k < L.nz - 1;
        const int nzm = zm ? c - s : c, nzp = zp ? c + s : c;
        const T czm = L.cf[2][c], czp = L.cf[2][c + s];
        const T zzm = (rold[nzm] - a * q[nzm]) * L.idg[nzm];
        const T zzp = (rold[nzp] - a * q[nzp]) * L.idg[nzp];
        acc = zm ? pl_fma(czm, zzm, acc) : acc;
        acc = zp ? pl_fma(czp, zzp, acc) : acc;
    }
    return acc;
}

// The CG update of one problem fused with the start of the next V-cycle on
// level 0: x += a d, rnew = rold - a q, and z (level 0's x) = the zero-start
// red half sweep followed by the black one.  The owners of the red cells
// write only rnew, so each black cell recomputes its red neighbours' values
// from rold and no grid barrier separates the two half sweeps.  One x-pair
// (one red and one black cell) per thread.  Returns this thread's r.r.
template <int D, typename T, typename XT>
__device__ T pb_update_start(const LevelT<T>& P0, XT* __restrict__ x, const T* __restrict__ dn,
                             const T* __restrict__ q, const T* __restrict__ rold, T* __restrict__ rnew, T a,
                             int t0, int TT) {
    T s_r2 = T(0);
    const int NP = pl_npairs(P0);
    for (int p = t0; p < NP; p += TT) {
        int i0, j, k, c0;
        pb_pair<D>(P0, p, i0, j, k, c0);
        const bool two = i0 + 1 < P0.nx;
        // the black cell of the pair (if the pair has only a red cell, the
        // neighbour sum is taken at cell 0 and not used)
        const int ob = ((i0 + j + k) & 1) ^ 1;
        const int ib = (ob && two) ? i0 + 1 : i0;
        const T sb = pb_red_offsum<D>(P0, rold, q, a, c0 + (ib - i0), ib, j, k);
        T xv[2], rv[2], zv[2];
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            const int i = (o && two) ? i0 + 1 : i0, c = c0 + (i - i0);
            xv[o] = (T)x[c] + a * dn[c];
            rv[o] = rold[c] - a * q[c];
            zv[o] = (o == ob ? rv[o] + sb : rv[o]) * P0.idg[c];
        }
        x[c0] = (XT)xv[0];
        rnew[c0] = rv[0];
        P0.x[c0] = zv[0];
        s_r2 += rv[0] * rv[0];
        if (two) {
            x[c0 + 1] = (XT)xv[1];
            rnew[c0 + 1] = rv[1];
            P0.x[c0 + 1] = zv[1];
            s_r2 += rv[1] * rv[1];
        }
    }
    return s_r2;
}

// ---------------------------------------------------------------- V-cycle
// level l of problem Dz as the V-cycle sees it: level 0's b is the residual
// buffer rbuf[rsel]
template <typename MT>
__device__ __forceinline__ LevelT<MT> pb_level(const PcgbDesign<MT>& Dz, int l, int rsel) {
    LevelT<MT> L = Dz.M.lv[l];
    if (l == 0) L.b = Dz.rbuf[rsel];
    return L;
}

// z = B r for every active problem, r = rbuf[rsel]; the level-0 zero-start
// red half sweep is done, and so is the black one when `started` (the CG
// update fuses both).  The final red half sweep of level 0 accumulates r.z
// into QB_RZ.
template <int D, typename MT>
__device__ void pb_vcycle(const PcgbArgs<MT>& A, const PbState& S, int t0, int TT, int rsel, bool started) {
    const int B = A.B;
    if (!started) {
        for (int b = 0; b < B; ++b)
            if (!S.done[b]) pl_smooth<D>(pb_level(A.D[b], 0, rsel), 1, t0, TT);
        pb_sync(A, PH_VC_SMOOTH0);
    }
    // Down: restriction (with the coarse level's zero-start red half sweep),
    // then the black half sweep.  (Folding the black half sweep into the
    // restriction, with each black coarse cell recomputing its red
    // neighbours from their children, measured three times slower than the
    // two phases.)
    for (int l = 0; l + 1 < A.maxlev; ++l) {
        bool any = false;
        for (int b = 0; b < B; ++b) {
            const PcgbDesign<MT>& Dz = A.D[b];
            if (S.done[b]) continue;
            const int lf = Dz.lf, nl = Dz.M.nl;
            if (l + 1 < lf) {
                pl_restrict<D>(pb_level(Dz, l, rsel), Dz.M.lv[l + 1], true, t0, TT);
                any = true;
            } else if (l + 1 == lf && lf < nl) {
                pl_restrict<D>(pb_level(Dz, l, rsel), Dz.M.lv[l + 1], false, t0, TT);
                any = true;
            }
        }
        if (!any) break;
        pb_sync(A, PH_VC_RESTRICT);
        bool smooth = false;
        for (int b = 0; b < B; ++b) {
            const PcgbDesign<MT>& Dz = A.D[b];
            if (!S.done[b] && l + 1 < Dz.lf) {
                pl_smooth<D>(Dz.M.lv[l + 1], 1, t0, TT);
                smooth = true;
            }
        }
        // (after the restriction into a tail level nothing is smoothed here)
        if (smooth) pb_sync(A, PH_VC_SMOOTH);
    }
    // coarse tails: problem b on block b
    bool tails = false;
    for (int b = 0; b < B; ++b) {
        const PcgbDesign<MT>& Dz = A.D[b];
        if (S.done[b] || Dz.lf >= Dz.M.nl) continue;
        tails = true;
        if (b != (int)blockIdx.x) continue;
        const int lf = Dz.lf;
        if (Dz.smem_tail) {
            const MgLevelsT<MT>& T = *pb_table<MT>();
            const LevelT<MT> G = Dz.M.lv[lf];
            const int n = (int)G.N;
            for (int c = threadIdx.x; c < n; c += blockDim.x) T.lv[lf].b[c] = G.b[c];
            __syncthreads();
            pb_mark(A, PH_TAIL_IN);
            pl_tail<D>(T, lf, A.coarse_sweeps, PbMark<MT>{&A});
            __syncthreads();
            pb_mark(A, PH_TAIL_DONE);
            for (int c = threadIdx.x; c < n; c += blockDim.x) G.x[c] = T.lv[lf].x[c];
            __syncthreads();
        } else {
            pl_tail<D>(Dz.M, lf, A.coarse_sweeps, PbMark<MT>{&A});
        }
    }
    if (tails) pb_sync(A, PH_VC_TAIL);
    // Up: prolongation with the black half sweep, then the red half sweep.
    // In 2D the red half sweep of a grid level l >= 1 has no phase of its
    // own: the prolongation into level l - 1 recomputes the red values it
    // reads (pl_prolong_black_red), which saves one grid phase per level.
    // (In 3D a fine black cell would recompute six coarse red cells, more
    // work than the phase it saves.)
    constexpr bool fold_red = D == 2;
    for (int l = A.maxlev - 1; l >= 0; --l) {
        bool any = false;
        for (int b = 0; b < B; ++b) {
            const PcgbDesign<MT>& Dz = A.D[b];
            if (S.done[b] || l >= Dz.lf) continue;
            any = true;
            if (l + 1 < Dz.M.nl) {
                if (fold_red && l + 1 < Dz.lf)
                    pl_prolong_black_red<D>(pb_level(Dz, l, rsel), Dz.M.lv[l + 1], t0, TT);
                else
                    pl_prolong_black<D>(pb_level(Dz, l, rsel), Dz.M.lv[l + 1], t0, TT);
            } else {
                pl_smooth<D>(pb_level(Dz, l, rsel), 1, t0, TT);
            }
        }
        if (!any) continue;
        pb_sync(A, PH_VC_PROLONG);
        if (l > 0 && !fold_red) {
            for (int b = 0; b < B; ++b) {
                const PcgbDesign<MT>& Dz = A.D[b];
                if (!S.done[b] && l < Dz.lf) pl_smooth<D>(pb_level(Dz, l, rsel), 0, t0, TT);
            }
            pb_sync(A, PH_VC_UPSMOOTH);
        }
    }
    // last red half sweep of level 0 with r.z
    for (int b = 0; b < B; ++b) {
        if (S.done[b]) continue;
        const PcgbDesign<MT>& Dz = A.D[b];
        const LevelT<MT> L0 = pb_level(Dz, 0, rsel);
        MT rz = MT(0);
        const int NP = pl_npairs(L0);
        for (int p = t0; p < NP; p += TT) {
            int i0, j, k, c0;
            pb_pair<D>(L0, p, i0, j, k, c0);
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                if (i0 + o >= L0.nx) break;
                const int c = c0 + o;
                if (((i0 + o + j + k) & 1) == 0)
                    L0.x[c] = (L0.b[c] + pl_offsum<D>(L0, L0.x, c, i0 + o, j, k)) * L0.idg[c];
                rz += L0.b[c] * L0.x[c];
            }
        }
        pb_partial(Dz.part, QB_RZ, rz);
    }
    pb_sync(A, PH_VC_FINAL);
}

// ---------------------------------------------------------------- the solver
template <typename MT, int D>
__global__ void __launch_bounds__(1024, 1) k_pressure_pcg(PcgbArgs<MT> A) {
    constexpr bool fp32 = sizeof(MT) == 4;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    const int TT = gridDim.x * blockDim.x;
    const int B = A.B;
    __shared__ PbState S;
    if (threadIdx.x == 0) {
        pb_gen() = 0u;
        if (A.trace && blockIdx.x == 0) pb_tn() = (int)A.trace[0];
        for (int b = 0; b < B; ++b) S.off[b] = A.skip && A.D[b].F.scal[SC_DONE] != 0.0;
    }
    __syncthreads();
    pb_mark(A, PH_START);
    // ---- level-0 operators, then the grid-built coarse levels
    for (int b = 0; b < B; ++b)
        if (!S.off[b]) pb_build0<D>(A.D[b], t0, TT);
    pb_sync(A, PH_BUILD0);
    for (int l = 1; l < A.maxlev; ++l) {
        bool any = false;
        for (int b = 0; b < B; ++b) {
            const PcgbDesign<MT>& Dz = A.D[b];
            const int lend = (Dz.smem_tail && Dz.lf < Dz.M.nl) ? Dz.lf : Dz.M.nl;
            if (!S.off[b] && l < lend) {
                pl_coarsen<D>(Dz.M.lv[l - 1], Dz.M.lv[l], t0, TT);
                any = true;
            }
        }
        if (!any) break;
        pb_sync(A, PH_COARSEN);
    }
    // ---- r0 = rhs - A p (FP64), the residual sums and the red start; then
    // block b builds problem b's shared-memory tail (the other blocks go on
    // to the barrier).  Every block takes the same share of cells whatever
    // the batch, so a problem's sums round the same alone and in a batch.
    for (int b = 0; b < B; ++b) {
        if (S.off[b]) continue;
        const PcgbDesign<MT>& Dz = A.D[b];
        const Grid& g = Dz.g;
        const Fields& F = Dz.F;
        const Level L0 = Dz.L0d;
        const LevelT<MT> P0 = Dz.M.lv[0];
        double s_rr = 0, s1 = 0, s2 = 0, s3 = 0;
        const double pbar = F.scal[SC_SUM_P] * g.iN;
        const int N = (int)g.N;
        for (int c = t0; c < N; c += TT) {
            int i, j, k;
            pl_ijk<D>(L0, c, i, j, k);
            const uint16_t f = F.flags[c];
            const int idx[3] = {i, j, k};
            double div = 0.0, bout = 0.0, A1 = 0.0;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int fl = d == 0 ? pl_fx(L0, i, j, k) : (d == 1 ? pl_fy(L0, i, j, k) : c);
                const int fs = d == 0 ? 1 : (d == 1 ? L0.nx : L0.nx * L0.ny);
                div += F.phiH[d][fl + fs] - F.phiH[d][fl];
                if (idx[d] == 0 && p_fixed(g, 2 * d)) { bout += L0.cf[d][fl] * g.p_out; A1 += L0.cf[d][fl]; }
                if (idx[d] == g.n[d] - 1 && p_fixed(g, 2 * d + 1)) {
                    bout += L0.cf[d][fl + fs] * g.p_out;
                    A1 += L0.cf[d][fl + fs];
                }
            }
            const double rhs = -masked_div(g, F.lam, f, c, div) + bout;
            const double pc = F.p[c];
            const double Ap = L0.diag[c] * pc - pl_offsum<D>(L0, F.p, c, i, j, k);
            const double r = rhs - Ap;
            const MT rb = (MT)r;
            if constexpr (fp32) {
                P0.b[c] = rb;
                Dz.x32[c] = 0.0f;
            } else {
                F.r[c] = r;
                F.pn[c] = pc;
            }
            if (((i + j + k) & 1) == 0) P0.x[c] = rb * P0.idg[c];
            s_rr += r * r;
            s1 += fabs(r);
            s2 += fabs(Ap - A1 * pbar);
            s3 += fabs(rhs - A1 * pbar);
        }
        pb_partial(Dz.part, QB_RR, s_rr);
        pb_partial(Dz.part, QB_R1, s1);
        pb_partial(Dz.part, QB_R2, s2);
        pb_partial(Dz.part, QB_R3, s3);
    }
    pb_mark(A, PH_R0_SHARE);
    if ((int)blockIdx.x < B && !S.off[blockIdx.x] && A.D[blockIdx.x].smem_tail &&
        A.D[blockIdx.x].lf < A.D[blockIdx.x].M.nl)
        pb_build_tail<D>(A, A.D[blockIdx.x]);
    pb_sync(A, PH_R0);
    const double reltol = fp32 ? fmax(A.reltol, PB_FP32_RELTOL) : A.reltol;
    for (int b = 0; b < B; ++b) {
        if (S.off[b]) {
            if (threadIdx.x == 0) S.done[b] = 1;
            continue;
        }
        const PcgbDesign<MT>& Dz = A.D[b];
        static_assert(QB_R1 == QB_RR + 1 && QB_R2 == QB_RR + 2 && QB_R3 == QB_RR + 3, "slot order");
        double tot[4];
        pb_totals<4>(Dz.part, QB_RR, tot);
        const double rr0 = tot[0], r1 = tot[1], r2 = tot[2], r3 = tot[3];
        if (threadIdx.x == 0) {
            S.tol2[b] = reltol * reltol * rr0;
            S.done[b] = (rr0 > 0.0 && isfinite(rr0) && A.maxit > 0) ? 0 : 1;
            S.it[b] = 0;
            S.rzp[b] = 1.0;
            if (blockIdx.x == 0) {
                Dz.F.scal[SC_PCG_INIT + 1] = rr0;
                Dz.F.scal[SC_PCG_INIT + 3] = r1;
                Dz.F.scal[SC_PCG_INIT + 4] = r2;
                Dz.F.scal[SC_PCG_INIT + 5] = r3;
            }
        }
    }
    __syncthreads();
    pb_vcycle<D>(A, S, t0, TT, 0, false);
    for (int b = 0; b < B; ++b) {
        if (S.off[b]) continue;
        const double rz = pb_total(A.D[b].part, QB_RZ);
        if (threadIdx.x == 0) {
            S.rz[b] = rz;
            S.beta[b] = 0.0;
        }
    }
    __syncthreads();
    for (int iter = 0; iter < A.maxit; ++iter) {
        bool all = true;
        for (int b = 0; b < B; ++b) all = all && S.done[b];
        if (all) break;
        // d = z + beta d_old; q = A d = A z + beta q_old (by linearity the
        // neighbours' d need not be rebuilt); d.q
        for (int b = 0; b < B; ++b) {
            if (S.done[b]) continue;
            const PcgbDesign<MT>& Dz = A.D[b];
            const int it = S.it[b];
            const double beta = S.beta[b];
            // one x-pair per thread: both cells' loads issue before the
            // first store (a cell loop would wait for its first cell's
            // stores before loading the second)
            if constexpr (fp32) {
                const LevelT<float> P0 = Dz.M.lv[0];
                const float* __restrict__ z = P0.x;
                const float* __restrict__ dold = Dz.d32[it & 1];
                float* __restrict__ dnew = Dz.d32[(it + 1) & 1];
                float* __restrict__ q = Dz.q32;
                const float fb = (float)beta;
                float s_dq = 0.0f;
                const int NP = pl_npairs(P0);
                for (int p = t0; p < NP; p += TT) {
                    int i0, j, k, c0;
                    pb_pair<D>(P0, p, i0, j, k, c0);
                    const bool two = i0 + 1 < P0.nx;
                    float dP[2], qv[2];
#pragma unroll
                    for (int o = 0; o < 2; ++o) {
                        const int i = (o && two) ? i0 + 1 : i0, c = c0 + (i - i0);
                        const float zc = z[c];
                        const float Az = P0.diag[c] * zc - pl_offsum<D>(P0, z, c, i, j, k);
                        dP[o] = it == 0 ? zc : zc + fb * dold[c];
                        qv[o] = it == 0 ? Az : Az + fb * q[c];
                    }
                    dnew[c0] = dP[0];
                    q[c0] = qv[0];
                    s_dq += dP[0] * qv[0];
                    if (two) {
                        dnew[c0 + 1] = dP[1];
                        q[c0 + 1] = qv[1];
                        s_dq += dP[1] * qv[1];
                    }
                }
                pb_mark(A, PH_B0_LOOP);
                pb_partial(Dz.part, QB_DQ, s_dq);
                pb_mark(A, PH_B0_PART);
            } else {
                const Fields& F = Dz.F;
                const Level L0 = Dz.L0d;
                const double* __restrict__ z = Dz.M.lv[0].x;
                const double* __restrict__ dold = F.d[it & 1];
                double* __restrict__ dnew = F.d[(it + 1) & 1];
                double* __restrict__ q = F.q;
                double s_dq = 0.0;
                const int NP = pl_npairs(L0);
                for (int p = t0; p < NP; p += TT) {
                    int i0, j, k, c0;
                    pb_pair<D>(L0, p, i0, j, k, c0);
                    const bool two = i0 + 1 < L0.nx;
                    double dP[2], qv[2];
#pragma unroll
                    for (int o = 0; o < 2; ++o) {
                        const int i = (o && two) ? i0 + 1 : i0, c = c0 + (i - i0);
                        const double zc = z[c];
                        const double Az = L0.diag[c] * zc - pl_offsum<D>(L0, z, c, i, j, k);
                        dP[o] = it == 0 ? zc : zc + beta * dold[c];
                        qv[o] = it == 0 ? Az : Az + beta * q[c];
                    }
                    dnew[c0] = dP[0];
                    q[c0] = qv[0];
                    s_dq += dP[0] * qv[0];
                    if (two) {
                        dnew[c0 + 1] = dP[1];
                        q[c0 + 1] = qv[1];
                        s_dq += dP[1] * qv[1];
                    }
                }
                pb_partial(Dz.part, QB_DQ, s_dq);
            }
        }
        pb_sync(A, PH_CG_PRODUCT);
        for (int b = 0; b < B; ++b) {
            if (S.done[b]) continue;
            const double dq = pb_total(A.D[b].part, QB_DQ);
            if (threadIdx.x == 0) {
                S.dq[b] = dq;
                S.alpha[b] = dq != 0.0 ? S.rz[b] / dq : 0.0;
            }
        }
        __syncthreads();
        // x += alpha d (FP64 path: p += alpha d); r -= alpha q into the other
        // residual buffer; r.r; and level 0's two zero-start half sweeps of
        // the next V-cycle
        const int rin = iter & 1, rout = (iter + 1) & 1;
        for (int b = 0; b < B; ++b) {
            if (S.done[b]) continue;
            const PcgbDesign<MT>& Dz = A.D[b];
            const LevelT<MT> P0 = Dz.M.lv[0];
            const double alpha = S.alpha[b];
            const int it1 = (S.it[b] + 1) & 1;
            if constexpr (fp32) {
                const float s_r2 = pb_update_start<D, float, float>(P0, Dz.x32, Dz.d32[it1], Dz.q32, Dz.rbuf[rin],
                                                                    Dz.rbuf[rout], (float)alpha, t0, TT);
                pb_mark(A, PH_B0_LOOP);
                pb_partial(Dz.part, QB_RR, s_r2);
                pb_mark(A, PH_B0_PART);
            } else {
                const Fields& F = Dz.F;
                const double s_r2 = pb_update_start<D, double, double>(P0, F.pn, F.d[it1], F.q, Dz.rbuf[rin],
                                                                       Dz.rbuf[rout], alpha, t0, TT);
                pb_partial(Dz.part, QB_RR, s_r2);
            }
        }
        pb_sync(A, PH_CG_UPDATE);
        for (int b = 0; b < B; ++b) {
            if (S.done[b]) continue;
            const double rr = pb_total(A.D[b].part, QB_RR);
            if (threadIdx.x == 0) S.rr[b] = rr;
        }
        __syncthreads();
        pb_vcycle<D>(A, S, t0, TT, rout, true);
        for (int b = 0; b < B; ++b) {
            if (S.done[b]) continue;
            const double rz = pb_total(A.D[b].part, QB_RZ);
            if (threadIdx.x == 0) {
                S.rzp[b] = S.rz[b];
                S.rz[b] = rz;
                S.beta[b] = rz / S.rzp[b];
                S.it[b] += 1;
                if (!(S.rr[b] > S.tol2[b]) || S.it[b] >= A.maxit) S.done[b] = 1;
            }
        }
        __syncthreads();
        // no grid barrier here: every partial slot read above is written again
        // only after the next iteration's product and update barriers
    }
    // mixed: the FP64 solution p + x (no barrier needed: the kernel ends)
    if constexpr (fp32) {
        for (int b = 0; b < B; ++b) {
            if (S.off[b]) continue;
            const PcgbDesign<MT>& Dz = A.D[b];
            const Fields& F = Dz.F;
            const float* __restrict__ x = Dz.x32;
            const int N = (int)Dz.g.N;
            // two cells per thread, both loaded before either store
            for (int c = 2 * t0; c < N; c += 2 * TT) {
                const bool two = c + 1 < N;
                const double v0 = F.p[c] + (double)x[c];
                const double v1 = F.p[two ? c + 1 : c] + (double)x[two ? c + 1 : c];
                F.pn[c] = v0;
                if (two) F.pn[c + 1] = v1;
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int b = 0; b < B; ++b) {
            if (S.off[b]) continue;
            const Fields& F = A.D[b].F;
            F.scal[SC_PCG_ITERS] = (double)S.it[b];
            F.scal[SC_PCG_DONE] = 1.0;
        }
    }
    pb_mark(A, PH_END);
}

// zero the arrival counter and the error word before a launch (a kernel, so
// that the reset can sit inside a graph's conditional body)
__global__ void k_pressure_reset(unsigned int* bar, int* err) {
    *bar = 0u;
    *err = 0;
}
void launch_pressure_reset(unsigned int* bar, int* err, cudaStream_t s) { k_pressure_reset<<<1, 1, 0, s>>>(bar, err); }

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

// Fill the descriptor (host copy) of one problem; returns its tail bytes
// (0 when the tail runs in global memory or there is none).
template <typename MT>
static size_t pb_describe(PcgbDesign<MT>& D, const Grid& g, const Fields& F, const MgLevels& M64,
                          const MgLevelsT<MT>& M, double* part, long long tail_cells, size_t smem_budget) {
    memset((void*)&D, 0, sizeof(D));
    D.g = g;
    D.F = F;
    D.L0d = M64.lv[0];
    D.M = M;
    D.part = part;
    D.d32[0] = F.pd32[0];
    D.d32[1] = F.pd32[1];
    D.q32 = F.pq32;
    D.x32 = F.px32;
    D.rbuf[0] = M.lv[0].b;
    if constexpr (sizeof(MT) == 4) D.rbuf[1] = F.pr32;
    else D.rbuf[1] = F.r_alt;
    // the tail: the first level of at most tail_cells cells whose levels fit
    // the shared-memory budget; if none fits, the first level of at most
    // tail_cells cells, run in global memory
    D.lf = M.nl;
    D.smem_tail = 0;
    for (int l = 1; l < M.nl; ++l) {
        if (M.lv[l].N > tail_cells) continue;
        const size_t b = pb_tail_bytes(M, g.dims, l);
        if (b <= smem_budget) {
            D.lf = l;
            D.smem_tail = 1;
            return b;
        }
    }
    for (int l = 1; l < M.nl; ++l)
        if (M.lv[l].N <= tail_cells) {
            D.lf = l;
            break;
        }
    return 0;
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
// byte offset of the Fields member in a descriptor (its p / pr pointers are
// swapped on the device by a batch's sweep end)
size_t pcgb_fields_offset(int mixed) {
    return mixed ? offsetof(PcgbDesign<float>, F) : offsetof(PcgbDesign<double>, F);
}
int pcgb_max_batch() { return PB_MAXB; }

template <typename MT, int D>
static cudaError_t pb_launch(const PcgbArgs<MT>& A, int nblk, int threads, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_pressure_pcg<MT, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
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
    PcgbArgs<MT> a = A;
    void* args[] = {&a};
    return cudaLaunchKernelExC(&cfg, (const void*)k_pressure_pcg<MT, D>, args);
}

cudaError_t launch_pressure_batched(int mixed, int dims, const void* ddesc, int B, int maxlev, int coarse_sweeps,
                                    double reltol, int maxit, int nblk, int threads, size_t smem,
                                    unsigned int* bar, int* err, long long spin_limit, long long* trace,
                                    int trace_cap, int skip, cudaStream_t s) {
    if (mixed) {
        PcgbArgs<float> A{(const PcgbDesign<float>*)ddesc, B, maxlev, coarse_sweeps, reltol, maxit, bar, err,
                          spin_limit, trace, trace_cap, skip};
        return dims == 3 ? pb_launch<float, 3>(A, nblk, threads, smem, s)
                         : pb_launch<float, 2>(A, nblk, threads, smem, s);
    }
    PcgbArgs<double> A{(const PcgbDesign<double>*)ddesc, B, maxlev, coarse_sweeps, reltol, maxit, bar, err,
                       spin_limit, trace, trace_cap, skip};
    return dims == 3 ? pb_launch<double, 3>(A, nblk, threads, smem, s)
                     : pb_launch<double, 2>(A, nblk, threads, smem, s);
}

template <typename MT, int D>
static cudaError_t pb_allow_smem(size_t smem) {
    return cudaFuncSetAttribute(k_pressure_pcg<MT, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// blocks of the launch that fit on one SM (the dynamic shared-memory limit of
// the kernel is raised to smem first, as the launch does)
int pcgb_fits(int mixed, int dims, int threads, size_t smem, int* blocks_per_sm) {
    int occ = 0;
    cudaError_t e = mixed ? (dims == 3 ? pb_allow_smem<float, 3>(smem) : pb_allow_smem<float, 2>(smem))
                          : (dims == 3 ? pb_allow_smem<double, 3>(smem) : pb_allow_smem<double, 2>(smem));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    if (mixed)
        e = dims == 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pressure_pcg<float, 3>, threads, smem)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pressure_pcg<float, 2>, threads, smem);
    else
        e = dims == 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pressure_pcg<double, 3>, threads, smem)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pressure_pcg<double, 2>, threads, smem);
    if (e != cudaSuccess) return -1;
    *blocks_per_sm = occ;
    return 0;
}

}  // namespace hf
