// pressure.cu -- pressure corrector of the sweep (Sec. 2.5.1): the
// lambda-masked pressure equation
//     laplacian(rAU_f, p) = m div(phiHbyA),   m = 1 where lambda < 1
// (Eq. hfdibrans_2 read as a masked source), solved with preconditioned CG.
//
// Operator: -laplacian as an SPD matrix: face coefficient cf = rAU_f S/Delta
// inside (rAU_f the mean of the two cells), rAU_P S/(Delta/2) on outlet
// faces (p = p_out), zero on the other boundary faces.  The face
// coefficients of the fine level are stored once per sweep and shared by the
// CG product, the multigrid smoother and the flux correction.
//
// Preconditioners: Jacobi, or one geometric-multigrid V-cycle: cell-centred
// coarsening by 2 per direction, piecewise-constant prolongation P and
// restriction R = P^T (sum over children), coarse face coefficients half the
// sum of the fine faces they cover, red-black Gauss-Seidel smoothing (red
// then black before, black then red after: the cycle is a symmetric
// positive-definite operator).  Levels of at most TAIL_CELLS cells run inside
// one thread block; the others are one launch per step.
#include "common.cuh"
#include "kernels.cuh"

namespace hf {

// ---------------------------------------------------------------- level helpers
template <typename T>
__device__ inline long long lv_face(const LevelT<T>& L, int d, int i, int j, int k) {
    if (d == 0) return ((long long)k * L.ny + j) * (L.nx + 1) + i;
    if (d == 1) return ((long long)k * (L.ny + 1) + j) * L.nx + i;
    return ((long long)k * L.ny + j) * L.nx + i;
}
template <typename T>
__device__ inline long long lv_fstride(const LevelT<T>& L, int d) {
    return d == 0 ? 1 : (d == 1 ? L.nx : (long long)L.nx * L.ny);
}
template <typename T>
__device__ inline long long lv_cstride(const LevelT<T>& L, int d) {
    return d == 0 ? 1 : (d == 1 ? L.nx : (long long)L.nx * L.ny);
}
template <typename T>
__device__ inline void lv_ijk(const LevelT<T>& L, long long c, int& i, int& j, int& k) {
    unsigned int cc = (unsigned int)c, nx = (unsigned int)L.nx;
    unsigned int r = cc / nx;
    i = (int)(cc - r * nx);
    if (L.nz == 1) { j = (int)r; k = 0; return; }
    unsigned int ny = (unsigned int)L.ny;
    unsigned int kk = r / ny;
    j = (int)(r - kk * ny);
    k = (int)kk;
}

// (A x)_P = diag x_P - sum over interior faces cf x_N
__device__ inline double lv_offsum(const Level& L, int dims, const double* x, long long c, int i, int j, int k) {
    double acc = 0.0;
    const int idx[3] = {i, j, k};
    const int nn[3] = {L.nx, L.ny, L.nz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= dims) break;
        long long fl = lv_face(L, d, i, j, k);
        long long cs = lv_cstride(L, d);
        if (idx[d] > 0) acc += L.cf[d][fl] * x[c - cs];
        if (idx[d] < nn[d] - 1) acc += L.cf[d][fl + lv_fstride(L, d)] * x[c + cs];
    }
    return acc;
}

// ---------------------------------------------------------------- fine coefficients
__global__ void k_p_coef(Grid g, Level L, const double* __restrict__ rAU) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const int idx[3] = {i, j, k};
    double diag = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= g.dims) break;
        long long fl = lv_face(L, d, i, j, k);
        long long fs = lv_fstride(L, d);
        double clo, chi;
        if (idx[d] > 0) clo = 0.5 * (rAU[c] + rAU[c - g.stride[d]]) * g.SoD[d];
        else clo = p_fixed(g, 2 * d) ? rAU[c] * g.SoHD[d] : 0.0;
        if (idx[d] < g.n[d] - 1) chi = 0.5 * (rAU[c] + rAU[c + g.stride[d]]) * g.SoD[d];
        else chi = p_fixed(g, 2 * d + 1) ? rAU[c] * g.SoHD[d] : 0.0;
        L.cf[d][fl] = clo;
        if (idx[d] == g.n[d] - 1) L.cf[d][fl + fs] = chi;
        diag += clo + chi;
    }
    L.diag[c] = diag;
    L.idg[c] = diag > 0.0 ? 1.0 / diag : 0.0;
}

// coarse level coefficients: half the sum of the covered fine faces
template <typename T>
__device__ void coarsen_cell(const LevelT<T>& F, const LevelT<T>& Cc, int dims, long long C) {
    int I, J, K;
    lv_ijk(Cc, C, I, J, K);
    const int idx[3] = {I, J, K};
    const int nc[3] = {Cc.nx, Cc.ny, Cc.nz};
    const int nf[3] = {F.nx, F.ny, F.nz};
    T diag = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= dims) break;
        for (int side = 0; side < 2; ++side) {
            if (side == 1 && idx[d] != nc[d] - 1) continue;  // high faces: boundary only (owner writes low faces)
            int fpos = side == 0 ? 2 * idx[d] : nf[d];
            T sum = T(0);
            // the fine faces at position fpos along d covered by this coarse face
            int a1 = (d + 1) % 3, a2 = (d + 2) % 3;
            for (int o1 = 0; o1 < 2; ++o1)
                for (int o2 = 0; o2 < 2; ++o2) {
                    int fi[3];
                    fi[d] = fpos;
                    fi[a1] = 2 * idx[a1] + o1;
                    fi[a2] = 2 * idx[a2] + o2;
                    if (fi[a1] >= nf[a1] || fi[a2] >= nf[a2]) continue;
                    sum += F.cf[d][lv_face(F, d, fi[0], fi[1], fi[2])];
                }
            long long cfi = lv_face(Cc, d, I, J, K) + (side ? lv_fstride(Cc, d) : 0);
            Cc.cf[d][cfi] = T(0.5) * sum;
        }
    }
    // diagonal: all faces of the coarse cell (low faces of this cell and the
    // low faces of the +d neighbours are written by their owners, so compute
    // the sums directly from the fine level again)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= dims) break;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            int fpos = side == 0 ? 2 * idx[d] : (idx[d] == nc[d] - 1 ? nf[d] : 2 * idx[d] + 2);
            int a1 = (d + 1) % 3, a2 = (d + 2) % 3;
            T sum = T(0);
            for (int o1 = 0; o1 < 2; ++o1)
                for (int o2 = 0; o2 < 2; ++o2) {
                    int fi[3];
                    fi[d] = fpos;
                    fi[a1] = 2 * idx[a1] + o1;
                    fi[a2] = 2 * idx[a2] + o2;
                    if (fi[a1] >= nf[a1] || fi[a2] >= nf[a2]) continue;
                    sum += F.cf[d][lv_face(F, d, fi[0], fi[1], fi[2])];
                }
            diag += T(0.5) * sum;
        }
    }
    Cc.diag[C] = diag;
    Cc.idg[C] = diag > T(0) ? T(1) / diag : T(0);
}

template <typename T>
__global__ void k_coarsen(LevelT<T> F, LevelT<T> Cc, int dims) {
    long long C = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (C >= Cc.N) return;
    coarsen_cell(F, Cc, dims, C);
}

// ---------------------------------------------------------------- cycle steps
// red-black Gauss-Seidel half sweep on A x = b; zero_init: x is taken as 0
__device__ inline void smooth_cell(const Level& L, int dims, long long c, int colour, bool zero_init) {
    int i, j, k;
    lv_ijk(L, c, i, j, k);
    if (((i + j + k) & 1) != colour) return;
    double v = L.b[c];
    if (!zero_init) v += lv_offsum(L, dims, L.x, c, i, j, k);
    L.x[c] = v * L.idg[c];
}

// prolongation fused with the first (black) post-smoothing half sweep: a
// black cell reads red neighbours corrected on the fly; red cells keep stale
// values that the following red half sweep overwrites without reading them
__device__ inline void prolong_smooth_black(const Level& L, const Level& Cc, int dims, long long c) {
    int i, j, k;
    lv_ijk(L, c, i, j, k);
    if (((i + j + k) & 1) != 1) return;
    const int idx[3] = {i, j, k};
    const int nn[3] = {L.nx, L.ny, L.nz};
    double acc = L.b[c];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= dims) break;
        long long fl = lv_face(L, d, i, j, k);
        long long cs = lv_cstride(L, d);
        for (int side = 0; side < 2; ++side) {
            if (side == 0 && idx[d] == 0) continue;
            if (side == 1 && idx[d] == nn[d] - 1) continue;
            int ni[3] = {i, j, k};
            ni[d] += side ? 1 : -1;
            long long nc = side ? c + cs : c - cs;
            long long C = ((long long)(ni[2] >> 1) * Cc.ny + (ni[1] >> 1)) * Cc.nx + (ni[0] >> 1);
            double cfv = L.cf[d][fl + (side ? lv_fstride(L, d) : 0)];
            acc += cfv * (L.x[nc] + Cc.x[C]);
        }
    }
    L.x[c] = acc * L.idg[c];
}

// residual of the children, summed into the parent's right-hand side
__device__ inline void restrict_cell(const Level& F, const Level& Cc, int dims, long long C) {
    int I, J, K;
    lv_ijk(Cc, C, I, J, K);
    double sum = 0.0;
#pragma unroll
    for (int oz = 0; oz < 2; ++oz) {
        if (oz == 1 && dims != 3) break;
#pragma unroll
        for (int oy = 0; oy < 2; ++oy)
#pragma unroll
            for (int ox = 0; ox < 2; ++ox) {
                int i = 2 * I + ox, j = 2 * J + oy, k = 2 * K + oz;
                if (i >= F.nx || j >= F.ny || k >= F.nz) continue;
                long long c = ((long long)k * F.ny + j) * F.nx + i;
                double Ax = F.diag[c] * F.x[c] - lv_offsum(F, dims, F.x, c, i, j, k);
                sum += F.b[c] - Ax;
            }
    }
    Cc.b[C] = sum;
}

__device__ inline void prolong_cell(const Level& F, const Level& Cc, long long c) {
    int i, j, k;
    lv_ijk(F, c, i, j, k);
    long long C = ((long long)(k >> 1) * Cc.ny + (j >> 1)) * Cc.nx + (i >> 1);
    F.x[c] += Cc.x[C];
}

__global__ void k_smooth(Level L, int dims, int colour, int zero_init, const double* done) {
    if (*done != 0.0) return;
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.N) return;
    smooth_cell(L, dims, c, colour, zero_init != 0);
}

// last post-smoothing half sweep of the finest level, fused with r.z
__global__ void k_smooth_dot(Level L, int dims, int colour, const double* __restrict__ r, double* partials,
                             unsigned int* counter, double* out, const double* done) {
    if (*done != 0.0) return;
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[1] = {0.0};
    if (c < L.N) {
        smooth_cell(L, dims, c, colour, false);
        v[0] = r[c] * L.x[c];
    }
    grid_reduce<1, false>(v, partials, counter, out);
}

__global__ void k_prolong_black(Level L, Level Cc, int dims, const double* done) {
    if (*done != 0.0) return;
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L.N) return;
    prolong_smooth_black(L, Cc, dims, c);
}

__global__ void k_restrict(Level F, Level Cc, int dims, const double* done) {
    if (*done != 0.0) return;
    long long C = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (C >= Cc.N) return;
    restrict_cell(F, Cc, dims, C);
}

__global__ void k_prolong(Level F, Level Cc, const double* done) {
    if (*done != 0.0) return;
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= F.N) return;
    prolong_cell(F, Cc, c);
}

// ---------------------------------------------------------------- block tail
// Levels l0 .. nl-1 of one V-cycle inside one thread block.
constexpr int TAIL_THREADS = 1024;

template <typename T>
__global__ void __launch_bounds__(TAIL_THREADS) k_tail_coarsen(MgLevelsT<T> M, int dims, int l0) {
    for (int l = l0; l < M.nl; ++l) {
        const LevelT<T>& F = M.lv[l - 1];
        const LevelT<T>& Cc = M.lv[l];
        for (long long C = threadIdx.x; C < Cc.N; C += blockDim.x) coarsen_cell(F, Cc, dims, C);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(TAIL_THREADS) k_tail_cycle(MgLevels M, int dims, int l0, int coarse_sweeps,
                                                             const double* done) {
    if (*done != 0.0) return;
    const int T = blockDim.x;
    // l0 is entered with b set (restricted by the caller); x is computed here
    for (int l = l0; l < M.nl - 1; ++l) {
        const Level& L = M.lv[l];
        for (long long c = threadIdx.x; c < L.N; c += T) smooth_cell(L, dims, c, 0, true);
        __syncthreads();
        for (long long c = threadIdx.x; c < L.N; c += T) smooth_cell(L, dims, c, 1, false);
        __syncthreads();
        const Level& Cc = M.lv[l + 1];
        for (long long C = threadIdx.x; C < Cc.N; C += T) restrict_cell(L, Cc, dims, C);
        __syncthreads();
    }
    {
        const Level& L = M.lv[M.nl - 1];
        for (int s = 0; s < coarse_sweeps; ++s) {
            for (long long c = threadIdx.x; c < L.N; c += T) smooth_cell(L, dims, c, 0, s == 0);
            __syncthreads();
            for (long long c = threadIdx.x; c < L.N; c += T) smooth_cell(L, dims, c, 1, false);
            __syncthreads();
        }
        for (int s = 0; s < coarse_sweeps; ++s) {
            for (long long c = threadIdx.x; c < L.N; c += T) smooth_cell(L, dims, c, 1, false);
            __syncthreads();
            for (long long c = threadIdx.x; c < L.N; c += T) smooth_cell(L, dims, c, 0, false);
            __syncthreads();
        }
    }
    for (int l = M.nl - 2; l >= l0; --l) {
        const Level& L = M.lv[l];
        const Level& Cc = M.lv[l + 1];
        for (long long c = threadIdx.x; c < L.N; c += T) prolong_smooth_black(L, Cc, dims, c);
        __syncthreads();
        for (long long c = threadIdx.x; c < L.N; c += T) smooth_cell(L, dims, c, 0, false);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- PCG
// The iteration counter, r.z history and the convergence flag live in device
// scalars, so the same kernels run host-driven or as the body of a graph
// while-loop (k_pcg_next ends the loop through the conditional handle).
__device__ inline bool pcg_done(const Fields& F) { return F.scal[SC_PCG_DONE] != 0.0; }

// r = rhs - A p with rhs = -m div(phiHbyA) + outlet terms; Jacobi z; sums
__global__ void k_pcg_init(Grid g, Fields F, Level L0, int jacobi) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double red[6] = {0, 0, 0, 0, 0, 0};
    if (c < g.N) {
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
        double dg = L0.diag[c];
        double Ap = dg * F.p[c] - lv_offsum(L0, g.dims, F.p, c, i, j, k);
        double r = rhs - Ap;
        F.r[c] = r;
        F.d[0][c] = 0.0;
        F.d[1][c] = 0.0;
        F.pn[c] = F.p[c];
        double z = 0.0;
        if (jacobi) { z = dg > 0.0 ? r / dg : 0.0; F.z[c] = z; }
        double pbar = F.scal[SC_SUM_P] * g.iN;
        red[0] = r * z;
        red[1] = r * r;
        red[2] = rhs * rhs;
        red[3] = fabs(r);
        red[4] = fabs(Ap - A1 * pbar);
        red[5] = fabs(rhs - A1 * pbar);
    }
    // the initial V-cycle that follows must run: clear the flag of the last solve
    if (blockIdx.x == 0 && threadIdx.x == 0) F.scal[SC_PCG_DONE] = 0.0;
    grid_reduce<6, false>(red, F.partials, F.counters + 3, F.scal + SC_PCG_INIT);
}

// loop state after the initial preconditioning
__global__ void k_pcg_start(Fields F, int jacobi, double reltol, int maxit, cudaGraphConditionalHandle hcond,
                            int use_cond) {
    double* s = F.scal;
    double rr0 = s[SC_PCG_INIT + 1];
    s[SC_PCG_RZ] = jacobi ? s[SC_PCG_INIT] : s[SC_PCG_RZN];
    s[SC_PCG_RZP] = 1.0;
    s[SC_PCG_IT] = 0.0;
    s[SC_PCG_ITERS] = 0.0;
    s[SC_PCG_TOL2] = reltol * reltol * rr0;
    bool done = !(rr0 > 0.0) || maxit <= 0 || !isfinite(rr0);
    s[SC_PCG_DONE] = done ? 1.0 : 0.0;
    if (use_cond && done) cudaGraphSetConditional(hcond, 0);
}

// d = z + beta d_old (neighbours on the fly); q = A d; d.q
__global__ void k_pcg_A(Grid g, Fields F, Level L0) {
    if (pcg_done(F)) return;
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double red[1] = {0.0};
    int it = (int)F.scal[SC_PCG_IT];
    double beta = it == 0 ? 0.0 : F.scal[SC_PCG_RZ] / F.scal[SC_PCG_RZP];
    const double* dold = F.d[it & 1];
    double* dnew = F.d[(it + 1) & 1];
    if (c < g.N) {
        int i, j, k;
        cell_ijk(g, c, i, j, k);
        const int idx[3] = {i, j, k};
        double dP = F.z[c] + beta * dold[c];
        double acc = L0.diag[c] * dP;
    #pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d >= g.dims) break;
            long long fl = face_lo(g, d, i, j, k);
            if (idx[d] > 0) {
                long long nc = c - g.stride[d];
                acc -= L0.cf[d][fl] * (F.z[nc] + beta * dold[nc]);
            }
            if (idx[d] < g.n[d] - 1) {
                long long nc = c + g.stride[d];
                acc -= L0.cf[d][fl + face_stride(g, d)] * (F.z[nc] + beta * dold[nc]);
            }
        }
        dnew[c] = dP;
        F.q[c] = acc;
        red[0] = dP * acc;
    }
    grid_reduce<1, false>(red, F.partials, F.counters + 4, F.scal + SC_PCG_DQ);
}

// alpha = r.z/d.q; p += alpha d; r -= alpha q; r.r (and Jacobi z, r.z)
__global__ void k_pcg_update(Grid g, Fields F, Level L0, int jacobi) {
    if (pcg_done(F)) return;
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double red[2] = {0.0, 0.0};
    int it = (int)F.scal[SC_PCG_IT];
    double dq = F.scal[SC_PCG_DQ];
    double alpha = dq != 0.0 ? F.scal[SC_PCG_RZ] / dq : 0.0;
    const double* dn = F.d[(it + 1) & 1];
    if (c < g.N) {
        F.pn[c] += alpha * dn[c];
        double r = F.r[c] - alpha * F.q[c];
        F.r[c] = r;
        red[1] = r * r;
        if (jacobi) {
            double dg = L0.diag[c];
            double z = dg > 0.0 ? r / dg : 0.0;
            F.z[c] = z;
            red[0] = r * z;
        }
    }
    // [RZN, RR] are adjacent slots
    if (jacobi) {
        grid_reduce<2, false>(red, F.partials, F.counters + 5, F.scal + SC_PCG_RZN);
    } else {
        double v[1] = {red[1]};
        grid_reduce<1, false>(v, F.partials, F.counters + 5, F.scal + SC_PCG_RR);
    }
}

// shift r.z, count the iteration, test |r|^2 <= tol^2 |r0|^2 or the cap
__global__ void k_pcg_next(Fields F, int maxit, cudaGraphConditionalHandle hcond, int use_cond) {
    double* s = F.scal;
    if (s[SC_PCG_DONE] != 0.0) {
        if (use_cond) cudaGraphSetConditional(hcond, 0);
        return;
    }
    s[SC_PCG_RZP] = s[SC_PCG_RZ];
    s[SC_PCG_RZ] = s[SC_PCG_RZN];
    double it = s[SC_PCG_IT] + 1.0;
    s[SC_PCG_IT] = it;
    s[SC_PCG_ITERS] = it;
    double rr = s[SC_PCG_RR];
    bool done = !(rr > s[SC_PCG_TOL2]) || it >= (double)maxit;
    if (done) {
        s[SC_PCG_DONE] = 1.0;
        if (use_cond) cudaGraphSetConditional(hcond, 0);
    }
}

// ---------------------------------------------------------------- launchers
void launch_p_coef(const Grid& g, const MgLevels& M, const double* rAU, int ntail_from, cudaStream_t s) {
    k_p_coef<<<nblocks(g.N), BLOCK, 0, s>>>(g, M.lv[0], rAU);
    for (int l = 1; l < M.nl && l < ntail_from; ++l)
        k_coarsen<double><<<nblocks(M.lv[l].N), BLOCK, 0, s>>>(M.lv[l - 1], M.lv[l], g.dims);
    if (ntail_from < M.nl) k_tail_coarsen<double><<<1, TAIL_THREADS, 0, s>>>(M, g.dims, ntail_from);
}

// FP32 copy of the level-0 operator, then FP32 coarsening (mixed path)
__global__ void k_p_coef32(Grid g, Level L, Level32 P) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const int idx[3] = {i, j, k};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= g.dims) break;
        long long fl = lv_face(L, d, i, j, k);
        P.cf[d][fl] = (float)L.cf[d][fl];
        if (idx[d] == g.n[d] - 1) {
            long long fh = fl + lv_fstride(L, d);
            P.cf[d][fh] = (float)L.cf[d][fh];
        }
    }
    P.diag[c] = (float)L.diag[c];
    P.idg[c] = (float)L.idg[c];
}

void launch_p_coef32(const Grid& g, const MgLevels& M, const MgLevels32& M32, cudaStream_t s) {
    k_p_coef32<<<nblocks(g.N), BLOCK, 0, s>>>(g, M.lv[0], M32.lv[0]);
    int tail = M32.nl;
    for (int l = 1; l < M32.nl; ++l)
        if (M32.lv[l].N <= TAIL_CELLS) { tail = l; break; }
    for (int l = 1; l < M32.nl && l < tail; ++l)
        k_coarsen<float><<<nblocks(M32.lv[l].N), BLOCK, 0, s>>>(M32.lv[l - 1], M32.lv[l], g.dims);
    if (tail < M32.nl) k_tail_coarsen<float><<<1, TAIL_THREADS, 0, s>>>(M32, g.dims, tail);
}

// z = B r (one V-cycle) with r.z written to *dot_out; skipped once the
// solve has converged (device flag)
void launch_vcycle(const Grid& g, const MgLevels& M, int ntail_from, const Fields& F, double* dot_out,
                   int coarse_sweeps, cudaStream_t s) {
    int dims = g.dims;
    const double* done = F.scal + SC_PCG_DONE;
    if (M.nl == 1) {
        const Level& L = M.lv[0];
        k_smooth<<<nblocks(L.N), BLOCK, 0, s>>>(L, dims, 0, 1, done);
        k_smooth<<<nblocks(L.N), BLOCK, 0, s>>>(L, dims, 1, 0, done);
        k_smooth<<<nblocks(L.N), BLOCK, 0, s>>>(L, dims, 1, 0, done);
        k_smooth_dot<<<nblocks(L.N), BLOCK, 0, s>>>(L, dims, 0, F.r, F.partials, F.counters + 9, dot_out, done);
        return;
    }
    int lf = ntail_from;  // levels 0 .. lf-1 by grid launches
    for (int l = 0; l < lf; ++l) {
        const Level& L = M.lv[l];
        k_smooth<<<nblocks(L.N), BLOCK, 0, s>>>(L, dims, 0, 1, done);
        k_smooth<<<nblocks(L.N), BLOCK, 0, s>>>(L, dims, 1, 0, done);
        if (l + 1 < M.nl) k_restrict<<<nblocks(M.lv[l + 1].N), BLOCK, 0, s>>>(L, M.lv[l + 1], dims, done);
    }
    if (lf < M.nl) k_tail_cycle<<<1, TAIL_THREADS, 0, s>>>(M, dims, lf, coarse_sweeps, done);
    for (int l = lf - 1; l >= 0; --l) {
        const Level& L = M.lv[l];
        if (l + 1 < M.nl) k_prolong_black<<<nblocks(L.N), BLOCK, 0, s>>>(L, M.lv[l + 1], dims, done);
        else k_smooth<<<nblocks(L.N), BLOCK, 0, s>>>(L, dims, 1, 0, done);
        if (l == 0)
            k_smooth_dot<<<nblocks(L.N), BLOCK, 0, s>>>(L, dims, 0, F.r, F.partials, F.counters + 9, dot_out,
                                                        done);
        else
            k_smooth<<<nblocks(L.N), BLOCK, 0, s>>>(L, dims, 0, 0, done);
    }
}

void launch_pcg_init(const Grid& g, const Fields& F, const MgLevels& M, int jacobi, cudaStream_t s) {
    k_pcg_init<<<nblocks(g.N), BLOCK, 0, s>>>(g, F, M.lv[0], jacobi);
}
void launch_pcg_start(const Fields& F, int jacobi, double reltol, int maxit, cudaGraphConditionalHandle h,
                      int use_cond, cudaStream_t s) {
    k_pcg_start<<<1, 1, 0, s>>>(F, jacobi, reltol, maxit, h, use_cond);
}
void launch_pcg_body(const Grid& g, const Fields& F, const MgLevels& M, int ntail_from, int jacobi,
                     int coarse_sweeps, int maxit, cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
    k_pcg_A<<<nblocks(g.N), BLOCK, 0, s>>>(g, F, M.lv[0]);
    k_pcg_update<<<nblocks(g.N), BLOCK, 0, s>>>(g, F, M.lv[0], jacobi);
    if (!jacobi) launch_vcycle(g, M, ntail_from, F, F.scal + SC_PCG_RZN, coarse_sweeps, s);
    k_pcg_next<<<1, 1, 0, s>>>(F, maxit, h, use_cond);
}

}  // namespace hf
