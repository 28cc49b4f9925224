// pcg_ops.cuh -- device operations of the multigrid-preconditioned CG of the
// persistent pressure kernel (pcgb.cu): red-black half sweeps, restriction
// with the fused red start, prolongation fused with the black half sweep,
// the coarse tail run by one thread block (its smallest levels by one warp)
// and the coarse operator.
//
// Templated on the level precision T (double, or float for the FP32
// preconditioner of the mixed path) and on the number of dimensions D (2 or
// 3).  Each operation first copies its level descriptors into registers: the
// descriptors live in memory that the operation's own stores could alias
// (the shared-memory table of the tail, the global batch descriptors), so a
// reference would be re-read after every store.  Cell and face indices are 32-bit ints: a level has fewer than 2^31
// cells and faces (checked when a handle is created).
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace hf {

// levels of at most this many cells run on one warp inside the tail (their
// red-black half sweeps then need only warp barriers); a half sweep updates
// cells of one colour independently, so the result is the same as on a
// whole block
constexpr int PL_WARP_CELLS = 128;

// low x face of cell (i,j,k) in the x-face layout of the level; the high
// face is the next one
template <typename T>
__device__ __forceinline__ int pl_fx(const LevelT<T>& L, int i, int j, int k) {
    return (k * L.ny + j) * (L.nx + 1) + i;
}
// low y face; the high face is nx further on
template <typename T>
__device__ __forceinline__ int pl_fy(const LevelT<T>& L, int i, int j, int k) {
    return (k * (L.ny + 1) + j) * L.nx + i;
}
// the low z face of cell c is face c; the high face is nx*ny further on

template <int D, typename T>
__device__ __forceinline__ void pl_ijk(const LevelT<T>& L, int c, int& i, int& j, int& k) {
    const int r = c / L.nx;
    i = c - r * L.nx;
    if (D == 2) {
        j = r;
        k = 0;
    } else {
        k = r / L.ny;
        j = r - k * L.ny;
    }
}

// acc + a b with one rounding (what the compiler makes of acc += a * b)
__device__ __forceinline__ double pl_fma(double a, double b, double acc) { return __fma_rn(a, b, acc); }
__device__ __forceinline__ float pl_fma(float a, float b, float acc) { return __fmaf_rn(a, b, acc); }

// sum over the neighbours of cf * x (the off-diagonal part, sign folded in),
// in the order x-, x+, y-, y+, z-, z+.  Branch-free: a missing neighbour
// (domain edge) loads the cell itself, so every load is in bounds and all of
// them issue before the first is used, and its term is dropped by a select
// (never multiplied by zero: the cell's own x may not be set yet, and
// 0 * NaN is NaN).  The result equals the sum over the existing neighbours
// bit for bit.
template <int D, typename T, typename X>
__device__ __forceinline__ T pl_offsum(const LevelT<T>& L, const X* x, int c, int i, int j, int k) {
    const int fx = pl_fx(L, i, j, k);
    const int fy = pl_fy(L, i, j, k);
    const bool xm = i > 0, xp = i < L.nx - 1, ym = j > 0, yp = j < L.ny - 1;
    // (face fx + 1 and fy + nx exist for every cell: the face arrays hold
    // the boundary faces too)
    const T cxm = L.cf[0][fx], cxp = L.cf[0][fx + 1], cym = L.cf[1][fy], cyp = L.cf[1][fy + L.nx];
    const T vxm = (T)x[xm ? c - 1 : c];
    const T vxp = (T)x[xp ? c + 1 : c];
    const T vym = (T)x[ym ? c - L.nx : c];
    const T vyp = (T)x[yp ? c + L.nx : c];
    T acc = T(0);
    acc = xm ? pl_fma(cxm, vxm, acc) : acc;
    acc = xp ? pl_fma(cxp, vxp, acc) : acc;
    acc = ym ? pl_fma(cym, vym, acc) : acc;
    acc = yp ? pl_fma(cyp, vyp, acc) : acc;
    if (D == 3) {
        const int s = L.nx * L.ny;
        const bool zm = k > 0, zp = k < L.nz - 1;
        const T czm = L.cf[2][c], czp = L.cf[2][c + s];
        const T vzm = (T)x[zm ? c - s : c];
        const T vzp = (T)x[zp ? c + s : c];
        acc = zm ? pl_fma(czm, vzm, acc) : acc;
        acc = zp ? pl_fma(czp, vzp, acc) : acc;
    }
    return acc;
}

// Red-black passes visit the cells as x-pairs: pair p of row (j, k) holds
// cells 2p and 2p + 1, one of each colour (the last pair of an odd row has
// one cell), so a colour pass runs half the iterations of a full pass with
// no lane skipping its cell.
template <typename T>
__device__ __forceinline__ int pl_npairs(const LevelT<T>& L) {
    return ((L.nx + 1) >> 1) * L.ny * L.nz;
}
// the cell of colour `colour` in pair p; false if the pair has none
template <int D, typename T>
__device__ __forceinline__ bool pl_pair_cell(const LevelT<T>& L, int p, int colour, int& i, int& j, int& k,
                                             int& c) {
    const int npx = (L.nx + 1) >> 1;
    const int r = p / npx;          // row index k*ny + j
    const int pi = p - r * npx;
    if (D == 2) {
        j = r;
        k = 0;
    } else {
        k = r / L.ny;
        j = r - k * L.ny;
    }
    i = 2 * pi + ((j + k + colour) & 1);
    c = r * L.nx + i;
    return i < L.nx;
}

template <int D, typename T>
__device__ void pl_smooth(const LevelT<T>& Lr, int colour, int t0, int TT) {
    const LevelT<T> L = Lr;
    const int NP = pl_npairs(L);
    for (int p = t0; p < NP; p += TT) {
        int i, j, k, c;
        if (!pl_pair_cell<D>(L, p, colour, i, j, k, c)) continue;
        L.x[c] = (L.b[c] + pl_offsum<D>(L, L.x, c, i, j, k)) * L.idg[c];
    }
}

// zero-start red half sweep: x = b / diag on red cells
template <int D, typename T>
__device__ void pl_red_start(const LevelT<T>& Lr, int t0, int TT) {
    const LevelT<T> L = Lr;
    const int NP = pl_npairs(L);
    for (int p = t0; p < NP; p += TT) {
        int i, j, k, c;
        if (!pl_pair_cell<D>(L, p, 0, i, j, k, c)) continue;
        L.x[c] = L.b[c] * L.idg[c];
    }
}

// sum of the residuals b - A x of the children of coarse cell (I, J, K) on
// fine level F.  The children's loads are issued together: a missing child
// (odd fine size) is computed on the first child, which always exists, and
// dropped by a select, so the sum equals the sum over the existing children
// bit for bit.  (3D: one layer of four children at a time, which bounds the
// registers that the loads in flight take.)
template <int D, typename T>
__device__ __forceinline__ T pl_child_sum(const LevelT<T>& F, int I, int J, int K) {
    T sum = T(0);
#pragma unroll 1
    for (int oz = 0; oz < (D == 3 ? 2 : 1); ++oz) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = 2 * I + (q & 1), j = 2 * J + (q >> 1), k = 2 * K + oz;
            const bool in = i < F.nx && j < F.ny && (D == 2 || k < F.nz);
            const int ic = in ? i : 2 * I, jc = in ? j : 2 * J, kc = in ? k : 2 * K;
            const int c = (kc * F.ny + jc) * F.nx + ic;
            const T r = F.b[c] - (F.diag[c] * F.x[c] - pl_offsum<D>(F, F.x, c, ic, jc, kc));
            sum += in ? r : T(0);
        }
    }
    return sum;
}

// b_C = sum of the children's residuals; fuse_red: also the zero-start red
// half sweep of the coarse level (x_C = b_C / diag_C on red cells)
template <int D, typename T>
__device__ void pl_restrict(const LevelT<T>& Fr, const LevelT<T>& Cr, bool fuse_red, int t0, int TT) {
    const LevelT<T> F = Fr, Cc = Cr;
    const int NC = (int)Cc.N;
    for (int C = t0; C < NC; C += TT) {
        int I, J, K;
        pl_ijk<D>(Cc, C, I, J, K);
        const T sum = pl_child_sum<D>(F, I, J, K);
        Cc.b[C] = sum;
        if (fuse_red && ((I + J + K) & 1) == 0) Cc.x[C] = sum * Cc.idg[C];
    }
}

// prolongation fused with the black half sweep: the neighbours' values are
// taken with their parent's coarse correction added (red cells are then
// overwritten by the following red half sweep without being read).
// Branch-free like pl_offsum: a missing neighbour loads the cell itself and
// its term is dropped by a select.
template <int D, typename T>
__device__ void pl_prolong_black(const LevelT<T>& Lr, const LevelT<T>& Cr, int t0, int TT) {
    const LevelT<T> L = Lr, Cc = Cr;
    const int NP = pl_npairs(L);
    for (int p = t0; p < NP; p += TT) {
        int i, j, k, c;
        if (!pl_pair_cell<D>(L, p, 1, i, j, k, c)) continue;
        const bool xm = i > 0, xp = i < L.nx - 1, ym = j > 0, yp = j < L.ny - 1;
        const int im = xm ? i - 1 : i, ip = xp ? i + 1 : i, jm = ym ? j - 1 : j, jp = yp ? j + 1 : j;
        const int base = (k >> 1) * Cc.ny;
        const int fx = pl_fx(L, i, j, k), fy = pl_fy(L, i, j, k);
        const T cxm = L.cf[0][fx], cxp = L.cf[0][fx + 1], cym = L.cf[1][fy], cyp = L.cf[1][fy + L.nx];
        const int Cj = (base + (j >> 1)) * Cc.nx;
        const T vxm = L.x[c + (im - i)] + Cc.x[Cj + (im >> 1)];
        const T vxp = L.x[c + (ip - i)] + Cc.x[Cj + (ip >> 1)];
        const T vym = L.x[c + (jm - j) * L.nx] + Cc.x[(base + (jm >> 1)) * Cc.nx + (i >> 1)];
        const T vyp = L.x[c + (jp - j) * L.nx] + Cc.x[(base + (jp >> 1)) * Cc.nx + (i >> 1)];
        T acc = L.b[c];
        acc = xm ? pl_fma(cxm, vxm, acc) : acc;
        acc = xp ? pl_fma(cxp, vxp, acc) : acc;
        acc = ym ? pl_fma(cym, vym, acc) : acc;
        acc = yp ? pl_fma(cyp, vyp, acc) : acc;
        if (D == 3) {
            const int s = L.nx * L.ny;
            const bool zm = k > 0, zp = k < L.nz - 1;
            const int km = zm ? k - 1 : k, kp = zp ? k + 1 : k;
            const T czm = L.cf[2][c], czp = L.cf[2][c + s];
            const T vzm = L.x[c + (km - k) * s] + Cc.x[((km >> 1) * Cc.ny + (j >> 1)) * Cc.nx + (i >> 1)];
            const T vzp = L.x[c + (kp - k) * s] + Cc.x[((kp >> 1) * Cc.ny + (j >> 1)) * Cc.nx + (i >> 1)];
            acc = zm ? pl_fma(czm, vzm, acc) : acc;
            acc = zp ? pl_fma(czp, vzp, acc) : acc;
        }
        L.x[c] = acc * L.idg[c];
    }
}

// The value of coarse cell P = (I, J, K) after the coarse level's red half
// sweep of the way up: stored for a black cell; for a red cell recomputed
// from its (black) neighbours exactly as pl_smooth computes it.  Lets a
// prolongation read the red half sweep's result without a grid phase for it.
template <int D, typename T>
__device__ __forceinline__ T pl_coarse_final(const LevelT<T>& C, int I, int J, int K) {
    const int P = (K * C.ny + J) * C.nx + I;
    if (((I + J + K) & 1) != 0) return C.x[P];
    return (C.b[P] + pl_offsum<D>(C, C.x, P, I, J, K)) * C.idg[P];
}

// pl_prolong_black with the coarse level's red half sweep folded in: the
// coarse values are read through pl_coarse_final (the coarse level's red
// cells are then never written; nothing reads them before the next V-cycle
// sets them again)
template <int D, typename T>
__device__ void pl_prolong_black_red(const LevelT<T>& Lr, const LevelT<T>& Cr, int t0, int TT) {
    const LevelT<T> L = Lr, Cc = Cr;
    const int NP = pl_npairs(L);
    for (int p = t0; p < NP; p += TT) {
        int i, j, k, c;
        if (!pl_pair_cell<D>(L, p, 1, i, j, k, c)) continue;
        const bool xm = i > 0, xp = i < L.nx - 1, ym = j > 0, yp = j < L.ny - 1;
        const int im = xm ? i - 1 : i, ip = xp ? i + 1 : i, jm = ym ? j - 1 : j, jp = yp ? j + 1 : j;
        const int K = k >> 1;
        const int fx = pl_fx(L, i, j, k), fy = pl_fy(L, i, j, k);
        const T cxm = L.cf[0][fx], cxp = L.cf[0][fx + 1], cym = L.cf[1][fy], cyp = L.cf[1][fy + L.nx];
        const T vxm = L.x[c + (im - i)] + pl_coarse_final<D>(Cc, im >> 1, j >> 1, K);
        const T vxp = L.x[c + (ip - i)] + pl_coarse_final<D>(Cc, ip >> 1, j >> 1, K);
        const T vym = L.x[c + (jm - j) * L.nx] + pl_coarse_final<D>(Cc, i >> 1, jm >> 1, K);
        const T vyp = L.x[c + (jp - j) * L.nx] + pl_coarse_final<D>(Cc, i >> 1, jp >> 1, K);
        T acc = L.b[c];
        acc = xm ? pl_fma(cxm, vxm, acc) : acc;
        acc = xp ? pl_fma(cxp, vxp, acc) : acc;
        acc = ym ? pl_fma(cym, vym, acc) : acc;
        acc = yp ? pl_fma(cyp, vyp, acc) : acc;
        if (D == 3) {
            const int s = L.nx * L.ny;
            const bool zm = k > 0, zp = k < L.nz - 1;
            const int km = zm ? k - 1 : k, kp = zp ? k + 1 : k;
            const T czm = L.cf[2][c], czp = L.cf[2][c + s];
            const T vzm = L.x[c + (km - k) * s] + pl_coarse_final<D>(Cc, i >> 1, j >> 1, km >> 1);
            const T vzp = L.x[c + (kp - k) * s] + pl_coarse_final<D>(Cc, i >> 1, j >> 1, kp >> 1);
            acc = zm ? pl_fma(czm, vzm, acc) : acc;
            acc = zp ? pl_fma(czp, vzp, acc) : acc;
        }
        L.x[c] = acc * L.idg[c];
    }
}

// coarse operator: face coefficients half the sum of the covered fine faces
// (the same rule as pressure.cu), diagonal and inverse diagonal
template <int D, typename T>
__device__ void pl_coarsen(const LevelT<T>& Fr, const LevelT<T>& Cr, int t0, int TT) {
    const LevelT<T> F = Fr, Cc = Cr;
    const int nf[3] = {F.nx, F.ny, F.nz};
    const int nc[3] = {Cc.nx, Cc.ny, Cc.nz};
    const int NC = (int)Cc.N;
    for (int C = t0; C < NC; C += TT) {
        int I, J, K;
        pl_ijk<D>(Cc, C, I, J, K);
        const int idx[3] = {I, J, K};
        T diag = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int fpos = side == 0 ? 2 * idx[d] : (idx[d] == nc[d] - 1 ? nf[d] : 2 * idx[d] + 2);
                const int a1 = (d + 1) % 3, a2 = (d + 2) % 3;
                T sum = T(0);
#pragma unroll
                for (int o1 = 0; o1 < 2; ++o1)
#pragma unroll
                    for (int o2 = 0; o2 < 2; ++o2) {
                        int fi[3];
                        fi[d] = fpos;
                        fi[a1] = 2 * idx[a1] + o1;
                        fi[a2] = 2 * idx[a2] + o2;
                        if (fi[a1] >= nf[a1] || fi[a2] >= nf[a2]) continue;
                        const int f = d == 0 ? pl_fx(F, fi[0], fi[1], fi[2])
                                             : (d == 1 ? pl_fy(F, fi[0], fi[1], fi[2])
                                                       : (fi[2] * F.ny + fi[1]) * F.nx + fi[0]);
                        sum += F.cf[d][f];
                    }
                const T v = T(0.5) * sum;
                diag += v;
                const int fc = d == 0 ? pl_fx(Cc, I, J, K) : (d == 1 ? pl_fy(Cc, I, J, K) : C);
                const int fs = d == 0 ? 1 : (d == 1 ? Cc.nx : Cc.nx * Cc.ny);
                if (side == 0) Cc.cf[d][fc] = v;
                else if (idx[d] == nc[d] - 1) Cc.cf[d][fc + fs] = v;
            }
        }
        Cc.diag[C] = diag;
        Cc.idg[C] = diag > T(0) ? T(1) / diag : T(0);
    }
}

// The coarsest level's red-black sweeps (`sweeps` each way: red-black from a
// zero start, then black-red) on one warp, for a level of at most 32
// x-pairs: lane p owns pair p, and its two cells' indices are found once and
// kept in registers over all the passes, so a pass is its loads, its
// arithmetic and a warp barrier.  The same updates as pl_red_start and
// pl_smooth with 32 threads.
template <int D, typename T>
__device__ __noinline__ void pl_coarse_warp(const LevelT<T>& Lr, int sweeps, int lane) {
    const LevelT<T> L = Lr;
    int ci[2], ii[2], jj[2], kk[2];
    bool ok[2];
#pragma unroll
    for (int colour = 0; colour < 2; ++colour)
        ok[colour] = lane < pl_npairs(L) && pl_pair_cell<D>(L, lane, colour, ii[colour], jj[colour], kk[colour],
                                                            ci[colour]);
    auto pass = [&](int colour) {
        if (ok[colour]) {
            const int c = ci[colour];
            L.x[c] = (L.b[c] + pl_offsum<D>(L, L.x, c, ii[colour], jj[colour], kk[colour])) * L.idg[c];
        }
        __syncwarp();
    };
    for (int s = 0; s < sweeps; ++s) {
        if (s == 0) {
            if (ok[0]) L.x[ci[0]] = L.b[ci[0]] * L.idg[ci[0]];
            __syncwarp();
        } else {
            pass(0);
        }
        pass(1);
    }
    for (int s = 0; s < sweeps; ++s) {
        pass(1);
        pass(0);
    }
}

// marks of the tail's progress (a trace hook; the default does nothing)
enum { PL_MARK_DOWN = 19, PL_MARK_WARP = 20, PL_MARK_UP = 21 };
struct PlNoMark {
    __device__ void operator()(int) const {}
};

// One V-cycle on levels l0..nl-1 inside one block; b of level l0 is set on
// entry, x of level l0 holds the result.  Levels of at most PL_WARP_CELLS
// cells (from the first such level down to the coarsest) run on warp 0 with
// warp barriers; the coarsest level gets `sweeps` red-black sweeps each
// way.
template <int D, typename T, class Mark = PlNoMark>
__device__ void pl_tail(const MgLevelsT<T>& M, int l0, int sweeps, Mark mark = Mark()) {
    const int t0 = threadIdx.x, TT = blockDim.x;
    const int nl = M.nl;
    int lw = nl;   // first level of the warp part (nl: none)
    if (M.lv[nl - 1].N <= PL_WARP_CELLS) {
        lw = nl - 1;
        while (lw > l0 && M.lv[lw - 1].N <= PL_WARP_CELLS) --lw;
    }
    const int lb = lw < nl - 1 ? lw : nl - 1;   // block-wide down to this level
    for (int l = l0; l < lb; ++l) {
        pl_red_start<D>(M.lv[l], t0, TT);
        __syncthreads();
        pl_smooth<D>(M.lv[l], 1, t0, TT);
        __syncthreads();
        pl_restrict<D>(M.lv[l], M.lv[l + 1], false, t0, TT);
        __syncthreads();
        mark(PL_MARK_DOWN);
    }
    if (lw < nl) {
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            for (int l = lw; l < nl - 1; ++l) {
                pl_red_start<D>(M.lv[l], lane, 32);
                __syncwarp();
                pl_smooth<D>(M.lv[l], 1, lane, 32);
                __syncwarp();
                pl_restrict<D>(M.lv[l], M.lv[l + 1], false, lane, 32);
                __syncwarp();
            }
            const LevelT<T>& Lc = M.lv[nl - 1];
            if (pl_npairs(Lc) <= 32) {
                pl_coarse_warp<D>(Lc, sweeps, lane);
            } else {
                for (int s = 0; s < sweeps; ++s) {
                    if (s == 0) pl_red_start<D>(Lc, lane, 32);
                    else pl_smooth<D>(Lc, 0, lane, 32);
                    __syncwarp();
                    pl_smooth<D>(Lc, 1, lane, 32);
                    __syncwarp();
                }
                for (int s = 0; s < sweeps; ++s) {
                    pl_smooth<D>(Lc, 1, lane, 32);
                    __syncwarp();
                    pl_smooth<D>(Lc, 0, lane, 32);
                    __syncwarp();
                }
            }
            for (int l = nl - 2; l >= lw; --l) {
                pl_prolong_black<D>(M.lv[l], M.lv[l + 1], lane, 32);
                __syncwarp();
                pl_smooth<D>(M.lv[l], 0, lane, 32);
                __syncwarp();
            }
        }
        __syncthreads();
        mark(PL_MARK_WARP);
    } else {
        const LevelT<T>& Lc = M.lv[nl - 1];
        for (int s = 0; s < sweeps; ++s) {
            if (s == 0) pl_red_start<D>(Lc, t0, TT);
            else pl_smooth<D>(Lc, 0, t0, TT);
            __syncthreads();
            pl_smooth<D>(Lc, 1, t0, TT);
            __syncthreads();
        }
        for (int s = 0; s < sweeps; ++s) {
            pl_smooth<D>(Lc, 1, t0, TT);
            __syncthreads();
            pl_smooth<D>(Lc, 0, t0, TT);
            __syncthreads();
        }
        mark(PL_MARK_WARP);
    }
    for (int l = (lw < nl ? lw : nl - 1) - 1; l >= l0; --l) {
        pl_prolong_black<D>(M.lv[l], M.lv[l + 1], t0, TT);
        __syncthreads();
        pl_smooth<D>(M.lv[l], 0, t0, TT);
        __syncthreads();
        mark(PL_MARK_UP);
    }
}

}  // namespace hf
