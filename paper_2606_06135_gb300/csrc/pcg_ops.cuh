// pcg_ops.cuh -- device operations of the multigrid-preconditioned CG used
// by the persistent pressure kernels (single problem and batched): level
// indexing, red-black half sweeps, restriction with the fused red start,
// prolongation fused with the black half sweep, the in-block coarse tail and
// the coarse operator.  Templated on the level precision (double / float).
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace hf {

// ---------------------------------------------------------------- level ops
template <typename T>
__device__ inline long long pl_face(const LevelT<T>& L, int d, int i, int j, int k) {
    if (d == 0) return ((long long)k * L.ny + j) * (L.nx + 1) + i;
    if (d == 1) return ((long long)k * (L.ny + 1) + j) * L.nx + i;
    return ((long long)k * L.ny + j) * L.nx + i;
}
template <typename T>
__device__ inline long long pl_fstride(const LevelT<T>& L, int d) {
    return d == 0 ? 1 : (d == 1 ? L.nx : (long long)L.nx * L.ny);
}
template <typename T>
__device__ inline void pl_ijk(const LevelT<T>& L, long long c, int& i, int& j, int& k) {
    unsigned int cc = (unsigned int)c, nx = (unsigned int)L.nx;
    unsigned int r = cc / nx;
    i = (int)(cc - r * nx);
    if (L.nz == 1) { j = (int)r; k = 0; return; }
    unsigned int ny = (unsigned int)L.ny;
    unsigned int kk = r / ny;
    j = (int)(r - kk * ny);
    k = (int)kk;
}
// Red-black passes visit the cells as x-pairs: pair p of row (j, k) holds
// cells 2p and 2p + 1, one of each colour (the last pair of an odd row has
// one cell).  A colour pass then runs half the iterations of a full pass with
// no lane of a warp skipping its cell.
template <typename T>
__device__ inline long long pl_npairs(const LevelT<T>& L) {
    return (long long)((L.nx + 1) >> 1) * L.ny * L.nz;
}
// first cell of pair p: i0 = 2 * (pair column), j, k, its linear index
template <typename T>
__device__ inline void pl_pair(const LevelT<T>& L, long long p, int& i0, int& j, int& k, long long& c0) {
    unsigned int npx = (unsigned int)((L.nx + 1) >> 1);
    unsigned int pp = (unsigned int)p;
    unsigned int r = pp / npx;
    unsigned int pi = pp - r * npx;
    if (L.nz == 1) {
        j = (int)r;
        k = 0;
    } else {
        unsigned int ny = (unsigned int)L.ny;
        unsigned int kk = r / ny;
        j = (int)(r - kk * ny);
        k = (int)kk;
    }
    i0 = 2 * (int)pi;
    c0 = ((long long)k * L.ny + j) * L.nx + i0;
}
// the cell of colour `colour` in pair p; false if the pair has none (odd rows)
template <typename T>
__device__ inline bool pl_pair_cell(const LevelT<T>& L, long long p, int colour, int& i, int& j, int& k,
                                    long long& c) {
    int i0;
    long long c0;
    pl_pair(L, p, i0, j, k, c0);
    int o = (i0 + j + k + colour) & 1;
    i = i0 + o;
    c = c0 + o;
    return i < L.nx;
}

// the loops over directions run to a fixed bound of 3 with a dims guard, so
// they unroll and the per-direction index arrays stay in registers
template <typename T, typename X>
__device__ inline T pl_offsum(const LevelT<T>& L, int dims, const X* x, long long c, int i, int j, int k) {
    T acc = T(0);
    const int idx[3] = {i, j, k};
    const int nn[3] = {L.nx, L.ny, L.nz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (d >= dims) break;
        long long fl = pl_face(L, d, i, j, k);
        long long cs = d == 0 ? 1 : (d == 1 ? L.nx : (long long)L.nx * L.ny);
        if (idx[d] > 0) acc += L.cf[d][fl] * (T)x[c - cs];
        if (idx[d] < nn[d] - 1) acc += L.cf[d][fl + pl_fstride(L, d)] * (T)x[c + cs];
    }
    return acc;
}

template <typename T>
__device__ inline void pl_smooth(const LevelT<T>& L, int dims, int colour, long long t0, long long TT) {
    const long long NP = pl_npairs(L);
    for (long long p = t0; p < NP; p += TT) {
        int i, j, k;
        long long c;
        if (!pl_pair_cell(L, p, colour, i, j, k, c)) continue;
        L.x[c] = (L.b[c] + pl_offsum(L, dims, L.x, c, i, j, k)) * L.idg[c];
    }
}

// zero-start red half sweep: x = b / diag on red cells
template <typename T>
__device__ inline void pl_red_start(const LevelT<T>& L, long long t0, long long TT) {
    const long long NP = pl_npairs(L);
    for (long long p = t0; p < NP; p += TT) {
        int i, j, k;
        long long c;
        if (!pl_pair_cell(L, p, 0, i, j, k, c)) continue;
        L.x[c] = L.b[c] * L.idg[c];
    }
}

// b_C = sum of the children's residuals; fuse_red: also the zero-start red
// half sweep of the coarse level (x_C = b_C / diag_C on red cells)
template <typename T>
__device__ inline void pl_restrict(const LevelT<T>& F, const LevelT<T>& Cc, int dims, bool fuse_red, long long t0,
                                   long long TT) {
    for (long long C = t0; C < Cc.N; C += TT) {
        int I, J, K;
        pl_ijk(Cc, C, I, J, K);
        T sum = T(0);
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
                    sum += F.b[c] - (F.diag[c] * F.x[c] - pl_offsum(F, dims, F.x, c, i, j, k));
                }
        }
        Cc.b[C] = sum;
        if (fuse_red && ((I + J + K) & 1) == 0) Cc.x[C] = sum * Cc.idg[C];
    }
}

// prolongation fused with the black half sweep (red cells are overwritten by
// the following red half sweep without being read)
template <typename T>
__device__ inline void pl_prolong_black(const LevelT<T>& L, const LevelT<T>& Cc, int dims, long long t0, long long TT) {
    const long long NP = pl_npairs(L);
    for (long long p = t0; p < NP; p += TT) {
        int i, j, k;
        long long c;
        if (!pl_pair_cell(L, p, 1, i, j, k, c)) continue;
        const int idx[3] = {i, j, k};
        const int nn[3] = {L.nx, L.ny, L.nz};
        T acc = L.b[c];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d >= dims) break;
            long long fl = pl_face(L, d, i, j, k);
            long long cs = d == 0 ? 1 : (d == 1 ? L.nx : (long long)L.nx * L.ny);
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                if (side == 0 && idx[d] == 0) continue;
                if (side == 1 && idx[d] == nn[d] - 1) continue;
                int ni[3] = {i, j, k};
                ni[d] += side ? 1 : -1;
                long long nc = side ? c + cs : c - cs;
                long long C = ((long long)(ni[2] >> 1) * Cc.ny + (ni[1] >> 1)) * Cc.nx + (ni[0] >> 1);
                acc += L.cf[d][fl + (side ? pl_fstride(L, d) : 0)] * (L.x[nc] + Cc.x[C]);
            }
        }
        L.x[c] = acc * L.idg[c];
    }
}

// levels l0..nl-1 inside one block: b of level l0 is set on entry
template <typename T>
__device__ void pl_tail(const MgLevelsT<T>& M, int dims, int l0, int sweeps) {
    const long long t0 = threadIdx.x, TT = blockDim.x;
    for (int l = l0; l < M.nl - 1; ++l) {
        const LevelT<T>& L = M.lv[l];
        pl_red_start(L, t0, TT);
        __syncthreads();
        pl_smooth(L, dims, 1, t0, TT);
        __syncthreads();
        pl_restrict(L, M.lv[l + 1], dims, false, t0, TT);
        __syncthreads();
    }
    const LevelT<T>& Lc = M.lv[M.nl - 1];
    for (int s = 0; s < sweeps; ++s) {
        if (s == 0) {
            pl_red_start(Lc, t0, TT);
        } else {
            pl_smooth(Lc, dims, 0, t0, TT);
        }
        __syncthreads();
        pl_smooth(Lc, dims, 1, t0, TT);
        __syncthreads();
    }
    for (int s = 0; s < sweeps; ++s) {
        pl_smooth(Lc, dims, 1, t0, TT);
        __syncthreads();
        pl_smooth(Lc, dims, 0, t0, TT);
        __syncthreads();
    }
    for (int l = M.nl - 2; l >= l0; --l) {
        const LevelT<T>& L = M.lv[l];
        pl_prolong_black(L, M.lv[l + 1], dims, t0, TT);
        __syncthreads();
        pl_smooth(L, dims, 0, t0, TT);
        __syncthreads();
    }
}

// coarse operator: face coefficients half the sum of the covered fine faces
// (same rule as pressure.cu), diagonal and inverse diagonal
template <typename T>
__device__ inline void pl_coarsen(const LevelT<T>& F, const LevelT<T>& Cc, int dims, long long t0, long long TT) {
    const int nf[3] = {F.nx, F.ny, F.nz};
    const int nc[3] = {Cc.nx, Cc.ny, Cc.nz};
    for (long long C = t0; C < Cc.N; C += TT) {
        int I, J, K;
        pl_ijk(Cc, C, I, J, K);
        const int idx[3] = {I, J, K};
        T diag = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d >= dims) break;
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                int fpos = side == 0 ? 2 * idx[d] : (idx[d] == nc[d] - 1 ? nf[d] : 2 * idx[d] + 2);
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
                        sum += F.cf[d][pl_face(F, d, fi[0], fi[1], fi[2])];
                    }
                T v = T(0.5) * sum;
                diag += v;
                if (side == 0) Cc.cf[d][pl_face(Cc, d, I, J, K)] = v;
                else if (idx[d] == nc[d] - 1) Cc.cf[d][pl_face(Cc, d, I, J, K) + pl_fstride(Cc, d)] = v;
            }
        }
        Cc.diag[C] = diag;
        Cc.idg[C] = diag > T(0) ? T(1) / diag : T(0);
    }
}

}  // namespace hf
