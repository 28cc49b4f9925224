// ib.cu -- immersed-boundary steps of the sweep (Sec. 2.3-2.5).
//
// a0 (once per lambda): cell groups ic/bc/fc, closed boundary faces, the
//    continuity mask, the compacted boundary-cell list and its geometry:
//    normal, in-solid neighbour, y_perp case and value, y_eff, interpolation
//    points X1 = P + h n, X2 = P + 2h n with bi/trilinear stencils and the
//    quadratic Lagrange weights (wS, w1, w2).
// a1 max over bc u fc of omega_old (eps_old) (Eq. imval).
// a2 u_tau (Eq. frictionvel), y+ (Eq. yplus), alpha_u = alpha_k (Eq.
//    alphauk), u_ib and k_ib (quadratic interpolation, surface k of Eq. kws),
//    omega_ib (Eq. omegaws; eps_ib = C_mu k omega_ib for k-epsilon, k = k_ib
//    in laminar-branch cells, k_P elsewhere).
//
// This file is compiled with -fmad=false: the geometry uses IEEE double
// +,-,*,/ and sqrt in a fixed order, so every integer decision (tags,
// neighbour, y_perp case, interpolation cells) is reproducible bit for bit.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"
#include "batch.cuh"

namespace hf {

// ---------------------------------------------------------------- a0: groups
__global__ void k_classify(Grid g, const double* __restrict__ lam, uint16_t* __restrict__ flags) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    double l = lam[c];
    int tag;
    if (l >= 0.5) {
        tag = TAG_IC;
    } else if (l > 0.0) {
        tag = TAG_BC;
    } else {
        bool any_ic = false;
        int kz0 = g.dims == 3 ? -1 : 0, kz1 = g.dims == 3 ? 1 : 0;
        for (int oz = kz0; oz <= kz1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    if (ox == 0 && oy == 0 && oz == 0) continue;
                    int ii = i + ox, jj = j + oy, kk = k + oz;
                    if (ii < 0 || jj < 0 || kk < 0 || ii >= g.nx || jj >= g.ny || kk >= g.nz) continue;
                    if (lam[((long long)kk * g.ny + jj) * g.nx + ii] >= 0.5) any_ic = true;
                }
        tag = any_ic ? TAG_BC : TAG_FC;
    }
    uint16_t f = (uint16_t)tag;
    if (l < 1.0) f |= F_M;
    if (tag == TAG_IC) f |= F_AU;
    // closed boundary faces: wall/slip sides where lambda > 0, inlet sides
    // where lambda >= 0.5 (walls inside the solid phase, Sec. 3.1)
    #pragma unroll
    for (int s = 0; s < 6 && s < 2 * g.dims; ++s) {
        int d = s >> 1;
        int pos = coord(d, i, j, k);
        bool on = (s & 1) ? (pos == g.n[d] - 1) : (pos == 0);
        if (!on) continue;
        int kind = g.kind[s];
        bool cl = false;
        if (kind == HFDIB_BC_WALL || kind == HFDIB_BC_SLIP) cl = l > 0.0;
        else if (kind == HFDIB_BC_INLET) cl = l >= 0.5;
        if (cl) f |= (uint16_t)(1u << (F_CLOSED_SHIFT + s));
    }
    flags[c] = f;
}

// ---------------------------------------------------------------- a0: compaction
// Ordered stream compaction of the bc cells: per-block counts, one-block
// exclusive scan, ordered scatter.  Chunk = one block of BLOCK cells.
__global__ void k_count_bc(long long N, const uint16_t* __restrict__ flags, int* __restrict__ counts) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int v = (c < N && tag_of(flags[c]) == TAG_BC) ? 1 : 0;
    int s = __syncthreads_count(v);
    if (threadIdx.x == 0) counts[blockIdx.x] = s;
}

__global__ void k_scan_counts(int nb, int* __restrict__ counts, int* __restrict__ total) {
    // single block, sequential chunks of BLOCK with a block scan each
    __shared__ int sm[BLOCK];
    int carry = 0;
    for (int base = 0; base < nb; base += BLOCK) {
        int idx = base + threadIdx.x;
        int v = idx < nb ? counts[idx] : 0;
        sm[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < BLOCK; o <<= 1) {
            int t = threadIdx.x >= o ? sm[threadIdx.x - o] : 0;
            __syncthreads();
            sm[threadIdx.x] += t;
            __syncthreads();
        }
        int incl = sm[threadIdx.x];
        if (idx < nb) counts[idx] = carry + incl - v;
        __syncthreads();
        carry += sm[BLOCK - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scatter_bc(long long N, const uint16_t* __restrict__ flags,
                             const int* __restrict__ offsets, int* __restrict__ cells) {
    __shared__ int sm[BLOCK];
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int v = (c < N && tag_of(flags[c]) == TAG_BC) ? 1 : 0;
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < BLOCK; o <<= 1) {
        int t = threadIdx.x >= o ? sm[threadIdx.x - o] : 0;
        __syncthreads();
        sm[threadIdx.x] += t;
        __syncthreads();
    }
    if (v) cells[offsets[blockIdx.x] + sm[threadIdx.x] - 1] = (int)c;
}

// ---------------------------------------------------------------- a0: geometry
__device__ inline double lam_at(const Grid& g, const double* lam, int i, int j, int k) {
    return lam[((long long)k * g.ny + j) * g.nx + i];
}

// n = -grad(lambda)/|grad(lambda)| with central differences (one-sided at the
// domain edges); if |grad lambda| < 1e-12/h, the unit vector from the vertex
// neighbour of largest lambda (ties: most shared vertices, lowest index) to P.
__device__ bool surface_normal(const Grid& g, const double* lam, int i, int j, int k, double n[3]) {
    int idx[3] = {i, j, k};
    double gr[3];
    for (int d = 0; d < 3; ++d) {
        int nd = g.n[d];
        if (nd == 1) { gr[d] = 0.0; continue; }
        int lo[3] = {i, j, k}, hi[3] = {i, j, k};
        if (idx[d] == 0) {
            hi[d] += 1;
            gr[d] = (lam_at(g, lam, hi[0], hi[1], hi[2]) - lam_at(g, lam, i, j, k)) / g.D[d];
        } else if (idx[d] == nd - 1) {
            lo[d] -= 1;
            gr[d] = (lam_at(g, lam, i, j, k) - lam_at(g, lam, lo[0], lo[1], lo[2])) / g.D[d];
        } else {
            hi[d] += 1;
            lo[d] -= 1;
            gr[d] = (lam_at(g, lam, hi[0], hi[1], hi[2]) - lam_at(g, lam, lo[0], lo[1], lo[2])) / (2.0 * g.D[d]);
        }
    }
    double mag = sqrt((gr[0] * gr[0] + gr[1] * gr[1]) + gr[2] * gr[2]);
    if (mag < 1e-12 / g.h) {
        double bl = -1.0;
        int bo[3] = {0, 0, 0}, bnz = 99;
        int kz0 = g.dims == 3 ? -1 : 0, kz1 = g.dims == 3 ? 1 : 0;
        for (int oz = kz0; oz <= kz1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    if (ox == 0 && oy == 0 && oz == 0) continue;
                    int ii = i + ox, jj = j + oy, kk = k + oz;
                    if (ii < 0 || jj < 0 || kk < 0 || ii >= g.nx || jj >= g.ny || kk >= g.nz) continue;
                    double lv = lam_at(g, lam, ii, jj, kk);
                    int nz = abs(ox) + abs(oy) + abs(oz);
                    if (bnz == 99 || lv > bl || (lv == bl && nz < bnz)) {
                        bl = lv; bo[0] = ox; bo[1] = oy; bo[2] = oz; bnz = nz;
                    }
                }
        double v0 = (double)(-bo[0]) * g.D[0], v1 = (double)(-bo[1]) * g.D[1], v2 = (double)(-bo[2]) * g.D[2];
        double nv = sqrt((v0 * v0 + v1 * v1) + v2 * v2);
        n[0] = v0 / nv; n[1] = v1 / nv; n[2] = v2 / nv;
        return true;
    }
    n[0] = -gr[0] / mag; n[1] = -gr[1] / mag; n[2] = -gr[2] / mag;
    return false;
}

__device__ inline void centre(const Grid& g, int i, int j, int k, double P[3]) {
    P[0] = g.o[0] + ((double)i + 0.5) * g.D[0];
    P[1] = g.o[1] + ((double)j + 0.5) * g.D[1];
    P[2] = g.o[2] + ((double)k + 0.5) * g.D[2];
}

__device__ inline void interp_stencil(const Grid& g, const double X[3], int base[3], double t[3]) {
    for (int d = 0; d < 3; ++d) {
        int nd = g.n[d];
        if (nd == 1) { base[d] = 0; t[d] = 0.0; continue; }
        double xi = (X[d] - g.o[d]) / g.D[d] - 0.5;
        double fl = floor(xi);
        int i0;
        if (!(fl >= 0.0)) i0 = 0;                       // also catches NaN
        else if (fl > (double)(nd - 2)) i0 = nd - 2;
        else i0 = (int)fl;
        double td = xi - (double)i0;
        if (td < 0.0) td = 0.0;
        if (td > 1.0) td = 1.0;
        base[d] = i0;
        t[d] = td;
    }
}

__global__ void k_bc_geometry(Grid g, const double* __restrict__ lam, const uint16_t* __restrict__ flags,
                              BcList bl) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= bl.nbc) return;
    long long c = bl.cell[q];
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    double P[3];
    centre(g, i, j, k, P);
    double nP[3];
    surface_normal(g, lam, i, j, k, nP);
    // in-solid neighbour: argmin over ic vertex neighbours of -n.(P - N)
    bool have = false;
    double bs = 0.0;
    int bnz = 99, bi = 0, bj = 0, bk = 0;
    int kz0 = g.dims == 3 ? -1 : 0, kz1 = g.dims == 3 ? 1 : 0;
    for (int oz = kz0; oz <= kz1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                if (ox == 0 && oy == 0 && oz == 0) continue;
                int ii = i + ox, jj = j + oy, kk = k + oz;
                if (ii < 0 || jj < 0 || kk < 0 || ii >= g.nx || jj >= g.ny || kk >= g.nz) continue;
                if (tag_of(flags[((long long)kk * g.ny + jj) * g.nx + ii]) != TAG_IC) continue;
                double s = (nP[0] * ((double)ox * g.D[0]) + nP[1] * ((double)oy * g.D[1])) +
                           nP[2] * ((double)oz * g.D[2]);
                int nz = abs(ox) + abs(oy) + abs(oz);
                if (!have || s < bs || (s == bs && nz < bnz)) {
                    have = true; bs = s; bnz = nz; bi = ii; bj = jj; bk = kk;
                }
            }
    double h = g.h;
    double lp = lam[c];
    int cas;
    double yp;
    if (lp > 0.0) {
        cas = 0;
        yp = fabs(h * atanh(1.0 - 2.0 * lp));
    } else {
        double lN = lam_at(g, lam, bi, bj, bk);
        double Nc[3];
        centre(g, bi, bj, bk, Nc);
        if (lN < 1.0) {
            cas = 1;
            double nN[3];
            surface_normal(g, lam, bi, bj, bk, nN);
            double sN = fabs(h * atanh(1.0 - 2.0 * lN));
            double Q0 = Nc[0] + sN * nN[0], Q1 = Nc[1] + sN * nN[1], Q2 = Nc[2] + sN * nN[2];
            yp = (nN[0] * (P[0] - Q0) + nN[1] * (P[1] - Q1)) + nN[2] * (P[2] - Q2);
        } else {
            cas = 2;
            double v0 = 0.5 * (P[0] + Nc[0]), v1 = 0.5 * (P[1] + Nc[1]), v2 = 0.5 * (P[2] + Nc[2]);
            double e0 = P[0] - v0, e1 = P[1] - v1, e2 = P[2] - v2;
            yp = sqrt((e0 * e0 + e1 * e1) + e2 * e2);
        }
    }
    int clamped = 0;
    if (yp < 1e-3 * h) { yp = 1e-3 * h; clamped = 1; }
    bl.nbr[q] = have ? (int)(((long long)bk * g.ny + bj) * g.nx + bi) : -1;
    bl.cas[q] = cas;
    bl.clamped[q] = clamped;
    for (int d = 0; d < 3; ++d) bl.n[3 * q + d] = nP[d];
    bl.yp[q] = yp;
    bl.ye[q] = 0.5 * (yp + 0.5 * h);
    double X1[3], X2[3];
    double h2 = 2.0 * h;
    for (int d = 0; d < 3; ++d) {
        X1[d] = P[d] + h * nP[d];
        X2[d] = P[d] + h2 * nP[d];
    }
    int b1[3], b2[3];
    double t1[3], t2[3];
    interp_stencil(g, X1, b1, t1);
    interp_stencil(g, X2, b2, t2);
    for (int d = 0; d < 3; ++d) {
        bl.b1[3 * q + d] = b1[d]; bl.t1[3 * q + d] = t1[d];
        bl.b2[3 * q + d] = b2[d]; bl.t2[3 * q + d] = t2[d];
    }
    double d1 = yp + h, d2 = yp + h2, dp = yp;
    bl.wS[q] = ((dp - d1) * (dp - d2)) / ((0.0 - d1) * (0.0 - d2));
    bl.w1[q] = ((dp - 0.0) * (dp - d2)) / ((d1 - 0.0) * (d1 - d2));
    bl.w2[q] = ((dp - 0.0) * (dp - d1)) / ((d2 - 0.0) * (d2 - d1));
}

// ---------------------------------------------------------------- a1
__device__ __forceinline__ void b_max_not_ic(Pos pos, const Grid& g, const uint16_t* __restrict__ flags,
                                             const double* __restrict__ w, double* partials, unsigned int* counter,
                                             double* out) {
    long long c = (long long)pos.bid * blockDim.x + threadIdx.x;
    double v[1] = {0.0};
    if (c < g.N && tag_of(flags[c]) != TAG_IC) v[0] = w[c];
    grid_reduce<1, true>(v, partials, counter, out, pos);
}
__global__ void k_max_not_ic(Grid g, const uint16_t* __restrict__ flags, const double* __restrict__ w,
                             double* partials, unsigned int* counter, double* out) {
    b_max_not_ic(grid_pos(), g, flags, w, partials, counter, out);
}

// ---------------------------------------------------------------- a2
__device__ inline double interp_cell(const Grid& g, const double* f, const int* b, const double* t) {
    double val = 0.0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                double w = 1.0;
                int id[3];
                int cc[3] = {cx, cy, cz};
                for (int d = 0; d < 3; ++d) {
                    if (g.n[d] == 1) {
                        if (cc[d] == 1) w = w * 0.0;
                        id[d] = b[d];
                    } else {
                        w = w * (cc[d] == 1 ? t[d] : (1.0 - t[d]));
                        id[d] = b[d] + cc[d];
                    }
                }
                val = val + w * f[((long long)id[2] * g.ny + id[1]) * g.nx + id[0]];
            }
    return val;
}

__device__ __forceinline__ void b_imposed(Pos pos, const Grid& g, int model, int freeze, const BcList& bl,
                                          uint16_t* __restrict__ flags, double* scal, const double* __restrict__ ux,
                                          const double* __restrict__ uy, const double* __restrict__ uz,
                                          const double* __restrict__ kf, double* __restrict__ uibx,
                                          double* __restrict__ uiby, double* __restrict__ uibz,
                                          double* __restrict__ kib, double* __restrict__ wib) {
    int q = pos.bid * blockDim.x + threadIdx.x;
    if (q >= bl.nbc) return;
    int c = bl.cell[q];
    const int* b1 = bl.b1 + 3 * q;
    const int* b2 = bl.b2 + 3 * q;
    const double* t1 = bl.t1 + 3 * q;
    const double* t2 = bl.t2 + 3 * q;
    double wS = bl.wS[q], w1 = bl.w1[q], w2 = bl.w2[q], ye = bl.ywf[q];
    bool turb = model != HFDIB_LAMINAR;
    double kP = turb ? kf[c] : 0.0;
    double ut = sqrt(sqrt(C_MU)) * sqrt(kP);   // C_mu^(1/4) sqrt(k)
    double yplus = ye * ut / g.nu;
    bool lamb = turb ? (yplus <= YPLUS_LAM) : true;
    int old = bl.lamb[q];
    // opt-in (not in the paper): from sweep `freeze` on a cell may leave the
    // laminar branch but not re-enter it (ends limit cycles of the switch)
    if (turb && freeze > 0 && scal[SC_NSWEEP] >= (double)freeze) lamb = lamb && (old != 0);
    bl.yplus[q] = yplus;
    bl.lamb[q] = lamb ? 1 : 0;
    // diagnostics: branch population and changes (integer-valued sums are
    // exact in any order), counted per warp and added once per warp: a
    // floating-point atomic per cell on one address serialises at L2
    {
        const unsigned int act = __activemask();
        const unsigned int nl = __popc(__ballot_sync(act, lamb));
        const unsigned int ns = __popc(__ballot_sync(act, old != (lamb ? 1 : 0)));
        if ((int)(threadIdx.x & 31) == __ffs(act) - 1) {
            if (nl) atomicAdd(scal + SC_NLAM, (double)nl);
            if (ns) atomicAdd(scal + SC_NSWITCH, (double)ns);
        }
    }
    uint16_t f = flags[c];
    f = lamb ? (uint16_t)(f | F_AU) : (uint16_t)(f & ~F_AU);
    flags[c] = f;
    const double* us[3] = {ux, uy, uz};
    double* ub[3] = {uibx, uiby, uibz};
    #pragma unroll
    for (int cpt = 0; cpt < 3 && cpt < g.dims; ++cpt) {
        double v1 = interp_cell(g, us[cpt], b1, t1);
        double v2 = interp_cell(g, us[cpt], b2, t2);
        ub[cpt][c] = lamb ? (wS * g.u_s[cpt] + w1 * v1 + w2 * v2) : 0.0;
    }
    if (turb) {
        double Cf = 1.0 / ((yplus + C_WF) * (yplus + C_WF)) + 2.0 * yplus / (C_WF * C_WF * C_WF) -
                    1.0 / (C_WF * C_WF);
        double kvis = 2400.0 * Cf / (C_EPS2 * C_EPS2);
        double kS = kvis * ut * ut;
        double v1 = interp_cell(g, kf, b1, t1);
        double v2 = interp_cell(g, kf, b2, t2);
        double kv = wS * kS + w1 * v1 + w2 * v2;
        double kimp = fmax(kv, 0.0);
        kib[c] = lamb ? kimp : 0.0;
        // Eq. omegaws with y+ = y_eff u_tau / nu substituted
        double w = lamb ? 6.0 * g.nu / (BETA1_WF * ye * ye) : ut / (KAPPA * sqrt(C_MU) * ye);
        // eps = C_mu k omega with the k the cell takes this sweep: k_ib where
        // k is imposed (laminar branch), the old k_P where k is solved
        wib[c] = eps_model(model) ? C_MU * (lamb ? kimp : kP) * w : w;
    }
}
__global__ void k_imposed(Grid g, int model, int freeze, BcList bl, uint16_t* __restrict__ flags, double* scal,
                          const double* __restrict__ ux, const double* __restrict__ uy, const double* __restrict__ uz,
                          const double* __restrict__ kf, double* __restrict__ uibx, double* __restrict__ uiby,
                          double* __restrict__ uibz, double* __restrict__ kib, double* __restrict__ wib) {
    b_imposed(grid_pos(), g, model, freeze, bl, flags, scal, ux, uy, uz, kf, uibx, uiby, uibz, kib, wib);
}

// export of the bc list for comparison with the oracle
__global__ void k_export_bc(BcList bl, long long* ints, long long* ints2, double* reals) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= bl.nbc) return;
    if (ints) {
        long long* o = ints + 8 * (long long)q;
        o[0] = bl.cell[q]; o[1] = bl.nbr[q]; o[2] = bl.cas[q]; o[3] = bl.clamped[q];
        o[4] = bl.b1[3 * q]; o[5] = bl.b1[3 * q + 1]; o[6] = bl.b1[3 * q + 2]; o[7] = bl.lamb[q];
    }
    if (ints2) {
        long long* o = ints2 + 3 * (long long)q;
        o[0] = bl.b2[3 * q]; o[1] = bl.b2[3 * q + 1]; o[2] = bl.b2[3 * q + 2];
    }
    if (reals) {
        double* r = reals + 14 * (long long)q;
        r[0] = bl.n[3 * q]; r[1] = bl.n[3 * q + 1]; r[2] = bl.n[3 * q + 2];
        r[3] = bl.yp[q]; r[4] = bl.ye[q]; r[5] = bl.wS[q]; r[6] = bl.w1[q]; r[7] = bl.w2[q];
        for (int d = 0; d < 3; ++d) { r[8 + d] = bl.t1[3 * q + d]; r[11 + d] = bl.t2[3 * q + d]; }
    }
}

// ---------------------------------------------------------------- launchers
void launch_classify(const Grid& g, const double* lam, uint16_t* flags, cudaStream_t s) {
    k_classify<<<nblocks(g.N), BLOCK, 0, s>>>(g, lam, flags);
}
void launch_compact_bc(const Grid& g, const uint16_t* flags, int* counts, int* total, int* cells,
                       cudaStream_t s) {
    unsigned int nb = nblocks(g.N);
    k_count_bc<<<nb, BLOCK, 0, s>>>(g.N, flags, counts);
    k_scan_counts<<<1, BLOCK, 0, s>>>((int)nb, counts, total);
    k_scatter_bc<<<nb, BLOCK, 0, s>>>(g.N, flags, counts, cells);
}
void launch_bc_geometry(const Grid& g, const double* lam, const uint16_t* flags, const BcList& bl,
                        cudaStream_t s) {
    if (bl.nbc == 0) return;
    k_bc_geometry<<<nblocks(bl.nbc), BLOCK, 0, s>>>(g, lam, flags, bl);
}
void launch_max_not_ic(const Grid& g, const uint16_t* flags, const double* w, double* partials,
                       unsigned int* counter, double* out, cudaStream_t s) {
    k_max_not_ic<<<nblocks(g.N), BLOCK, 0, s>>>(g, flags, w, partials, counter, out);
}
void launch_imposed(const Grid& g, int model, int freeze, const BcList& bl, uint16_t* flags, double* scal, const double* ux,
                    const double* uy, const double* uz, const double* k, double* uibx, double* uiby,
                    double* uibz, double* kib, double* wib, cudaStream_t s) {
    if (bl.nbc == 0) return;
    // one warp per block: a few thousand bc cells of a few hundred FP64
    // operations each spread over as many SMs as there are warps (full
    // blocks would leave the work to a handful of SMs' FP64 units)
    k_imposed<<<(unsigned int)((bl.nbc + 31) / 32), 32, 0, s>>>(g, model, freeze, bl, flags, scal, ux, uy, uz, k, uibx,
                                                               uiby, uibz, kib, wib);
}
void launch_export_bc(const BcList& bl, long long* ints, long long* ints2, double* reals, cudaStream_t s) {
    if (bl.nbc == 0) return;
    k_export_bc<<<nblocks(bl.nbc), BLOCK, 0, s>>>(bl, ints, ints2, reals);
}

// ---------------------------------------------------------------- batched launches
struct OpMaxNotIc {
    __device__ void operator()(Pos p, const SweepProblem& s) const {
        b_max_not_ic(p, s.g, s.F.flags, s.F.w, s.F.partials, s.F.counters + 0, s.F.scal + SC_WMAX);
    }
};
struct OpImposed {
    __device__ void operator()(Pos p, const SweepProblem& s) const {
        const Fields& F = s.F;
        b_imposed(p, s.g, s.P.model, s.freeze, s.bl, F.flags, F.scal, F.u[0], F.u[1], F.u[2], F.k, F.uib[0],
                  F.uib[1], F.uib[2], F.kib, F.wib);
    }
};
void launchb_max_not_ic(const BatchTab& T, const int* tot, cudaStream_t s) {
    k_batched<BK_CELLS, OpMaxNotIc><<<tot[BK_CELLS], BLOCK, 0, s>>>(T, OpMaxNotIc{});
}
void launchb_imposed(const BatchTab& T, const int* tot, cudaStream_t s) {
    if (tot[BK_BC] > 0) k_batched<BK_BC, OpImposed><<<tot[BK_BC], BLOCK, 0, s>>>(T, OpImposed{});
}

}  // namespace hf
