// flow.cu -- momentum predictor, pressure corrector and velocity update of
// the extended SIMPLE sweep (Sec. 2.5.1, Fig. simplehfdibrans), FP64.
//
// Rows are matrix-free: every kernel rebuilds the coefficients of a cell from
// the face fluxes phi and nu_eff = nu + nu_t, so the only stored per-cell
// operator data are right-hand sides.  Discretisation (Sec. 3.1 "Numerical
// schemes"): upwind convection in bounded form, central diffusion with the
// arithmetic mean of the face diffusivity, Gauss-linear gradients, explicit
// div(nu_eff (grad u)^T), implicit under-relaxation of the momentum rows;
// the schemes of App. B as a deferred correction of the convection.
//
// Also here, as post-processing of a state: the force of the fluid on the
// body (Eqs. dragcoeff, dlcoeffs), the wall shear along a domain wall and the
// recirculation region behind a body (Sec. 3.3, 3.6).
#include "common.cuh"
#include "kernels.cuh"
#include "batch.cuh"

namespace hf {

__device__ inline long long nbr_cell(const Grid& g, long long c, int d, int side) {
    return side ? c + g.stride[d] : c - g.stride[d];
}
__device__ inline bool interior(const Grid& g, int d, int side, int i, int j, int k) {
    int pos = coord(d, i, j, k);
    return side ? pos < g.n[d] - 1 : pos > 0;
}

// fixed value of velocity component cpt imposed by the row of cell c (if any)
__device__ inline bool vel_row_fixed(const Grid& g, const Fields& F, long long c, int cpt, double& v) {
    uint16_t f = F.flags[c];
    if (tag_of(f) == TAG_IC) { v = g.u_s[cpt]; return true; }
    if (f & F_AU) { v = F.uib[cpt][c]; return true; }
    return false;
}

// momentum row of cell c (unrelaxed): aP per component, neighbour
// coefficients and the boundary right-hand side per component.  T = double
// for the FP64 operator, float for the FP32 smoother of the mixed path
// (from FP32 mirrors of phi and nu_t).
template <typename T>
struct MomRowT {
    T aP[3];
    T a[6];
    long long nb[6];
    bool has[6];
    T bnd[3];
};
using MomRow = MomRowT<double>;

template <typename T>
__device__ void mom_row_t(const Grid& g, T* const* phi, const T* nut, long long c, int i, int j, int k, uint16_t f,
                          MomRowT<T>& R) {
    const T nu = (T)g.nu;
    T nuP = nu + nut[c];
    for (int q = 0; q < 3; ++q) { R.aP[q] = T(0); R.bnd[q] = T(0); }
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        long long fl = face_lo(g, d, i, j, k);
        long long fs = face_stride(g, d);
        for (int side = 0; side < 2; ++side) {
            int s = 2 * d + side;
            T Fb = phi[d][fl + side * fs];
            T Fout = side ? Fb : -Fb;
            if (interior(g, d, side, i, j, k)) {
                long long nc = nbr_cell(g, c, d, side);
                T nuN = nu + nut[nc];
                T Dif = T(0.5) * (nuP + nuN) * (T)g.SoD[d];
                R.a[s] = fmin(Fout, T(0)) - Dif;
                R.nb[s] = nc;
                R.has[s] = true;
                T add = fmax(-Fout, T(0)) + Dif;
                #pragma unroll
                for (int q = 0; q < 3 && q < g.dims; ++q) R.aP[q] += add;
            } else {
                R.a[s] = T(0);
                R.nb[s] = c;
                R.has[s] = false;
                #pragma unroll
                for (int q = 0; q < 3 && q < g.dims; ++q) {
                    double val;
                    if (vel_fixed(g, f, s, q, val)) {
                        T coef = nuP * (T)g.SoHD[d] + fmax(-Fout, T(0));
                        R.aP[q] += coef;
                        R.bnd[q] += coef * (T)val;
                    }
                }
            }
        }
    }
}

__device__ inline void mom_row(const Grid& g, const Fields& F, long long c, int i, int j, int k, uint16_t f,
                               MomRow& R) {
    mom_row_t<double>(g, F.phi, F.nut, c, i, j, k, f, R);
}


// Gauss-linear gradient of the pressure-like field p at cell c (outlet faces
// carry p_out, the rest zero gradient)
__device__ inline double grad_p(const Grid& g, const double* p, long long c, int d, int i, int j, int k) {
    // between two interior faces (hi - lo) / Delta = (p_N - p_S) / (2 Delta):
    // two FP64 operations instead of six
    if (interior(g, d, 0, i, j, k) && interior(g, d, 1, i, j, k))
        return (p[c + g.stride[d]] - p[c - g.stride[d]]) * (0.5 * g.iD[d]);
    double pP = p[c];
    double lo, hi;
    if (interior(g, d, 0, i, j, k)) lo = 0.5 * (p[c - g.stride[d]] + pP);
    else lo = p_fixed(g, 2 * d) ? g.p_out : pP;
    if (interior(g, d, 1, i, j, k)) hi = 0.5 * (pP + p[c + g.stride[d]]);
    else hi = p_fixed(g, 2 * d + 1) ? g.p_out : pP;
    return (hi - lo) * g.iD[d];
}

// relaxed pressure p + a (pn - p), evaluated on the fly
__device__ inline double prelax(const double* p, const double* pn, long long c, double a) {
    double po = p[c];
    return po + a * (pn[c] - po);
}

// ---------------------------------------------------------------- initial flux
// phi of the current velocity: linear interpolation inside, inlet u_in S,
// outlet u_P S, zero on walls, slip and closed faces.
__device__ inline double bnd_flux_hbya(const Grid& g, uint16_t f, int s, double vP) {
    if (closed_side(f, s)) return 0.0;
    int d = s >> 1;
    int kind = g.kind[s];
    if (kind == HFDIB_BC_INLET) return g.u_in[d] * g.S[d];
    if (kind == HFDIB_BC_OUTLET) return vP * g.S[d];
    return 0.0;
}

__global__ void k_face_flux(Grid g, const uint16_t* __restrict__ flags, const double* vx, const double* vy,
                            const double* vz, double* fx, double* fy, double* fz) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    uint16_t f = flags[c];
    const double* v[3] = {vx, vy, vz};
    double* out[3] = {fx, fy, fz};
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        long long fl = face_lo(g, d, i, j, k);
        if (interior(g, d, 0, i, j, k))
            out[d][fl] = 0.5 * (v[d][c - g.stride[d]] + v[d][c]) * g.S[d];
        else
            out[d][fl] = bnd_flux_hbya(g, f, 2 * d, v[d][c]);
        if (!interior(g, d, 1, i, j, k))
            out[d][fl + face_stride(g, d)] = bnd_flux_hbya(g, f, 2 * d + 1, v[d][c]);
    }
}

// ---------------------------------------------------------------- means
// Sums of the fields the residual normalisation needs, with imposed rows
// replaced by their imposed values.
__device__ __forceinline__ void b_means(Pos pos, const Grid& g, const Params& P, const Fields& F) {
    double v[6] = {0, 0, 0, 0, 0, 0};
    // (unrolled: the loads of four cells in flight per thread on the
    // two-blocks-per-SM reduction grid)
    #pragma unroll 4
    for (long long c = (long long)pos.bid * blockDim.x + threadIdx.x; c < g.N;
         c += (long long)pos.nblk * blockDim.x) {
        uint16_t f = F.flags[c];
        int tag = tag_of(f);
        #pragma unroll
        for (int q = 0; q < 3 && q < g.dims; ++q) {
            double x;
            if (!vel_row_fixed(g, F, c, q, x)) x = F.u[q][c];
            v[q] += x;
        }
        v[3] += F.p[c];
        if (P.model != HFDIB_LAMINAR) {
            v[4] += tag == TAG_IC ? 0.0 : ((f & F_AU) ? F.kib[c] : F.k[c]);
            v[5] += tag == TAG_IC ? F.scal[SC_WMAX] : (tag == TAG_BC ? F.wib[c] : F.w[c]);
        }
    }
    grid_reduce<6, false>(v, F.partials, F.counters + 1, F.scal + SC_SUM_U, pos);
}
__global__ void k_means(Grid g, Params P, Fields F) {
    b_means(grid_pos(), g, P, F);
}

// ---------------------------------------------------------------- grad u
__device__ __forceinline__ void b_grad_u(Pos pos, const Grid& g, const Fields& F) {
    long long c = (long long)pos.bid * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    uint16_t f = F.flags[c];
    // between two interior faces (hi - lo) / D = (u_N - u_S) / (2 D): two FP64
    // operations instead of six (FP64 issue is this kernel's bound)
    double hiD[3];
    #pragma unroll
    for (int a = 0; a < 3 && a < g.dims; ++a) hiD[a] = 0.5 * g.iD[a];
    #pragma unroll
    for (int b = 0; b < 3 && b < g.dims; ++b) {
        const double* u = F.u[b];
        double uP = u[c];
        #pragma unroll
        for (int a = 0; a < 3 && a < g.dims; ++a) {
            const bool in_lo = interior(g, a, 0, i, j, k), in_hi = interior(g, a, 1, i, j, k);
            double G;
            if (in_lo && in_hi) {
                G = (u[c + g.stride[a]] - u[c - g.stride[a]]) * hiD[a];
            } else {
                double lo, hi, val;
                if (in_lo) lo = 0.5 * (u[c - g.stride[a]] + uP);
                else lo = vel_fixed(g, f, 2 * a, b, val) ? val : uP;
                if (in_hi) hi = 0.5 * (uP + u[c + g.stride[a]]);
                else hi = vel_fixed(g, f, 2 * a + 1, b, val) ? val : uP;
                G = (hi - lo) * g.iD[a];
            }
            F.G[(long long)(3 * a + b) * g.N + c] = G;
        }
    }
}
__global__ void k_grad_u(Grid g, Fields F) {
    b_grad_u(grid_pos(), g, F);
}

// explicit div(nu_eff (grad u)^T) of cell c, component q: face flux
// nu_f (d u_a/d x_q)_f S_a through the a-faces (cell values on boundary faces)
__device__ __forceinline__ double transpose_src(const Grid& g, const Fields& F, long long c, int i, int j, int k,
                                                int q, double nuP) {
    double T = 0.0;
    #pragma unroll
    for (int a = 0; a < 3 && a < g.dims; ++a) {
        const double* Gq = F.G + (long long)(3 * q + a) * g.N;
        double GP = Gq[c];
        double flo, fhi;
        if (interior(g, a, 0, i, j, k)) {
            long long nc = c - g.stride[a];
            flo = (0.5 * (nuP + g.nu + F.nut[nc])) * (0.5 * (GP + Gq[nc])) * g.S[a];
        } else {
            flo = nuP * GP * g.S[a];
        }
        if (interior(g, a, 1, i, j, k)) {
            long long nc = c + g.stride[a];
            fhi = (0.5 * (nuP + g.nu + F.nut[nc])) * (0.5 * (GP + Gq[nc])) * g.S[a];
        } else {
            fhi = nuP * GP * g.S[a];
        }
        T += fhi - flo;
    }
    return T;
}

// Deferred correction of the momentum convection (App. B schemes): the rows
// keep bounded upwind, and -sum over interior faces of F_out (u_f - u_U)
// goes to the right-hand side, from u and grad u at sweep start.  U is the
// upwind cell of the face, D the other, s = +1 when D lies at +d from U.
//   linearUpwind: u_f - u_U = s (Delta/2) du/dx_d|U (scheme 3: times the
//                 upwind cell's Barth-Jespersen limiter)
//   vanLeer:      u_f - u_U = psi(r) (u_D - u_U)/2, psi = (r + |r|)/(1 + |r|),
//                 r = 2 s Delta du/dx_d|U / (u_D - u_U) - 1 (no term where u_D = u_U)
// Barth-Jespersen limiter of cell U for component q (scheme 3): the largest
// l <= 1 keeping u_U + l (+-Delta_d/2) du/dx_d|U within the min/max of u over
// U and its interior neighbours
__device__ inline double conv_limiter(const Grid& g, const Fields& F, long long U, int iU, int jU, int kU, int q) {
    const double* u = F.u[q];
    const double uU = u[U];
    double umax = uU, umin = uU;
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        #pragma unroll
        for (int side = 0; side < 2; ++side) {
            if (!interior(g, d, side, iU, jU, kU)) continue;
            double v = u[nbr_cell(g, U, d, side)];
            umax = fmax(umax, v);
            umin = fmin(umin, v);
        }
    }
    double l = 1.0;
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        const double gd = F.G[(long long)(3 * d + q) * g.N + U];
        #pragma unroll
        for (int side = 0; side < 2; ++side) {
            double delta = (side ? -0.5 : 0.5) * g.D[d] * gd;
            if (delta > 0.0) l = fmin(l, (umax - uU) / delta);
            else if (delta < 0.0) l = fmin(l, (umin - uU) / delta);
        }
    }
    return l;
}

// scheme 3: the cell-limited velocity gradient, Glim = l G per component
__device__ __forceinline__ void b_conv_limit(Pos pos, const Grid& g, const Fields& F) {
    long long c = (long long)pos.bid * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    #pragma unroll
    for (int q = 0; q < 3 && q < g.dims; ++q) {
        double l = conv_limiter(g, F, c, i, j, k, q);
        #pragma unroll
        for (int d = 0; d < 3 && d < g.dims; ++d) {
            long long e = (long long)(3 * d + q) * g.N + c;
            F.Glim[e] = l * F.G[e];
        }
    }
}
__global__ void k_conv_limit(Grid g, Fields F) {
    b_conv_limit(grid_pos(), g, F);
}

__device__ inline double conv_src(const Grid& g, const Fields& F, long long c, int i, int j, int k, int q) {
    double corr = 0.0;
    const double* u = F.u[q];
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        long long fl = face_lo(g, d, i, j, k);
        long long fs = face_stride(g, d);
        // d u_q / d x_d (scheme 3: the limited copy written by k_conv_limit)
        const double* Gd = (g.conv == 3 ? F.Glim : F.G) + (long long)(3 * d + q) * g.N;
        #pragma unroll
        for (int side = 0; side < 2; ++side) {
            if (!interior(g, d, side, i, j, k)) continue;
            double Fb = F.phi[d][fl + side * fs];
            double Fout = side ? Fb : -Fb;
            long long n = nbr_cell(g, c, d, side);
            bool out = Fout >= 0.0;
            long long U = out ? c : n;
            double s = (out == (side == 1)) ? 1.0 : -1.0;
            double gU = Gd[U];
            double du;
            if (g.conv != 2) {
                du = s * (0.5 * g.D[d]) * gU;
            } else {
                double uU = u[U], uD = u[out ? n : c];
                double dd = uD - uU;
                if (dd != 0.0) {
                    double r = 2.0 * (s * g.D[d]) * gU / dd - 1.0;
                    double psi = (r + fabs(r)) / (1.0 + fabs(r));
                    du = 0.5 * psi * dd;
                } else {
                    du = 0.0;
                }
            }
            corr += Fout * du;
        }
    }
    return -corr;
}

// ---------------------------------------------------------------- a3 assembly
// The viscosity of each interior face, nu_f = (nu_eff,P + nu_eff,N)/2, is
// formed once and serves the row of every component and the explicit
// transpose term: FP64 arithmetic is the limit of this kernel on GB300.
__device__ __forceinline__ void b_mom_asm(Pos pos, const Grid& g, const Params& P, const Fields& F) {
    double red[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const long long N = g.N;
    // loop-invariant factors: (S/Delta)/2 and S/4 per direction, the means
    double hSoD[3], qS[3], hS[3], xbar[3];
    #pragma unroll
    for (int d = 0; d < 3; ++d) {
        hSoD[d] = 0.5 * g.SoD[d];
        qS[d] = 0.25 * g.S[d];
        hS[d] = 0.5 * g.S[d];
        xbar[d] = d < g.dims ? F.scal[SC_SUM_U + d] * g.iN : 0.0;
    }
    for (long long c = (long long)pos.bid * blockDim.x + threadIdx.x; c < N;
         c += (long long)pos.nblk * blockDim.x) {
        int i, j, k;
        cell_ijk(g, c, i, j, k);
        const uint16_t f = F.flags[c];
        const double nuP = g.nu + F.nut[c];
        const int idx[3] = {i, j, k};
        // faces s = 2d + side: neighbour, row coefficient, outflow, transpose
        // weight nu_f S/2 (a boundary face: nu_P S/2 with the cell itself as
        // the neighbour, so that w (G_P + G_N) is the flux nu_P G_P S of the
        // cell value)
        double a[6], fo[6], w[6];
        long long nb[6];
        bool has[6];
        double aPi = 0.0;   // the interior-face part of aP (= -sum a_N), common to the components
        #pragma unroll
        for (int s = 0; s < 6; ++s) {
            const int d = s >> 1, side = s & 1;
            has[s] = false;
            a[s] = 0.0;
            w[s] = 0.0;
            fo[s] = 0.0;
            nb[s] = c;
            if (d >= g.dims) continue;
            const double Fb = F.phi[d][face_lo(g, d, i, j, k) + (side ? face_stride(g, d) : 0)];
            fo[s] = side ? Fb : -Fb;
            w[s] = hS[d] * nuP;
            if (!(side ? idx[d] < g.n[d] - 1 : idx[d] > 0)) continue;
            const long long nc = side ? c + g.stride[d] : c - g.stride[d];
            // nu_f = (nu_eff,P + nu_eff,N)/2 folded into the factors
            const double nus = nuP + (g.nu + F.nut[nc]);
            const double Dif = nus * hSoD[d];
            has[s] = true;
            nb[s] = nc;
            a[s] = fmin(fo[s], 0.0) - Dif;
            aPi -= a[s];
            w[s] = qS[d] * nus;
        }
        // w_hi - w_lo per direction (the transpose term's weight of G_P)
        double dw[3];
        #pragma unroll
        for (int d = 0; d < 3; ++d) dw[d] = w[2 * d + 1] - w[2 * d];
        // keep the row for the smoother (FP64 path) and HbyA (same phi and nu_t later in the sweep)
        #pragma unroll
        for (int s = 0; s < 6 && s < 2 * g.dims; ++s) F.mrow[(long long)(3 + s) * N + c] = a[s];
        const bool fixed_row = (tag_of(f) == TAG_IC) || (f & F_AU);
        #pragma unroll
        for (int q = 0; q < 3 && q < g.dims; ++q) {
            // boundary faces carrying a fixed value of component q
            double aP = aPi, bnd = 0.0;
            #pragma unroll
            for (int s = 0; s < 6 && s < 2 * g.dims; ++s) {
                double val;
                if (!has[s] && vel_fixed(g, f, s, q, val)) {
                    const double coef = nuP * g.SoHD[s >> 1] + fmax(-fo[s], 0.0);
                    aP += coef;
                    bnd += coef * val;
                }
            }
            F.mrow[(long long)q * N + c] = aP;
            // explicit div(nu_eff (grad u)^T): face flux nu_f (d u_a/d x_q)_f S_a
            // through the a-faces (the cell's values on boundary faces):
            // w_hi (G_P + G_hi) - w_lo (G_P + G_lo), three FMAs per direction
            double T = 0.0;
            #pragma unroll
            for (int ad = 0; ad < 3 && ad < g.dims; ++ad) {
                const double* Gq = F.G + (long long)(3 * q + ad) * N;
                const double GP = Gq[c];
                T = fma(-w[2 * ad], Gq[nb[2 * ad]], T);
                T = fma(w[2 * ad + 1], Gq[nb[2 * ad + 1]], T);
                T = fma(dw[ad], GP, T);
            }
            double b0 = bnd + T;
            if (g.conv) b0 += conv_src(g, F, c, i, j, k, q);
            const double gp = grad_p(g, F.p, c, q, i, j, k);
            const double uold = F.u[q][c];
            const double bfull = b0 - gp * g.V;
            F.bm[q][c] = b0 + P.rlx_u * aP * uold - gp * g.V;
            // initial guess of the predictor: u_old, with the imposed rows
            // already at their imposed values (so an exact solution of the
            // sweep's system is left unchanged by the smoother)
            double fv;
            F.us[q][c] = vel_row_fixed(g, F, c, q, fv) ? fv : uold;
            if (!fixed_row) {
                double Ax = aP * uold;
                #pragma unroll
                for (int s = 0; s < 6 && s < 2 * g.dims; ++s) {
                    if (!has[s]) continue;
                    double xN;
                    if (!vel_row_fixed(g, F, nb[s], q, xN)) xN = F.u[q][nb[s]];
                    Ax += a[s] * xN;
                }
                // row sum: the boundary part of aP (the interior part cancels
                // the neighbour coefficients)
                const double A1 = aP - aPi;
                red[3 * q + 0] += fabs(bfull - Ax);
                red[3 * q + 1] += fabs(Ax - A1 * xbar[q]);
                red[3 * q + 2] += fabs(bfull - A1 * xbar[q]);
                // defect of the relaxed system at the initial guess: with
                // x_P = u_old the relaxation terms cancel, leaving b - A x
                if (F.mixed) F.r32[q][c] = (float)(bfull - Ax);
            } else if (F.mixed) {
                F.r32[q][c] = 0.0f;
            }
        }
    }
    grid_reduce<9, false>(red, F.partials, F.counters + 2, F.scal + SC_RES_U, pos);
}
__global__ void __launch_bounds__(BLOCK, 2) k_mom_asm(Grid g, Params P, Fields F) {
    b_mom_asm(grid_pos(), g, P, F);
}

// ---------------------------------------------------------------- a4 smoother
// Red-black Gauss-Seidel on the relaxed momentum rows; rows with alpha_u = 1
// hold u = u_ib (ic: u_s), which realises the correction of Eq. (corru).
__device__ __forceinline__ void b_mom_smooth(Pos pos, const Grid& g, const Params& P, const Fields& F, int colour) {
    long long p = (long long)pos.bid * blockDim.x + threadIdx.x;
    if (p >= npairs(g)) return;
    long long c;
    int i, j, k;
    if (!pair_cell(g, p, colour, c, i, j, k)) return;
    uint16_t f = F.flags[c];
    if (tag_of(f) == TAG_IC) {
        #pragma unroll
        for (int q = 0; q < 3 && q < g.dims; ++q) F.us[q][c] = g.u_s[q];
        return;
    }
    if (f & F_AU) {
        #pragma unroll
        for (int q = 0; q < 3 && q < g.dims; ++q) F.us[q][c] = F.uib[q][c];
        return;
    }
    // the row of this sweep, kept by the assembly (k_mom_asm)
    const long long N = g.N;
    const int idx[3] = {i, j, k};
    #pragma unroll
    for (int q = 0; q < 3 && q < g.dims; ++q) {
        double acc = F.bm[q][c];
        #pragma unroll
        for (int s = 0; s < 6 && s < 2 * g.dims; ++s) {
            const int d = s >> 1, side = s & 1;
            if (!(side ? idx[d] < g.n[d] - 1 : idx[d] > 0)) continue;
            acc -= F.mrow[(long long)(3 + s) * N + c] * F.us[q][side ? c + g.stride[d] : c - g.stride[d]];
        }
        F.us[q][c] = acc * P.urf_u / F.mrow[(long long)q * N + c];
    }
}
__global__ void k_mom_smooth(Grid g, Params P, Fields F, int colour) {
    b_mom_smooth(grid_pos(), g, P, F, colour);
}

// FP32 red-black sweep on the correction of the predictor (mixed path):
// (aP/urf) d_P + sum a_N d_N = r (FP64 defect rounded), d = 0 on imposed rows.
// zero_init: the other colour is taken as 0 (first half sweep).
__device__ __forceinline__ void b_mom_smooth32(Pos pos, const Grid& g, const Params& P, const Fields& F, int colour,
                                               int zero_init, int finalize) {
    long long p = (long long)pos.bid * blockDim.x + threadIdx.x;
    if (p >= npairs(g)) return;
    long long c;
    int i, j, k;
    if (!pair_cell(g, p, colour, c, i, j, k)) return;
    uint16_t f = F.flags[c];
    if (tag_of(f) == TAG_IC || (f & F_AU)) {
        #pragma unroll
        for (int q = 0; q < 3 && q < g.dims; ++q) F.d32[q][c] = 0.0f;
        return;
    }
    MomRowT<float> R;
    mom_row_t<float>(g, F.phi32, F.nut32, c, i, j, k, f, R);
    const float urf = (float)P.urf_u;
    #pragma unroll
    for (int q = 0; q < 3 && q < g.dims; ++q) {
        float acc = F.r32[q][c];
        if (!zero_init)
            #pragma unroll
            for (int s = 0; s < 6 && s < 2 * g.dims; ++s)
                if (R.has[s]) acc -= R.a[s] * F.d32[q][R.nb[s]];
        const float dq = acc * urf / R.aP[q];
        F.d32[q][c] = dq;
        // the last pass of this colour: u* = initial guess + correction, in FP64
        if (finalize) F.us[q][c] += (double)dq;
    }
}
// six resident blocks per SM (40 registers): the half sweeps are bound by
// the latency of their global loads, so more warps in flight pay
__global__ void __launch_bounds__(BLOCK, 6) k_mom_smooth32(Grid g, Params P, Fields F, int colour, int zero_init, int finalize) {
    b_mom_smooth32(grid_pos(), g, P, F, colour, zero_init, finalize);
}

// ---------------------------------------------------------------- a6 HbyA
__device__ __forceinline__ void b_hbya(Pos pos, const Grid& g, const Params& P, const Fields& F) {
    long long c = (long long)pos.bid * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const long long N = g.N;
    // the row of this sweep, kept by the assembly (k_mom_asm)
    double aavg = 0.0;
    double aPr[3];
    #pragma unroll
    for (int q = 0; q < 3 && q < g.dims; ++q) { aPr[q] = F.mrow[(long long)q * N + c] * P.iurf_u; aavg += aPr[q]; }
    aavg = aavg * (g.dims == 2 ? 0.5 : (1.0 / 3.0));
    double ia = 1.0 / aavg;
    #pragma unroll
    for (int q = 0; q < 3 && q < g.dims; ++q) {
        double br = F.bm[q][c] + grad_p(g, F.p, c, q, i, j, k) * g.V;
        double off = 0.0;
        #pragma unroll
        for (int s = 0; s < 6 && s < 2 * g.dims; ++s) {
            int d = s >> 1, side = s & 1;
            if (!interior(g, d, side, i, j, k)) continue;
            long long nb = side ? c + g.stride[d] : c - g.stride[d];
            off += F.mrow[(long long)(3 + s) * N + c] * F.us[q][nb];
        }
        double H = br - off - (aPr[q] - aavg) * F.us[q][c];
        F.HbyA[q][c] = H * ia;
    }
    F.rAU[c] = g.V * ia;
}
__global__ void k_hbya(Grid g, Params P, Fields F) {
    b_hbya(grid_pos(), g, P, F);
}

// ---------------------------------------------------------------- phiHbyA
__device__ __forceinline__ void b_phiH(Pos pos, const Grid& g, const Fields& F) {
    long long c = (long long)pos.bid * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    uint16_t f = F.flags[c];
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        long long fl = face_lo(g, d, i, j, k);
        const double* H = F.HbyA[d];
        if (interior(g, d, 0, i, j, k))
            F.phiH[d][fl] = 0.5 * (H[c - g.stride[d]] + H[c]) * g.S[d];
        else
            F.phiH[d][fl] = bnd_flux_hbya(g, f, 2 * d, H[c]);
        if (!interior(g, d, 1, i, j, k))
            F.phiH[d][fl + face_stride(g, d)] = bnd_flux_hbya(g, f, 2 * d + 1, H[c]);
    }
}
__global__ void k_phiH(Grid g, Fields F) {
    b_phiH(grid_pos(), g, F);
}

// ---------------------------------------------------------------- a8 update
// phi = phiHbyA - rAU_f (p_N - p_P)/Delta S with the new (unrelaxed) pressure;
// p <- p + urf_p (p_new - p); u = HbyA - rAU grad(p_relaxed); continuity error.
__device__ __forceinline__ void b_update(Pos pos, const Grid& g, const Params& P, const Fields& F, const Level& L0) {
    double red[1] = {0.0};
    for (long long c = (long long)pos.bid * blockDim.x + threadIdx.x; c < g.N;
         c += (long long)pos.nblk * blockDim.x) {
        int i, j, k;
        cell_ijk(g, c, i, j, k);
        uint16_t f = F.flags[c];
        double pnP = F.pn[c];
        double div = 0.0;
        #pragma unroll
        for (int d = 0; d < 3 && d < g.dims; ++d) {
            long long fl = face_lo(g, d, i, j, k);
            long long fs = face_stride(g, d);
            double flo, fhi;
            // L0.cf holds rAU_f S/Delta (inside) and rAU_P S/(Delta/2) (outlet)
            if (interior(g, d, 0, i, j, k)) {
                long long nc = c - g.stride[d];
                flo = F.phiH[d][fl] - L0.cf[d][fl] * (pnP - F.pn[nc]);
            } else if (p_fixed(g, 2 * d)) {
                flo = F.phiH[d][fl] - L0.cf[d][fl] * (pnP - g.p_out);
            } else {
                flo = F.phiH[d][fl];
            }
            if (interior(g, d, 1, i, j, k)) {
                long long nc = c + g.stride[d];
                fhi = F.phiH[d][fl + fs] - L0.cf[d][fl + fs] * (F.pn[nc] - pnP);
            } else if (p_fixed(g, 2 * d + 1)) {
                fhi = F.phiH[d][fl + fs] - L0.cf[d][fl + fs] * (g.p_out - pnP);
            } else {
                fhi = F.phiH[d][fl + fs];
            }
            F.phi[d][fl] = flo;
            if (!interior(g, d, 1, i, j, k)) F.phi[d][fl + fs] = fhi;
            if (F.mixed) {
                F.phi32[d][fl] = (float)flo;
                if (!interior(g, d, 1, i, j, k)) F.phi32[d][fl + fs] = (float)fhi;
            }
            div += fhi - flo;
        }
        red[0] += fabs(masked_div(g, F.lam, f, c, div));
        // relaxed pressure and the velocity update
        double a = P.urf_p;
        double prP = prelax(F.p, F.pn, c, a);
        #pragma unroll
        for (int d = 0; d < 3 && d < g.dims; ++d) {
            const bool in_lo = interior(g, d, 0, i, j, k), in_hi = interior(g, d, 1, i, j, k);
            double gp;
            if (in_lo && in_hi) {
                // (p_N - p_S) / (2 Delta) of the relaxed pressure
                gp = (prelax(F.p, F.pn, c + g.stride[d], a) - prelax(F.p, F.pn, c - g.stride[d], a)) *
                     (0.5 * g.iD[d]);
            } else {
                double lo, hi;
                if (in_lo) lo = 0.5 * (prelax(F.p, F.pn, c - g.stride[d], a) + prP);
                else lo = p_fixed(g, 2 * d) ? g.p_out : prP;
                if (in_hi) hi = 0.5 * (prP + prelax(F.p, F.pn, c + g.stride[d], a));
                else hi = p_fixed(g, 2 * d + 1) ? g.p_out : prP;
                gp = (hi - lo) * g.iD[d];
            }
            F.u[d][c] = F.HbyA[d][c] - F.rAU[c] * gp;
        }
        F.pr[c] = prP;
    }
    grid_reduce<1, false>(red, F.partials, F.counters + 6, F.scal + SC_CONT, pos);
}
__global__ void k_update(Grid g, Params P, Fields F, Level L0) {
    b_update(grid_pos(), g, P, F, L0);
}

// ---------------------------------------------------------------- force on the body
// Eq. dragcoeff read through the momentum balance of the imposed rows (ic and
// laminar-branch bc cells): there the row residual at the imposed values ut,
//   r_q = aP ut_P + sum_s a_s ut_N - b0_q + V dp/dx_q,
// is the forcing f_ib V of Eq. hfdibrans_1, and the force of the fluid on the
// body is -sum r.  Out: scal[SC_FORCE + q] = -sum V dp/dx_q (pressure part,
// f_n), scal[SC_FORCE + 3 + q] = the rest (viscous and convective, f_t).
// Needs the imposed fields and grad u of the current state.
__global__ void k_ib_force(Grid g, Fields F) {
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < g.N;
         c += (long long)gridDim.x * blockDim.x) {
        uint16_t f = F.flags[c];
        if (!((tag_of(f) == TAG_IC) || (f & F_AU))) continue;
        int i, j, k;
        cell_ijk(g, c, i, j, k);
        MomRow R;
        mom_row(g, F, c, i, j, k, f, R);
        double nuP = g.nu + F.nut[c];
        #pragma unroll
        for (int q = 0; q < 3 && q < g.dims; ++q) {
            double uP;
            vel_row_fixed(g, F, c, q, uP);
            double r = R.aP[q] * uP;
            #pragma unroll
            for (int s = 0; s < 6 && s < 2 * g.dims; ++s) {
                if (!R.has[s]) continue;
                long long nc = R.nb[s];
                double uN;
                if (!vel_row_fixed(g, F, nc, q, uN)) uN = F.u[q][nc];
                r += R.a[s] * uN;
            }
            double b0 = R.bnd[q] + transpose_src(g, F, c, i, j, k, q, nuP);
            if (g.conv) b0 += conv_src(g, F, c, i, j, k, q);
            r -= b0;
            v[q] -= g.V * grad_p(g, F.p, c, q, i, j, k);
            v[3 + q] -= r;
        }
    }
    grid_reduce<6, false>(v, F.partials, F.counters + 12, F.scal + SC_FORCE);
}

// Eq. dragcoeff: C_d = 2 F.v_d / (A_ref |u_in|^2) with v_d = (1, 0, 0);
// Eq. dlcoeffs: C_l the same with v_l = (-sin gamma, cos gamma, 0); F = f_n + f_t
// (kinematic, so rho drops out)
__global__ void k_force_coefficients(Fields F, double A_ref, double U2, double gamma) {
    const double* f = F.scal + SC_FORCE;
    double Fx = f[0] + f[3], Fy = f[1] + f[4];
    double q = 2.0 / (A_ref * U2);
    F.scal[SC_COEF] = q * Fx;
    F.scal[SC_COEF + 1] = q * (-sin(gamma) * Fx + cos(gamma) * Fy);
}

// ---------------------------------------------------------------- wall shear
// tau_w along one no-slip domain side (Sec. 3.3): the shear of the discrete
// wall flux, nu_eff,P (u_P - 0)/(Delta/2) per tangential component, with
// u_P the velocity the row sees (the imposed value in an imposed row); zero
// on closed faces (a wall inside the solid carries no flux) and for the
// normal component.  tau[q * n_faces + f], faces in cell order along the wall.
__global__ void k_wall_shear(Grid g, Fields F, int side, long long nf, double* tau) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nf) return;
    const int d = side >> 1, hi = side & 1;
    // the wall's cells: coordinate d fixed, the other two in x, y, z order
    const int n0 = (d == 0) ? g.n[1] : g.n[0];
    const int t0 = (int)(e % n0), t1 = (int)(e / n0);
    const int w = hi ? (d == 0 ? g.n[0] : (d == 1 ? g.n[1] : g.n[2])) - 1 : 0;
    int i, j, k;
    if (d == 0) { i = w; j = t0; k = t1; }
    else if (d == 1) { i = t0; j = w; k = t1; }
    else { i = t0; j = t1; k = w; }
    long long c = ((long long)k * g.n[1] + j) * g.n[0] + i;
    uint16_t f = F.flags[c];
    bool open = !closed_side(f, side);
    double nuP = g.nu + F.nut[c];
    #pragma unroll
    for (int q = 0; q < 3; ++q) {
        double val = 0.0;
        if (open && q != d && q < g.dims) {
            double uP;
            if (!vel_row_fixed(g, F, c, q, uP)) uP = F.u[q][c];
            val = nuP * uP * g.iD[d] * 2.0;
        }
        tau[(long long)q * nf + e] = val;
    }
}

// ---------------------------------------------------------------- recirculation
// The recirculation region behind a body (Sec. 3.6): cells outside the solid
// (not ic) with centre x > x_rear and u_x < 0.  Out: scal[SC_RECIRC] = the
// largest x_c - x_rear over them (-1e308 when there is none); *count = their
// number (integer atomics: exact), so the volume is count V.
__global__ void k_recirc(Grid g, Fields F, double x_rear, unsigned int* count) {
    double v[1] = {-1.0e308};
    unsigned int n = 0;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < g.N;
         c += (long long)gridDim.x * blockDim.x) {
        if (tag_of(F.flags[c]) == TAG_IC || !(F.u[0][c] < 0.0)) continue;
        int i, j, k;
        cell_ijk(g, c, i, j, k);
        // centre x without contraction into an FMA (the same rounding as a
        // plain multiply-add on the host)
        double dx = __dsub_rn(__dadd_rn(g.o[0], __dmul_rn(i + 0.5, g.D[0])), x_rear);
        if (dx > 0.0) {
            v[0] = fmax(v[0], dx);
            ++n;
        }
    }
    if (n) atomicAdd(count, n);
    grid_reduce<1, true>(v, F.partials, F.counters + 14, F.scal + SC_RECIRC);
}

// ---------------------------------------------------------------- sweep end
__device__ __forceinline__ void b_sweep_end(Pos pos, const Fields& F, int dims, int model, const int* err,
                                            double* res_out, double* hist, int nhist) {
    double* s = F.scal;
    if (err && *err) s[SC_TIMEOUT] = 1.0;
    res_out[HFDIB_NRES] = s[SC_TIMEOUT];
    auto sc = [](double r, double n1, double n2) { return r / ((n1 + n2) + 1e-20); };
    double res[HFDIB_NRES];
    for (int q = 0; q < 3; ++q)
        res[HFDIB_RES_UX + q] = q < dims ? sc(s[SC_RES_U + 3 * q], s[SC_RES_U + 3 * q + 1], s[SC_RES_U + 3 * q + 2]) : 0.0;
    res[HFDIB_RES_P] = sc(s[SC_PCG_INIT + 3], s[SC_PCG_INIT + 4], s[SC_PCG_INIT + 5]);
    if (model != HFDIB_LAMINAR) {
        res[HFDIB_RES_EPSW] = sc(s[SC_RES_W], s[SC_RES_W + 1], s[SC_RES_W + 2]);
        res[HFDIB_RES_K] = sc(s[SC_RES_K], s[SC_RES_K + 1], s[SC_RES_K + 2]);
    } else {
        res[HFDIB_RES_EPSW] = 0.0;
        res[HFDIB_RES_K] = 0.0;
    }
    res[HFDIB_RES_CONT] = s[SC_CONT];
    res[HFDIB_RES_PITER] = s[SC_PCG_ITERS];
    res[HFDIB_RES_NLAM] = s[SC_NLAM];
    res[HFDIB_RES_NSWITCH] = s[SC_NSWITCH];
    s[SC_NLAM] = 0.0;
    s[SC_NSWITCH] = 0.0;
    long long n = (long long)s[SC_NSWEEP];
    int slot = (int)(n % nhist);
    for (int q = 0; q < HFDIB_NRES; ++q) {
        res_out[q] = res[q];
        hist[slot * HFDIB_NRES + q] = res[q];
    }
    s[SC_NSWEEP] = (double)(n + 1);
}
__global__ void k_sweep_end(Fields F, int dims, int model, const int* err, double* res_out, double* hist, int nhist) {
    b_sweep_end(grid_pos(), F, dims, model, err, res_out, hist, nhist);
}

// ---------------------------------------------------------------- launchers
void launch_init_flux(const Grid& g, const Fields& F, cudaStream_t s) {
    k_face_flux<<<nblocks(g.N), BLOCK, 0, s>>>(g, F.flags, F.u[0], F.u[1], F.u[2], F.phi[0], F.phi[1],
                                                F.phi[2]);
}
void launch_means(const Grid& g, const Params& P, const Fields& F, cudaStream_t s) {
    k_means<<<rblocks(g.N), BLOCK, 0, s>>>(g, P, F);
}
void launch_grad_u(const Grid& g, const Fields& F, cudaStream_t s) {
    k_grad_u<<<nblocks(g.N), BLOCK, 0, s>>>(g, F);
}
void launch_conv_limit(const Grid& g, const Fields& F, cudaStream_t s) {
    k_conv_limit<<<nblocks(g.N), BLOCK, 0, s>>>(g, F);
}
void launch_mom_asm(const Grid& g, const Params& P, const Fields& F, cudaStream_t s) {
    k_mom_asm<<<rblocks(g.N), BLOCK, 0, s>>>(g, P, F);
}
void launch_mom_smooth(const Grid& g, const Params& P, const Fields& F, int colour, cudaStream_t s) {
    k_mom_smooth<<<nblocks(npairs(g)), BLOCK, 0, s>>>(g, P, F, colour);
}
void launch_mom_smooth32(const Grid& g, const Params& P, const Fields& F, int colour, int zero_init, int finalize,
                         cudaStream_t s) {
    k_mom_smooth32<<<nblocks(npairs(g)), BLOCK, 0, s>>>(g, P, F, colour, zero_init, finalize);
}
void launch_hbya(const Grid& g, const Params& P, const Fields& F, cudaStream_t s) {
    k_hbya<<<nblocks(g.N), BLOCK, 0, s>>>(g, P, F);
}
void launch_phiH(const Grid& g, const Fields& F, cudaStream_t s) {
    k_phiH<<<nblocks(g.N), BLOCK, 0, s>>>(g, F);
}
void launch_update(const Grid& g, const Params& P, const Fields& F, const Level& L0, cudaStream_t s) {
    k_update<<<rblocks(g.N), BLOCK, 0, s>>>(g, P, F, L0);
}
void launch_ib_force(const Grid& g, const Fields& F, cudaStream_t s) {
    k_ib_force<<<rblocks(g.N), BLOCK, 0, s>>>(g, F);
}
void launch_force_coefficients(const Fields& F, double A_ref, double U2, double gamma, cudaStream_t s) {
    k_force_coefficients<<<1, 1, 0, s>>>(F, A_ref, U2, gamma);
}
void launch_wall_shear(const Grid& g, const Fields& F, int side, long long nf, double* tau, cudaStream_t s) {
    if (nf > 0) k_wall_shear<<<nblocks(nf), BLOCK, 0, s>>>(g, F, side, nf, tau);
}
void launch_recirc(const Grid& g, const Fields& F, double x_rear, unsigned int* count, cudaStream_t s) {
    k_recirc<<<rblocks(g.N), BLOCK, 0, s>>>(g, F, x_rear, count);
}
void launch_sweep_end(const Params& P, const Fields& F, int dims, const int* err, double* res_out, double* hist,
                      int nhist, cudaStream_t s) {
    k_sweep_end<<<1, 1, 0, s>>>(F, dims, P.model, err, res_out, hist, nhist);
}

// ---------------------------------------------------------------- batched launches
struct OpMeans {
    __device__ void operator()(Pos p, const SweepProblem& s) const { b_means(p, s.g, s.P, s.F); }
};
struct OpGradU {
    __device__ void operator()(Pos p, const SweepProblem& s) const { b_grad_u(p, s.g, s.F); }
};
struct OpConvLimit {
    __device__ void operator()(Pos p, const SweepProblem& s) const { b_conv_limit(p, s.g, s.F); }
};
struct OpMomAsm {
    __device__ void operator()(Pos p, const SweepProblem& s) const { b_mom_asm(p, s.g, s.P, s.F); }
};
struct OpMomSmooth {
    int colour;
    __device__ void operator()(Pos p, const SweepProblem& s) const { b_mom_smooth(p, s.g, s.P, s.F, colour); }
};
struct OpMomSmooth32 {
    int colour, zero_init, finalize;
    __device__ void operator()(Pos p, const SweepProblem& s) const {
        b_mom_smooth32(p, s.g, s.P, s.F, colour, zero_init, finalize);
    }
};
struct OpHbyA {
    __device__ void operator()(Pos p, const SweepProblem& s) const { b_hbya(p, s.g, s.P, s.F); }
};
struct OpPhiH {
    __device__ void operator()(Pos p, const SweepProblem& s) const { b_phiH(p, s.g, s.F); }
};
struct OpUpdate {
    __device__ void operator()(Pos p, const SweepProblem& s) const { b_update(p, s.g, s.P, s.F, s.L0); }
};
// the residual record, then (batch solves) the stop test on the largest
// scaled residual, then the p / pr swap of this problem's device tables
struct OpSweepEnd {
    __device__ void operator()(Pos p, const SweepProblem& s) const {
        if (threadIdx.x != 0) return;
        b_sweep_end(p, s.F, s.g.dims, s.model_end, s.err, s.res_out, s.hist, s.nhist);
        double* sc = s.F.scal;
        if (sc[SC_STOP_ON] != 0.0 && sc[SC_DONE] == 0.0) {
            double mx = 0.0;
            bool bad = false;
            for (int q = 0; q <= HFDIB_RES_K; ++q) {
                const double v = s.res_out[q];
                if (!isfinite(v)) bad = true;
                mx = fmax(mx, v);
            }
            if (bad || mx <= sc[SC_STOP_TOL]) {
                sc[SC_DONE] = bad ? 2.0 : 1.0;
                sc[SC_DONE_AT] = sc[SC_NSWEEP];
            }
        }
        for (int t = 0; t < 2; ++t) {
            double* a = *s.swap_p[t];
            *s.swap_p[t] = *s.swap_pr[t];
            *s.swap_pr[t] = a;
        }
    }
};
__global__ void k_batch_next(BatchTab T, unsigned int* count, const unsigned int* max_iter,
                             cudaGraphConditionalHandle h) {
    const unsigned int n = *count + 1;
    *count = n;
    bool all = true;
    for (int b = 0; b < T.B; ++b) all = all && (*T.probs[b].done != 0.0);
    cudaGraphSetConditional(h, (!all && n < *max_iter) ? 1u : 0u);
}

void launchb_means(const BatchTab& T, const int* tot, cudaStream_t s) {
    k_batched<BK_REDUCE, OpMeans><<<tot[BK_REDUCE], BLOCK, 0, s>>>(T, OpMeans{});
}
void launchb_grad_u(const BatchTab& T, const int* tot, cudaStream_t s) {
    k_batched<BK_CELLS, OpGradU><<<tot[BK_CELLS], BLOCK, 0, s>>>(T, OpGradU{});
}
void launchb_conv_limit(const BatchTab& T, const int* tot, cudaStream_t s) {
    k_batched<BK_CELLS, OpConvLimit><<<tot[BK_CELLS], BLOCK, 0, s>>>(T, OpConvLimit{});
}
void launchb_mom_asm(const BatchTab& T, const int* tot, cudaStream_t s) {
    k_batched<BK_REDUCE, OpMomAsm><<<tot[BK_REDUCE], BLOCK, 0, s>>>(T, OpMomAsm{});
}
void launchb_mom_smooth(const BatchTab& T, const int* tot, int colour, cudaStream_t s) {
    k_batched<BK_PAIRS, OpMomSmooth><<<tot[BK_PAIRS], BLOCK, 0, s>>>(T, OpMomSmooth{colour});
}
void launchb_mom_smooth32(const BatchTab& T, const int* tot, int colour, int zero_init, int finalize,
                          cudaStream_t s) {
    k_batched<BK_PAIRS, OpMomSmooth32><<<tot[BK_PAIRS], BLOCK, 0, s>>>(T, OpMomSmooth32{colour, zero_init, finalize});
}
void launchb_hbya(const BatchTab& T, const int* tot, cudaStream_t s) {
    k_batched<BK_CELLS, OpHbyA><<<tot[BK_CELLS], BLOCK, 0, s>>>(T, OpHbyA{});
}
void launchb_phiH(const BatchTab& T, const int* tot, cudaStream_t s) {
    k_batched<BK_CELLS, OpPhiH><<<tot[BK_CELLS], BLOCK, 0, s>>>(T, OpPhiH{});
}
void launchb_update(const BatchTab& T, const int* tot, cudaStream_t s) {
    k_batched<BK_REDUCE, OpUpdate><<<tot[BK_REDUCE], BLOCK, 0, s>>>(T, OpUpdate{});
}
void launchb_sweep_end(const BatchTab& T, const int* tot, cudaStream_t s) {
    k_batched<BK_ONE, OpSweepEnd><<<tot[BK_ONE], BLOCK, 0, s>>>(T, OpSweepEnd{});
}
void launchb_next(const BatchTab& T, unsigned int* count, const unsigned int* max_iter,
                  cudaGraphConditionalHandle h, cudaStream_t s) {
    k_batch_next<<<1, 1, 0, s>>>(T, count, max_iter, h);
}

}  // namespace hf
