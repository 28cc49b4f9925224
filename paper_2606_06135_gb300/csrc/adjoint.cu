// adjoint.cu -- reverse pass of the frozen-turbulence SIMPLE sweep, for the
// gradient of the pressure drop or the drag with respect to the indicator
// lambda.
//
// The sweep (Fig. simplehfdibrans, steps a2-a8 with nu_t, k, eps/omega, the
// cell groups, the wall-function branch of every bc cell, the closed faces and
// the reading-A continuity mask held fixed; reading B's mask 1 - lambda is
// differentiated) is a map G: x = (u, p, phi) -> x' whose fixed
// point is the converged state.  The map differentiated here is the GPU sweep
// itself, with its n_u red-black Gauss-Seidel passes of the momentum predictor
// and with an exact pressure solve (any inner solver with the same fixed point
// gives the same gradient).  Its transpose is applied as a sequence of gather
// kernels, each the exact reverse of one forward kernel at the converged state:
//
//   a8  u' = HbyA - rAU grad p_r, p' = p_r = p + a_p (p_n - p),
//       phi' = phiHbyA - rAU_f S dp_n/Delta                    k_adj_update
//   a7  L(rAU) p_n = -m div phiHbyA + b_out (L symmetric: the adjoint solve is
//       another solve with L)                                   k_adj_pcg_init
//       (+ the PCG kernels of pressure.cu), k_adj_pressure
//   a6  HbyA, rAU, phiHbyA                                      k_adj_hbya
//   a4  red-black sweeps, last half-sweep first                 k_adj_gs
//   a3  b_m = b0 + rlx aP u - V grad p, b0 = bnd + div(nu_eff (grad u)^T),
//       coefficients aP, a_N from the face fluxes (upwind side frozen)
//                                                               k_adj_b0, k_adj_transpose,
//                                                               k_adj_gradu, k_adj_phi
//   a2  u_ib = wS u_s + w1 I1(u) + w2 I2(u) (Sec. 2.5)          k_adj_gradu (transposed
//       interpolation by a per-cell entry list, no atomics)
//
// The adjoint psi solves psi = G_x^T psi + J_x^T by this fixed-point iteration
// (reverse accumulation), and dJ/dlambda = G_lambda^T psi: lambda moves u_ib
// through the normal n = -grad(lambda)/|grad(lambda)| (Eq. yorthoaux), y_perp
// (Eq. yortho with sigma = h atanh(1 - 2 lambda)), the interpolation fractions
// and the quadratic weights (k_adj_dlambda).
#include "common.cuh"
#include "kernels.cuh"

namespace hf {

namespace {

__device__ inline bool has_nb(const Grid& g, int d, int side, int i, int j, int k) {
    int pos = coord(d, i, j, k);
    return side ? pos < g.n[d] - 1 : pos > 0;
}
__device__ inline bool fixed_row(uint16_t f) { return tag_of(f) == TAG_IC || (f & F_AU); }
__device__ inline bool au_row(uint16_t f) { return tag_of(f) != TAG_IC && (f & F_AU); }
__device__ inline int colour_of(int i, int j, int k) { return (i + j + k) & 1; }

// d(grad_d f)_c / d f_c for a Gauss-linear gradient whose boundary face takes
// a fixed value (fixed_lo / fixed_hi) or the cell value (zero gradient)
__device__ inline double own_grad_coef(bool int_lo, bool int_hi, bool fixed_lo, bool fixed_hi, double iD) {
    double hi = int_hi ? 0.5 : (fixed_hi ? 0.0 : 1.0);
    double lo = int_lo ? 0.5 : (fixed_lo ? 0.0 : 1.0);
    return (hi - lo) * iD;
}

// Gauss-linear gradient of the relaxed pressure p + a (pn - p) along d
__device__ inline double grad_pr(const Grid& g, const double* p, const double* pn, double a, long long c, int d,
                                 int i, int j, int k) {
    double pc = p[c] + a * (pn[c] - p[c]);
    double lo, hi;
    if (has_nb(g, d, 0, i, j, k)) {
        long long n = c - g.stride[d];
        lo = 0.5 * ((p[n] + a * (pn[n] - p[n])) + pc);
    } else {
        lo = p_fixed(g, 2 * d) ? g.p_out : pc;
    }
    if (has_nb(g, d, 1, i, j, k)) {
        long long n = c + g.stride[d];
        hi = 0.5 * (pc + (p[n] + a * (pn[n] - p[n])));
    } else {
        hi = p_fixed(g, 2 * d + 1) ? g.p_out : pc;
    }
    return (hi - lo) * g.iD[d];
}

}  // namespace

// ---------------------------------------------------------------- coefficients at x*
// Momentum-row coefficients of the converged state (frozen for the whole
// adjoint): a_s per side, the unrelaxed diagonal per component, aavg.
__global__ void k_adj_coef(Grid g, Params P, Fields F, Adj A) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    uint16_t f = F.flags[c];
    const double nu = g.nu;
    double nuP = nu + F.nut[c];
    double aP[3] = {0.0, 0.0, 0.0};
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        long long fl = face_lo(g, d, i, j, k);
        long long fs = face_stride(g, d);
        for (int side = 0; side < 2; ++side) {
            int s = 2 * d + side;
            double Fb = F.phi[d][fl + side * fs];
            double Fout = side ? Fb : -Fb;
            if (has_nb(g, d, side, i, j, k)) {
                long long nc = side ? c + g.stride[d] : c - g.stride[d];
                double Dif = 0.5 * (nuP + (nu + F.nut[nc])) * g.SoD[d];
                A.As[(long long)s * g.N + c] = fmin(Fout, 0.0) - Dif;
                double add = fmax(-Fout, 0.0) + Dif;
                #pragma unroll
                for (int q = 0; q < 3 && q < g.dims; ++q) aP[q] += add;
            } else {
                A.As[(long long)s * g.N + c] = 0.0;
                #pragma unroll
                for (int q = 0; q < 3 && q < g.dims; ++q) {
                    double val;
                    if (vel_fixed(g, f, s, q, val)) aP[q] += nuP * g.SoHD[d] + fmax(-Fout, 0.0);
                }
            }
        }
    }
    double avg = 0.0;
    #pragma unroll
    for (int q = 0; q < 3 && q < g.dims; ++q) {
        A.AP[(long long)q * g.N + c] = aP[q];
        avg += aP[q] * P.iurf_u;
    }
    A.aavg[c] = avg * (g.dims == 2 ? 0.5 : (1.0 / 3.0));
}

// ---------------------------------------------------------------- a8 reversed
// In: psi (adjoint of u', p', phi').  Out: HbyA-bar (partial), rAU-bar (partial),
// the right-hand side of the adjoint pressure solve and p-bar (partial).
__global__ void k_adj_update(Grid g, Params P, Fields F, Level L0, Adj A) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const double a = P.urf_p;
    double rAUb = 0.0;
    double prb = A.psp[c];
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        const double* psu = A.psu[d];
        double gp = grad_pr(g, F.p, F.pn, a, c, d, i, j, k);
        A.Hb[d][c] = psu[c];
        rAUb -= psu[c] * gp;
        // p_r-bar: transpose of the gradient applied to w = -rAU u'-bar
        bool lo = has_nb(g, d, 0, i, j, k), hi = has_nb(g, d, 1, i, j, k);
        prb += -F.rAU[c] * psu[c] * own_grad_coef(lo, hi, p_fixed(g, 2 * d), p_fixed(g, 2 * d + 1), g.iD[d]);
        if (lo) {
            long long n = c - g.stride[d];
            prb += -F.rAU[n] * psu[n] * 0.5 * g.iD[d];
        }
        if (hi) {
            long long n = c + g.stride[d];
            prb -= -F.rAU[n] * psu[n] * 0.5 * g.iD[d];
        }
    }
    A.xbp[c] = (1.0 - a) * prb;
    double pnb = a * prb;
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        long long fl = face_lo(g, d, i, j, k);
        long long fh = fl + face_stride(g, d);
        // phi'_lo = phiH - cf (pn_c - pn_lo | p_out); phi'_hi = phiH - cf (pn_hi | p_out - pn_c)
        if (has_nb(g, d, 0, i, j, k) || p_fixed(g, 2 * d)) pnb -= L0.cf[d][fl] * A.psf[d][fl];
        if (has_nb(g, d, 1, i, j, k) || p_fixed(g, 2 * d + 1)) pnb += L0.cf[d][fh] * A.psf[d][fh];
    }
    A.pnb[c] = pnb;
    A.rAUb[c] = rAUb;
}

// ---------------------------------------------------------------- a7 reversed: solve set-up
// r = rhs - L x0 with x0 = the previous adjoint solution (warm start); the
// loop kernels of pressure.cu then run unchanged on the redirected Fields.
// The slot the loop takes as |r0|^2 receives |rhs|^2 + |r0|^2, so the
// relative tolerance is measured against the right-hand side, not against the
// (small) warm-started residual: every solve is accurate to tol |rhs|.
__global__ void k_adj_pcg_init(Grid g, Fields F, Level L0, const double* __restrict__ rhs, int jacobi) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double red[6] = {0, 0, 0, 0, 0, 0};
    if (c < g.N) {
        int i, j, k;
        cell_ijk(g, c, i, j, k);
        int idx[3] = {i, j, k};
        double dg = L0.diag[c];
        double Ax = dg * F.pn[c];
        #pragma unroll
        for (int d = 0; d < 3 && d < g.dims; ++d) {
            long long fl = face_lo(g, d, i, j, k);
            if (idx[d] > 0) Ax -= L0.cf[d][fl] * F.pn[c - g.stride[d]];
            if (idx[d] < g.n[d] - 1) Ax -= L0.cf[d][fl + face_stride(g, d)] * F.pn[c + g.stride[d]];
        }
        double r = rhs[c] - Ax;
        F.r[c] = r;
        F.d[0][c] = 0.0;
        F.d[1][c] = 0.0;
        double z = 0.0;
        if (jacobi) { z = dg > 0.0 ? r / dg : 0.0; F.z[c] = z; }
        red[0] = r * z;
        red[1] = r * r + rhs[c] * rhs[c];
        red[2] = rhs[c] * rhs[c];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) F.scal[SC_PCG_DONE] = 0.0;
    grid_reduce<6, false>(red, F.partials, F.counters + 3, F.scal + SC_PCG_INIT);
}

// ---------------------------------------------------------------- a7/a6 reversed
// With the adjoint pressure ps: cf-bar per face (from phi' and from the solve),
// phiHbyA-bar per face, then rAU-bar and HbyA-bar of the cell (gathered over
// its own faces, so no two threads write one value).
__global__ void k_adj_pressure(Grid g, Fields F, Level L0, Adj A) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    uint16_t f = F.flags[c];
    const double* ps = A.ps;
    const double* pn = F.pn;
    double mc = cont_mask(g, F.lam, f, c);
    double rAUb = A.rAUb[c];
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        long long fl = face_lo(g, d, i, j, k);
        long long fh = fl + face_stride(g, d);
        double Hb = A.Hb[d][c];
        double half = 0.5 * g.SoD[d];
        // low face
        if (has_nb(g, d, 0, i, j, k)) {
            long long n = c - g.stride[d];
            double mn = cont_mask(g, F.lam, F.flags[n], n);
            double psi_f = A.psf[d][fl];
            double cfb = (pn[c] - pn[n]) * (-psi_f + ps[n] - ps[c]);
            rAUb += half * cfb;
            Hb += 0.5 * g.S[d] * (psi_f - mn * ps[n] + mc * ps[c]);
        } else {
            double psi_f = A.psf[d][fl];
            if (p_fixed(g, 2 * d)) rAUb += 2.0 * g.SoD[d] * (g.p_out - pn[c]) * (ps[c] + psi_f);
            if (g.kind[2 * d] == HFDIB_BC_OUTLET && !closed_side(f, 2 * d)) Hb += g.S[d] * (psi_f + mc * ps[c]);
        }
        // high face
        if (has_nb(g, d, 1, i, j, k)) {
            long long n = c + g.stride[d];
            double mn = cont_mask(g, F.lam, F.flags[n], n);
            double psi_f = A.psf[d][fh];
            double cfb = (pn[n] - pn[c]) * (-psi_f + ps[c] - ps[n]);
            rAUb += half * cfb;
            Hb += 0.5 * g.S[d] * (psi_f - mc * ps[c] + mn * ps[n]);
        } else {
            double psi_f = A.psf[d][fh];
            if (p_fixed(g, 2 * d + 1)) rAUb += 2.0 * g.SoD[d] * (g.p_out - pn[c]) * (ps[c] - psi_f);
            if (g.kind[2 * d + 1] == HFDIB_BC_OUTLET && !closed_side(f, 2 * d + 1))
                Hb += g.S[d] * (psi_f - mc * ps[c]);
        }
        A.Hb[d][c] = Hb;
    }
    A.rAUb[c] = rAUb;
}

// ---------------------------------------------------------------- a6 reversed
// HbyA_q = N_q / aavg, N_q = b0_q + rlx aP_q u_q - sum_s a_s us_q[nb] - (aP_q/urf - aavg) us_q,
// rAU = V / aavg, aavg = sum_q aP_q / (urf dims).  Writes b0-bar, u-bar (first
// term), us-bar of the final predictor iterate (gathered from the neighbours'
// rows), aP-bar and a_s-bar; clears bm-bar and u_ib-bar for the sweeps.
__global__ void k_adj_hbya(Grid g, Params P, Fields F, Adj A) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const long long N = g.N;
    double aavg = A.aavg[c];
    double ia = 1.0 / aavg;
    double urf = P.urf_u, rlx = P.rlx_u;
    double iab = g.V * A.rAUb[c];
    double avb = 0.0;
    double Hb[3] = {0.0, 0.0, 0.0};
    #pragma unroll
    for (int q = 0; q < 3 && q < g.dims; ++q) {
        Hb[q] = A.Hb[q][c];
        double us = F.us[q][c];
        double aPq = A.AP[q * N + c];
        A.b0b[q][c] = ia * Hb[q];
        A.xbu[q][c] = ia * Hb[q] * rlx * aPq;
        iab += F.HbyA[q][c] * aavg * Hb[q];
        avb += us * ia * Hb[q];
        double usb = -(aPq * P.iurf_u - aavg) * ia * Hb[q];
        #pragma unroll
        for (int d = 0; d < 3 && d < g.dims; ++d)
            for (int side = 0; side < 2; ++side) {
                if (!has_nb(g, d, side, i, j, k)) continue;
                long long r = side ? c + g.stride[d] : c - g.stride[d];
                int s_r = 2 * d + (1 - side);  // side of r that faces c
                usb -= A.As[s_r * N + r] * (1.0 / A.aavg[r]) * A.Hb[q][r];
            }
        A.usb[0][q][c] = usb;
        A.bmb[q][c] = 0.0;
        A.fixb[q][c] = 0.0;
    }
    avb += -ia * ia * iab;
    #pragma unroll
    for (int q = 0; q < 3 && q < g.dims; ++q)
        A.aPb[q][c] = ia * Hb[q] * (rlx * F.u[q][c] - F.us[q][c] / urf) + avb / (urf * g.dims);
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d)
        for (int side = 0; side < 2; ++side) {
            int s = 2 * d + side;
            double v = 0.0;
            if (has_nb(g, d, side, i, j, k)) {
                long long r = side ? c + g.stride[d] : c - g.stride[d];
                #pragma unroll
                for (int q = 0; q < 3 && q < g.dims; ++q) v -= F.us[q][r] * ia * Hb[q];
            }
            A.asb[s * N + c] = v;
        }
}

// ---------------------------------------------------------------- a4 reversed
// One red-black half-sweep in reverse.  Forward, cells of `colour` were set to
// (bm - sum_s a_s S_in[nb]) urf/aP (free rows) or to their imposed value
// (u_ib, u_s); the other colour was copied.  usb[in_buf] holds the adjoint of
// S_out, usb[1 - in_buf] receives the adjoint of S_in.
__global__ void k_adj_gs(Grid g, Params P, Fields F, Adj A, int colour, const double* __restrict__ Sin,
                         const double* __restrict__ Sout, int in_buf) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const long long N = g.N;
    uint16_t f = F.flags[c];
    double urf = P.urf_u;
    double* const* bin = A.usb[in_buf];
    double* const* bout = A.usb[1 - in_buf];
    if (colour_of(i, j, k) == colour) {
        if (tag_of(f) == TAG_IC) {
            #pragma unroll
            for (int q = 0; q < 3 && q < g.dims; ++q) bout[q][c] = 0.0;
            return;
        }
        if (f & F_AU) {
            #pragma unroll
            for (int q = 0; q < 3 && q < g.dims; ++q) {
                A.fixb[q][c] += bin[q][c];
                bout[q][c] = 0.0;
            }
            return;
        }
        double gq[3] = {0.0, 0.0, 0.0};
        #pragma unroll
        for (int q = 0; q < 3 && q < g.dims; ++q) {
            double ub = bin[q][c];
            double aPq = A.AP[q * N + c];
            gq[q] = ub * urf / aPq;
            A.bmb[q][c] += gq[q];
            A.aPb[q][c] += -Sout[q * N + c] / aPq * ub;
            bout[q][c] = 0.0;
        }
        #pragma unroll
        for (int d = 0; d < 3 && d < g.dims; ++d)
            for (int side = 0; side < 2; ++side) {
                if (!has_nb(g, d, side, i, j, k)) continue;
                long long r = side ? c + g.stride[d] : c - g.stride[d];
                double v = 0.0;
                #pragma unroll
                for (int q = 0; q < 3 && q < g.dims; ++q) v -= Sin[q * N + r] * gq[q];
                A.asb[(2 * d + side) * N + c] += v;
            }
        return;
    }
    #pragma unroll
    for (int q = 0; q < 3 && q < g.dims; ++q) {
        double v = bin[q][c];
        #pragma unroll
        for (int d = 0; d < 3 && d < g.dims; ++d)
            for (int side = 0; side < 2; ++side) {
                if (!has_nb(g, d, side, i, j, k)) continue;
                long long r = side ? c + g.stride[d] : c - g.stride[d];
                if (fixed_row(F.flags[r])) continue;
                int s_r = 2 * d + (1 - side);
                v -= A.As[s_r * N + r] * urf / A.AP[q * N + r] * bin[q][r];
            }
        bout[q][c] = v;
    }
}

// ---------------------------------------------------------------- a3 reversed (own cell)
// The predictor started from S_0 = u (free rows) or u_ib (imposed rows);
// b_m = b0 + rlx aP u - V grad p.  usb[buf] holds the adjoint of S_0.
__global__ void k_adj_b0(Grid g, Params P, Fields F, Adj A, int buf) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    uint16_t f = F.flags[c];
    const long long N = g.N;
    #pragma unroll
    for (int q = 0; q < 3 && q < g.dims; ++q) {
        double us0 = A.usb[buf][q][c];
        double bmb = A.bmb[q][c];
        double xu = A.xbu[q][c];
        if (tag_of(f) != TAG_IC) {
            if (f & F_AU) A.fixb[q][c] += us0;
            else xu += us0;
        }
        double aPq = A.AP[q * N + c];
        A.b0b[q][c] += bmb;
        xu += P.rlx_u * aPq * bmb;
        A.aPb[q][c] += P.rlx_u * F.u[q][c] * bmb;
        A.xbu[q][c] = xu;
    }
}

// ---------------------------------------------------------------- a3 reversed (gathers)
// p-bar from -V grad p in b_m; grad-u-bar from b0-bar through the explicit
// div(nu_eff (grad u)^T): face flux nu_f (d u_a/d x_q)_f S_a.
__global__ void k_adj_transpose(Grid g, Fields F, Adj A) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const long long N = g.N;
    double pb = 0.0;
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        bool lo = has_nb(g, d, 0, i, j, k), hi = has_nb(g, d, 1, i, j, k);
        pb += -g.V * A.bmb[d][c] * own_grad_coef(lo, hi, p_fixed(g, 2 * d), p_fixed(g, 2 * d + 1), g.iD[d]);
        if (lo) pb += -g.V * A.bmb[d][c - g.stride[d]] * 0.5 * g.iD[d];
        if (hi) pb -= -g.V * A.bmb[d][c + g.stride[d]] * 0.5 * g.iD[d];
    }
    A.xbp[c] += pb;
    double nuc = g.nu + F.nut[c];
    #pragma unroll
    for (int q = 0; q < 3 && q < g.dims; ++q) {
        const double* Tb = A.b0b[q];
        double Tc = Tb[c];
        #pragma unroll
        for (int a = 0; a < 3 && a < g.dims; ++a) {
            double v;
            if (has_nb(g, a, 1, i, j, k)) {
                long long n = c + g.stride[a];
                v = 0.25 * (nuc + (g.nu + F.nut[n])) * (Tc - Tb[n]);
            } else {
                v = nuc * Tc;
            }
            if (has_nb(g, a, 0, i, j, k)) {
                long long n = c - g.stride[a];
                v -= 0.25 * (nuc + (g.nu + F.nut[n])) * (Tc - Tb[n]);
            } else {
                v -= nuc * Tc;
            }
            A.Gb[(3 * q + a) * N + c] = v * g.S[a];
        }
    }
}

// weight of corner `corner` of stencil `st` (0: X1, 1: X2) of bc entry q in its u_ib
__device__ inline double interp_weight(const Grid& g, const BcList& bl, int q, int st, int corner) {
    const double* t = (st ? bl.t2 : bl.t1) + 3 * q;
    double w = st ? bl.w2[q] : bl.w1[q];
    for (int d = 0; d < 3; ++d) {
        int cc = (corner >> d) & 1;
        if (g.n[d] == 1) w = cc ? 0.0 : w;
        else w = w * (cc ? t[d] : (1.0 - t[d]));
    }
    return w;
}

// u-bar from grad-u-bar (transposed Gauss gradient with the velocity boundary
// values) and from u_ib-bar (transposed interpolation, entry list per cell)
__global__ void k_adj_gradu(Grid g, Fields F, BcList bl, Adj A) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const long long N = g.N;
    uint16_t f = F.flags[c];
    int e0 = A.tptr[c], e1 = A.tptr[c + 1];
    #pragma unroll
    for (int b = 0; b < 3 && b < g.dims; ++b) {
        double ub = 0.0;
        #pragma unroll
        for (int a = 0; a < 3 && a < g.dims; ++a) {
            const double* Gb = A.Gb + (3 * a + b) * N;
            double val;
            bool lo = has_nb(g, a, 0, i, j, k), hi = has_nb(g, a, 1, i, j, k);
            bool flo = !lo && vel_fixed(g, f, 2 * a, b, val);
            bool fhi = !hi && vel_fixed(g, f, 2 * a + 1, b, val);
            ub += Gb[c] * own_grad_coef(lo, hi, flo, fhi, g.iD[a]);
            if (lo) ub += Gb[c - g.stride[a]] * 0.5 * g.iD[a];
            if (hi) ub -= Gb[c + g.stride[a]] * 0.5 * g.iD[a];
        }
        for (int e = e0; e < e1; ++e) {
            int ent = A.tent[e];
            int q = ent >> 4;
            ub += interp_weight(g, bl, q, (ent >> 3) & 1, ent & 7) * A.fixb[b][bl.cell[q]];
        }
        A.xbu[b][c] += ub;
    }
}

// phi-bar of the interior faces from aP-bar and a_s-bar of the two rows that
// share the face (bounded upwind: a_s = min(F_out, 0) - D, aP += max(-F_out, 0) + D;
// the upwind side is taken from the converged flux)
__global__ void k_adj_phi(Grid g, Fields F, Adj A) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const long long N = g.N;
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        long long fl = face_lo(g, d, i, j, k);
        double v = 0.0;
        if (has_nb(g, d, 0, i, j, k)) {
            long long n = c - g.stride[d];
            double Fv = F.phi[d][fl];
            if (Fv < 0.0) {  // inflow into n through its high side
                v += A.asb[(2 * d + 1) * N + n];
                #pragma unroll
                for (int q = 0; q < 3 && q < g.dims; ++q) v -= A.aPb[q][n];
            } else if (Fv > 0.0) {  // inflow into c through its low side
                v -= A.asb[(2 * d) * N + c];
                #pragma unroll
                for (int q = 0; q < 3 && q < g.dims; ++q) v += A.aPb[q][c];
            }
        }
        A.xbf[d][fl] = v;
        if (!has_nb(g, d, 1, i, j, k)) A.xbf[d][fl + face_stride(g, d)] = 0.0;
    }
}

// psi <- x-bar + J_x^T (A.vb); max |change| and max |psi| for the stop test
__global__ void k_adj_next(Grid g, Fields F, Adj A, int first) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[2] = {0.0, 0.0};
    if (c < g.N) {
        int i, j, k;
        cell_ijk(g, c, i, j, k);
        #pragma unroll
        for (int q = 0; q < 3 && q < g.dims; ++q) {
            double nw = A.xbu[q][c] + A.vbu[q][c];
            double old = first ? 0.0 : A.psu[q][c];
            v[0] = fmax(v[0], fabs(nw - old));
            v[1] = fmax(v[1], fabs(nw));
            A.psu[q][c] = nw;
        }
        {
            double nw = A.xbp[c] + A.vbp[c];
            double old = first ? 0.0 : A.psp[c];
            v[0] = fmax(v[0], fabs(nw - old));
            v[1] = fmax(v[1], fabs(nw));
            A.psp[c] = nw;
        }
        #pragma unroll
        for (int d = 0; d < 3 && d < g.dims; ++d) {
            long long fl = face_lo(g, d, i, j, k);
            for (int e = 0; e < 2; ++e) {
                if (e == 1 && has_nb(g, d, 1, i, j, k)) break;
                long long fi = fl + e * face_stride(g, d);
                double nw = A.xbf[d][fi] + A.vbf[d][fi];
                double old = first ? 0.0 : A.psf[d][fi];
                v[0] = fmax(v[0], fabs(nw - old));
                v[1] = fmax(v[1], fabs(nw));
                A.psf[d][fi] = nw;
            }
        }
    }
    grid_reduce<2, true>(v, F.partials, F.counters + 10, F.scal + SC_ADJ_DIFF);
}

// J = sum jw p (pressure drop: mean p on open inlet faces - mean p on outlet faces)
__global__ void k_adj_objective(Grid g, Fields F, Adj A) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[1] = {0.0};
    if (c < g.N) v[0] = A.jw[c] * F.p[c];
    grid_reduce<1, false>(v, F.partials, F.counters + 11, F.scal + SC_ADJ_J);
}

// ---------------------------------------------------------------- drag objective
// Drag: the x force of the fluid on the body, minus the x-momentum row
// residual of the imposed rows (ic and laminar-branch bc cells):
//   r = aP ut + sum_s a_s ut_N - (bnd + T) + V dp/dx,
// the forcing the immersed boundary applies to the fluid there (Eq.
// hfdibrans_1).  ut = u_s in ic cells, u_ib in laminar-branch bc cells, u
// elsewhere; the row is that of the sweep at the converged state (k_adj_coef).
namespace {

__device__ inline double drag_ut(const Grid& g, const Fields& F, long long c, uint16_t f) {
    if (tag_of(f) == TAG_IC) return g.u_s[0];
    if (f & F_AU) return F.uib[0][c];
    return F.u[0][c];
}

// boundary part and explicit transpose term of the x row, as the assembly forms them
__device__ double drag_b0(const Grid& g, const Fields& F, long long c, int i, int j, int k, uint16_t f) {
    const long long N = g.N;
    double nuP = g.nu + F.nut[c];
    double bnd = 0.0, T = 0.0;
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        long long fl = face_lo(g, d, i, j, k);
        long long fs = face_stride(g, d);
        for (int side = 0; side < 2; ++side) {
            if (has_nb(g, d, side, i, j, k)) continue;
            double val;
            if (vel_fixed(g, f, 2 * d + side, 0, val)) {
                double Fb = F.phi[d][fl + side * fs];
                double Fout = side ? Fb : -Fb;
                bnd += (nuP * g.SoHD[d] + fmax(-Fout, 0.0)) * val;
            }
        }
    }
    #pragma unroll
    for (int a = 0; a < 3 && a < g.dims; ++a) {
        const double* Gq = F.G + (long long)a * N;   // d u_a / d x (component q = 0)
        double GP = Gq[c];
        double flo, fhi;
        if (has_nb(g, a, 0, i, j, k)) {
            long long nc = c - g.stride[a];
            flo = (0.5 * (nuP + g.nu + F.nut[nc])) * (0.5 * (GP + Gq[nc])) * g.S[a];
        } else {
            flo = nuP * GP * g.S[a];
        }
        if (has_nb(g, a, 1, i, j, k)) {
            long long nc = c + g.stride[a];
            fhi = (0.5 * (nuP + g.nu + F.nut[nc])) * (0.5 * (GP + Gq[nc])) * g.S[a];
        } else {
            fhi = nuP * GP * g.S[a];
        }
        T += fhi - flo;
    }
    return bnd + T;
}

}  // namespace

// J = -sum over imposed rows of r
__global__ void k_adj_drag_value(Grid g, Fields F, Adj A) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[1] = {0.0};
    if (c < g.N) {
        uint16_t f = F.flags[c];
        if (fixed_row(f)) {
            int i, j, k;
            cell_ijk(g, c, i, j, k);
            const long long N = g.N;
            double r = A.AP[c] * drag_ut(g, F, c, f);
            #pragma unroll
            for (int s = 0; s < 6 && s < 2 * g.dims; ++s) {
                int d = s >> 1, side = s & 1;
                if (!has_nb(g, d, side, i, j, k)) continue;
                long long n = side ? c + g.stride[d] : c - g.stride[d];
                r += A.As[(long long)s * N + c] * drag_ut(g, F, n, F.flags[n]);
            }
            r -= drag_b0(g, F, c, i, j, k, f);
            r += g.V * grad_pr(g, F.p, F.p, 0.0, c, 0, i, j, k);
            v[0] = -r;
        }
    }
    grid_reduce<1, false>(v, F.partials, F.counters + 11, F.scal + SC_ADJ_J);
}

// Seed of the drag's derivative, laid out for the reverse-pass kernels that
// follow (k_adj_transpose, k_adj_gradu, k_adj_phi): with w = dJ/dr = -1 in
// imposed rows, b0-bar = -w (r holds -b0), bm-bar = -w (their p-bar is the
// transposed gradient of -V bm-bar, and r holds +V dp/dx), aP-bar and
// a_s-bar of the x row, and ut-bar gathered from the rows that read ut: into
// u-bar in free cells, into u_ib-bar in laminar-branch bc cells.
__global__ void k_adj_drag_seed(Grid g, Fields F, Adj A) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    const long long N = g.N;
    uint16_t f = F.flags[c];
    double w = fixed_row(f) ? -1.0 : 0.0;
    #pragma unroll
    for (int q = 0; q < 3 && q < g.dims; ++q) {
        A.b0b[q][c] = 0.0;
        A.bmb[q][c] = 0.0;
        A.aPb[q][c] = 0.0;
        A.fixb[q][c] = 0.0;
        A.xbu[q][c] = 0.0;
    }
    A.xbp[c] = 0.0;
    A.b0b[0][c] = -w;
    A.bmb[0][c] = -w;
    A.aPb[0][c] = w * drag_ut(g, F, c, f);
    double utb = w * A.AP[c];
    #pragma unroll
    for (int s = 0; s < 6 && s < 2 * g.dims; ++s) {
        int d = s >> 1, side = s & 1;
        double as = 0.0;
        if (has_nb(g, d, side, i, j, k)) {
            long long n = side ? c + g.stride[d] : c - g.stride[d];
            uint16_t fn = F.flags[n];
            as = w * drag_ut(g, F, n, fn);
            if (fixed_row(fn)) utb -= A.As[(long long)(s ^ 1) * N + n];
        }
        A.asb[(long long)s * N + c] = as;
    }
    if (tag_of(f) != TAG_IC) {
        if (f & F_AU) A.fixb[0][c] = utb;
        else A.xbu[0][c] = utb;
    }
}

// ---------------------------------------------------------------- mask of reading B
// With m = 1 - lambda the pressure right-hand side -m div(phiHbyA) depends
// on lambda directly: d rhs_P / d lambda_P = div_P(phiHbyA), and ps is the
// adjoint of that right-hand side, so dJ/dlambda_P += ps_P div_P(phiHbyA).
__global__ void k_adj_dlambda_mask(Grid g, Fields F, Adj A) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    double div = 0.0;
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        long long fl = face_lo(g, d, i, j, k);
        div += F.phiH[d][fl + face_stride(g, d)] - F.phiH[d][fl];
    }
    A.dlam[c] += A.ps[c] * div;
}

// ---------------------------------------------------------------- lambda chain
namespace {

// grad(lambda) at cell (i,j,k) as the geometry step takes it (central, one-sided
// at the domain edges): g_d = (lam[hi_d] - lam[lo_d]) * inv_d
__device__ void lam_grad(const Grid& g, const double* lam, int i, int j, int k, double gr[3], long long lo[3],
                         long long hi[3], double inv[3]) {
    int idx[3] = {i, j, k};
    long long c = ((long long)k * g.ny + j) * g.nx + i;
    for (int d = 0; d < 3; ++d) {
        lo[d] = hi[d] = c;
        if (g.n[d] == 1) { gr[d] = 0.0; inv[d] = 0.0; continue; }
        long long st = d == 0 ? 1 : (d == 1 ? g.nx : (long long)g.nx * g.ny);
        if (idx[d] == 0) { hi[d] = c + st; inv[d] = 1.0 / g.D[d]; }
        else if (idx[d] == g.n[d] - 1) { lo[d] = c - st; inv[d] = 1.0 / g.D[d]; }
        else { lo[d] = c - st; hi[d] = c + st; inv[d] = 1.0 / (2.0 * g.D[d]); }
        gr[d] = (lam[hi[d]] - lam[lo[d]]) * inv[d];
    }
}

// dJ/dlambda += (dJ/dn) . dn/dlambda for n = -grad/|grad| at (i,j,k); nothing
// where the geometry step took its fall-back normal (a constant)
__device__ void push_normal(const Grid& g, const double* lam, int i, int j, int k, const double cv[3],
                            double* dlam, double nout[3], bool* fallback) {
    double gr[3], inv[3];
    long long lo[3], hi[3];
    lam_grad(g, lam, i, j, k, gr, lo, hi, inv);
    double mag = sqrt((gr[0] * gr[0] + gr[1] * gr[1]) + gr[2] * gr[2]);
    *fallback = !(mag >= 1e-12 / g.h);
    if (*fallback) return;
    double n[3] = {-gr[0] / mag, -gr[1] / mag, -gr[2] / mag};
    for (int d = 0; d < 3; ++d) nout[d] = n[d];
    double cn = cv[0] * n[0] + cv[1] * n[1] + cv[2] * n[2];
    for (int b = 0; b < 3; ++b) {
        if (g.n[b] == 1) continue;
        double sb = -(cv[b] - cn * n[b]) / mag;
        if (sb == 0.0) continue;
        atomicAdd(dlam + hi[b], sb * inv[b]);
        atomicAdd(dlam + lo[b], -sb * inv[b]);
    }
}

// d |h atanh(1 - 2 l)| / d l
__device__ inline double dsigma_abs(double l, double h) {
    double x = 1.0 - 2.0 * l;
    double s = atanh(x) >= 0.0 ? 1.0 : -1.0;
    return s * h * (-2.0) / (1.0 - x * x);
}

// interpolated value and d/dt_d of the bi/trilinear stencil (b, t) of field f
__device__ void interp_dt(const Grid& g, const double* f, const int* b, const double* t, double& val,
                          double dv[3]) {
    val = 0.0;
    dv[0] = dv[1] = dv[2] = 0.0;
    for (int corner = 0; corner < 8; ++corner) {
        int cc[3] = {corner & 1, (corner >> 1) & 1, (corner >> 2) & 1};
        double w[3];
        int id[3];
        bool skip = false;
        for (int d = 0; d < 3; ++d) {
            if (g.n[d] == 1) {
                if (cc[d]) skip = true;
                w[d] = 1.0;
                id[d] = b[d];
            } else {
                w[d] = cc[d] ? t[d] : 1.0 - t[d];
                id[d] = b[d] + cc[d];
            }
        }
        if (skip) continue;
        double fv = f[((long long)id[2] * g.ny + id[1]) * g.nx + id[0]];
        val += w[0] * w[1] * w[2] * fv;
        for (int d = 0; d < 3; ++d) {
            if (g.n[d] == 1) continue;
            double pr = cc[d] ? 1.0 : -1.0;
            for (int e = 0; e < 3; ++e)
                if (e != d) pr *= w[e];
            dv[d] += pr * fv;
        }
    }
}

}  // namespace

// One thread per bc cell in the laminar branch (imposed u_ib): the adjoint of
// u_ib times du_ib/dlambda, pushed to the lambda cells it depends on.
__global__ void k_adj_dlambda(Grid g, Fields F, BcList bl, const double* __restrict__ lam, Adj A) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= bl.nbc) return;
    long long c = bl.cell[q];
    if (!au_row(F.flags[c])) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    double P[3] = {g.o[0] + ((double)i + 0.5) * g.D[0], g.o[1] + ((double)j + 0.5) * g.D[1],
                   g.o[2] + ((double)k + 0.5) * g.D[2]};
    const double h = g.h;
    double yp = bl.yp[q];
    double d1 = yp + h, d2 = yp + 2.0 * h;
    double dwS = -2.0 * h * h * (2.0 * yp + 3.0 * h) / (d1 * d1 * d2 * d2);
    double dw1 = 2.0 * h / (d1 * d1);
    double dw2 = -2.0 * h / (d2 * d2);
    double w1 = bl.w1[q], w2 = bl.w2[q];
    const double* nP = bl.n + 3 * q;
    const int* b1 = bl.b1 + 3 * q;
    const int* b2 = bl.b2 + 3 * q;
    const double* t1 = bl.t1 + 3 * q;
    const double* t2 = bl.t2 + 3 * q;
    // interpolation fractions move with n where they are not clamped
    double unc1[3], unc2[3];
    for (int d = 0; d < 3; ++d) {
        unc1[d] = unc2[d] = 0.0;
        if (g.n[d] == 1) continue;
        double r1 = (P[d] + h * nP[d] - g.o[d]) / g.D[d] - 0.5 - b1[d];
        double r2 = (P[d] + 2.0 * h * nP[d] - g.o[d]) / g.D[d] - 0.5 - b2[d];
        unc1[d] = (r1 >= 0.0 && r1 <= 1.0) ? h / g.D[d] : 0.0;
        unc2[d] = (r2 >= 0.0 && r2 <= 1.0) ? 2.0 * h / g.D[d] : 0.0;
    }
    double dUdy = 0.0, dUdn[3] = {0.0, 0.0, 0.0};
    #pragma unroll
    for (int qq = 0; qq < 3 && qq < g.dims; ++qq) {
        double fb = A.fixb[qq][c];
        if (fb == 0.0) continue;
        double v1, v2, dv1[3], dv2[3];
        interp_dt(g, F.u[qq], b1, t1, v1, dv1);
        interp_dt(g, F.u[qq], b2, t2, v2, dv2);
        dUdy += fb * (dwS * g.u_s[qq] + dw1 * v1 + dw2 * v2);
        for (int d = 0; d < 3; ++d) dUdn[d] += fb * (w1 * dv1[d] * unc1[d] + w2 * dv2[d] * unc2[d]);
    }
    double* dl = A.dlam;
    double nn[3];
    bool fbk;
    push_normal(g, lam, i, j, k, dUdn, dl, nn, &fbk);
    if (bl.clamped[q] || dUdy == 0.0) return;
    int cs = bl.cas[q];
    if (cs == 0) {
        atomicAdd(dl + c, dUdy * dsigma_abs(lam[c], h));
    } else if (cs == 1 && bl.nbr[q] >= 0) {
        long long Nc = bl.nbr[q];
        int iN, jN, kN;
        cell_ijk(g, Nc, iN, jN, kN);
        double NP[3] = {g.o[0] + ((double)iN + 0.5) * g.D[0], g.o[1] + ((double)jN + 0.5) * g.D[1],
                        g.o[2] + ((double)kN + 0.5) * g.D[2]};
        double lN = lam[Nc];
        double sN = fabs(h * atanh(1.0 - 2.0 * lN));
        // the value of n_N first (zero sensitivity pushed), then its derivative
        double zero[3] = {0.0, 0.0, 0.0}, nN[3] = {0.0, 0.0, 0.0};
        bool fbN;
        push_normal(g, lam, iN, jN, kN, zero, dl, nN, &fbN);
        double nn2 = fbN ? 1.0 : (nN[0] * nN[0] + nN[1] * nN[1]) + nN[2] * nN[2];
        atomicAdd(dl + Nc, dUdy * (-nn2) * dsigma_abs(lN, h));
        if (!fbN) {
            double cv[3];
            for (int d = 0; d < 3; ++d) cv[d] = dUdy * (P[d] - NP[d] - 2.0 * sN * nN[d]);
            push_normal(g, lam, iN, jN, kN, cv, dl, nN, &fbN);
        }
    }
}

// ---------------------------------------------------------------- launchers
void launch_adj_coef(const Grid& g, const Params& P, const Fields& F, const Adj& A, cudaStream_t s) {
    k_adj_coef<<<nblocks(g.N), BLOCK, 0, s>>>(g, P, F, A);
}
void launch_adj_update(const Grid& g, const Params& P, const Fields& F, const Level& L0, const Adj& A,
                       cudaStream_t s) {
    k_adj_update<<<nblocks(g.N), BLOCK, 0, s>>>(g, P, F, L0, A);
}
void launch_adj_pcg_init(const Grid& g, const Fields& Fa, const Level& L0, const double* rhs, int jacobi,
                         cudaStream_t s) {
    k_adj_pcg_init<<<nblocks(g.N), BLOCK, 0, s>>>(g, Fa, L0, rhs, jacobi);
}
void launch_adj_pressure(const Grid& g, const Fields& F, const Level& L0, const Adj& A, cudaStream_t s) {
    k_adj_pressure<<<nblocks(g.N), BLOCK, 0, s>>>(g, F, L0, A);
}
void launch_adj_hbya(const Grid& g, const Params& P, const Fields& F, const Adj& A, cudaStream_t s) {
    k_adj_hbya<<<nblocks(g.N), BLOCK, 0, s>>>(g, P, F, A);
}
void launch_adj_gs(const Grid& g, const Params& P, const Fields& F, const Adj& A, int colour, const double* Sin,
                   const double* Sout, int in_buf, cudaStream_t s) {
    k_adj_gs<<<nblocks(g.N), BLOCK, 0, s>>>(g, P, F, A, colour, Sin, Sout, in_buf);
}
void launch_adj_b0(const Grid& g, const Params& P, const Fields& F, const Adj& A, int buf, cudaStream_t s) {
    k_adj_b0<<<nblocks(g.N), BLOCK, 0, s>>>(g, P, F, A, buf);
}
void launch_adj_transpose(const Grid& g, const Fields& F, const Adj& A, cudaStream_t s) {
    k_adj_transpose<<<nblocks(g.N), BLOCK, 0, s>>>(g, F, A);
}
void launch_adj_gradu(const Grid& g, const Fields& F, const BcList& bl, const Adj& A, cudaStream_t s) {
    k_adj_gradu<<<nblocks(g.N), BLOCK, 0, s>>>(g, F, bl, A);
}
void launch_adj_phi(const Grid& g, const Fields& F, const Adj& A, cudaStream_t s) {
    k_adj_phi<<<nblocks(g.N), BLOCK, 0, s>>>(g, F, A);
}
void launch_adj_next(const Grid& g, const Fields& F, const Adj& A, int first, cudaStream_t s) {
    k_adj_next<<<nblocks(g.N), BLOCK, 0, s>>>(g, F, A, first);
}
void launch_adj_dlambda_mask(const Grid& g, const Fields& F, const Adj& A, cudaStream_t s) {
    if (g.mask_b) k_adj_dlambda_mask<<<nblocks(g.N), BLOCK, 0, s>>>(g, F, A);
}
void launch_adj_drag_value(const Grid& g, const Fields& F, const Adj& A, cudaStream_t s) {
    k_adj_drag_value<<<nblocks(g.N), BLOCK, 0, s>>>(g, F, A);
}
void launch_adj_drag_seed(const Grid& g, const Fields& F, const Adj& A, cudaStream_t s) {
    k_adj_drag_seed<<<nblocks(g.N), BLOCK, 0, s>>>(g, F, A);
}
void launch_adj_objective(const Grid& g, const Fields& F, const Adj& A, cudaStream_t s) {
    k_adj_objective<<<nblocks(g.N), BLOCK, 0, s>>>(g, F, A);
}
void launch_adj_dlambda(const Grid& g, const Fields& F, const BcList& bl, const double* lam, const Adj& A,
                        cudaStream_t s) {
    if (bl.nbc > 0) k_adj_dlambda<<<(bl.nbc + BLOCK - 1) / BLOCK, BLOCK, 0, s>>>(g, F, bl, lam, A);
}

}  // namespace hf
