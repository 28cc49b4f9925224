// turb.cu -- two-equation turbulence part of the sweep (Fig. simplehfdibrans):
// production and the P_ib assignment (Eq. omegaws), the eps / omega equation
// with its rows fixed to eps_ib / omega_ib where alpha_omega = 1 (Eq.
// alphaomega, "matrix manipulation"), the k equation with its rows fixed to
// k_ib where alpha_k = 1 followed by the k correction, and nu_t.
//
// Models (Sec. 2.1): standard k-epsilon (Launder-Spalding), k-omega SST
// (Menter), the k-omega model of Eq. hfdibkomega, and realizable k-epsilon
// (Shih et al.), with their published coefficients.  eq = 0 is eps (k-eps
// models) or omega (k-omega models), eq = 1 is k.
#include "common.cuh"
#include "kernels.cuh"
#include "batch.cuh"

namespace hf {

__device__ inline bool interior_t(const Grid& g, int d, int side, int i, int j, int k) {
    int pos = coord(d, i, j, k);
    return side ? pos < g.n[d] - 1 : pos > 0;
}

// Gauss-linear gradient of a turbulence scalar (open inlet faces carry xin)
__device__ inline double grad_s(const Grid& g, const double* x, uint16_t f, double xin, long long c, int d,
                                int i, int j, int k) {
    double xP = x[c];
    double lo, hi;
    if (interior_t(g, d, 0, i, j, k)) lo = 0.5 * (x[c - g.stride[d]] + xP);
    else lo = scal_fixed(g, f, 2 * d) ? xin : xP;
    if (interior_t(g, d, 1, i, j, k)) hi = 0.5 * (xP + x[c + g.stride[d]]);
    else hi = scal_fixed(g, f, 2 * d + 1) ? xin : xP;
    return (hi - lo) * g.iD[d];
}

// tanh of x >= 0: 1 for x >= 19.5, where tanh(x) = 1 - 2 e^(-2x) + ... is
// within half an ulp of 1 and rounds to 1 (the call is skipped there)
__device__ inline double tanh_pos(double x) { return x >= 19.5 ? 1.0 : tanh(x); }

// Menter's F2 from k, 1/omega and 1/y (reciprocals shared with the caller:
// an FP64 division is many FP64 operations on this GPU)
__device__ inline double sst_F2(double kk, double iw, double iy, double nu) {
    double sk = sqrt(kk);
    double arg2 = fmin(fmax(2.0 * sk * iw * iy * (1.0 / SST_BSTAR), 500.0 * nu * iy * iy * iw), 100.0);
    return tanh_pos(arg2 * arg2);
}

__global__ void k_inv_wall_distance(Grid g, Fields F) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < g.N) F.iyw[c] = 1.0 / fmax(F.ywall[c], 1e-3 * g.h);
}
void launch_inv_wall_distance(const Grid& g, const Fields& F, cudaStream_t s) {
    k_inv_wall_distance<<<nblocks(g.N), BLOCK, 0, s>>>(g, F);
}

// ---------------------------------------------------------------- a9 production
__device__ __forceinline__ void b_turb_prep(Pos pos, const Grid& g, const Params& P, const Fields& F) {
    long long c = (long long)pos.bid * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    uint16_t f = F.flags[c];
    // S2 = 2 S:S with S = (G + G^T)/2: the diagonal gives 2 G_aa^2, each
    // off-diagonal pair (G_ab + G_ba)^2 (a third of the FP64 operations of
    // the full double sum)
    double Sd = 0.0, So = 0.0;
    #pragma unroll
    for (int a = 0; a < 3 && a < g.dims; ++a) {
        const double gaa = F.G[(long long)(4 * a) * g.N + c];
        Sd += gaa * gaa;
        #pragma unroll
        for (int b = a + 1; b < 3 && b < g.dims; ++b) {
            const double o = F.G[(long long)(3 * a + b) * g.N + c] + F.G[(long long)(3 * b + a) * g.N + c];
            So += o * o;
        }
    }
    const double S2 = 2.0 * Sd + So;
    double nut = F.nut[c];
    double Pk = tag_of(f) == TAG_IC ? 0.0 : nut * S2;
    F.S2[c] = S2;
    F.Pk[c] = Pk;
    double kold = F.k[c], wold = F.w[c];
    double V = g.V;
    if (P.model == HFDIB_KEPSILON) {
        double ratio = wold / fmax(kold, K_MIN);
        F.gam[c] = g.nu + nut * (1.0 / KE_SIGE);
        F.sp[c] = KE_C2 * ratio * V;
        F.src[c] = KE_C1 * (nut * S2) * ratio * V;
        F.gamk[c] = g.nu + nut * (1.0 / KE_SIGK);
        if (F.mixed) { F.gam32[c] = (float)F.gam[c]; F.gamk32[c] = (float)F.gamk[c]; }
    } else if (P.model == HFDIB_KOMEGA) {
        // Eq. hfdibkomega: omega source C_alpha1 (omega/k) P_k, sink C_beta1 omega^2
        F.gam[c] = g.nu + KW_AW * nut;
        F.sp[c] = KW_BETA * wold * V;
        F.src[c] = KW_GAMMA * wold / fmax(kold, K_MIN) * (nut * S2) * V;
        F.gamk[c] = g.nu + KW_AK * nut;
        if (F.mixed) { F.gam32[c] = (float)F.gam[c]; F.gamk32[c] = (float)F.gamk[c]; }
    } else if (P.model == HFDIB_REALIZABLE_KE) {
        // S_ij, Omega_ij of grad u; W = S_ij S_jk S_ki / S~^3 (0 where S~ = 0),
        // A_s = sqrt(6) cos(acos(sqrt(6) W)/3), U* = sqrt(S:S + Omega:Omega)
        double Sm[3][3], SS = 0.0, OO = 0.0;
        #pragma unroll
        for (int a = 0; a < 3; ++a)
            #pragma unroll
            for (int b = 0; b < 3; ++b) {
                double gab = (a < g.dims && b < g.dims) ? F.G[(long long)(3 * a + b) * g.N + c] : 0.0;
                double gba = (a < g.dims && b < g.dims) ? F.G[(long long)(3 * b + a) * g.N + c] : 0.0;
                Sm[a][b] = 0.5 * (gab + gba);
                double o = 0.5 * (gab - gba);
                SS += Sm[a][b] * Sm[a][b];
                OO += o * o;
            }
        double SSS = 0.0;
        #pragma unroll
        for (int a = 0; a < 3; ++a)
            #pragma unroll
            for (int b = 0; b < 3; ++b)
                #pragma unroll
                for (int d = 0; d < 3; ++d) SSS += Sm[a][b] * Sm[b][d] * Sm[d][a];
        double St = sqrt(SS);
        double W = St > 0.0 ? SSS / (St * St * St) : 0.0;
        double arg = fmin(fmax(sqrt(6.0) * W, -1.0), 1.0);
        // cos(acos(arg)/3) through cospi: its argument is in [0, 1/3], and
        // cospi needs no large-argument reduction (no local-memory path)
        double As = sqrt(6.0) * cospi(acos(arg) * (1.0 / (3.0 * 3.14159265358979323846)));
        F.asus[c] = As * sqrt(SS + OO);
        double S = sqrt(S2);
        double kk = fmax(kold, K_MIN);
        double eta = S * kk / wold;
        double C1 = fmax(0.43, eta / (eta + 5.0));
        F.gam[c] = g.nu + nut * (1.0 / RKE_SIGE);
        F.sp[c] = RKE_C2 * wold / (kk + sqrt(g.nu * wold)) * V;
        F.src[c] = C1 * S * wold * V;
        F.gamk[c] = g.nu + nut * (1.0 / RKE_SIGK);
        if (F.mixed) { F.gam32[c] = (float)F.gam[c]; F.gamk32[c] = (float)F.gamk[c]; }
    } else {
        double gk = 0.0;
        #pragma unroll
        for (int d = 0; d < 3 && d < g.dims; ++d)
            gk += grad_s(g, F.k, f, P.k_in, c, d, i, j, k) * grad_s(g, F.w, f, P.w_in, c, d, i, j, k);
        double kk = fmax(kold, K_MIN), ww = wold;
        // reciprocals once (1/y is stored): FP64 division is many FP64
        // operations on this GPU
        double iw = 1.0 / ww, iy = F.iyw[c];
        double CDkw = 2.0 * SST_AW2 * gk * iw;
        double CDp = fmax(CDkw, 1e-10);
        double sk = sqrt(kk);
        double t_k = sk * iw * iy * (1.0 / SST_BSTAR);     // sqrt(k) / (beta* omega y)
        double t_nu = 500.0 * g.nu * iy * iy * iw;          // 500 nu / (y^2 omega)
        double arg1 = fmin(fmax(t_k, t_nu), 4.0 * SST_AW2 * kk * iy * iy / CDp);
        double F1 = tanh_pos(arg1 * arg1 * arg1 * arg1);
        double arg2 = fmin(fmax(2.0 * t_k, t_nu), 100.0);   // F2 of the same k, omega, y
        double F2 = tanh_pos(arg2 * arg2);
        double gamma = F1 * SST_G1 + (1.0 - F1) * SST_G2;
        double beta = F1 * SST_B1 + (1.0 - F1) * SST_B2;
        double GbyNu = fmin(S2, (SST_C1 / SST_A1) * SST_BSTAR * wold * fmax(SST_A1 * wold, SST_BB1 * F2 * sqrt(S2)));
        double cdc = (F1 - 1.0) * CDkw * iw;
        F.gam[c] = g.nu + (F1 * SST_AW1 + (1.0 - F1) * SST_AW2) * nut;
        F.sp[c] = beta * wold * V + (cdc > 0.0 ? cdc : 0.0) * V;
        F.src[c] = gamma * GbyNu * V - (cdc > 0.0 ? 0.0 : cdc) * wold * V;
        F.gamk[c] = g.nu + (F1 * SST_AK1 + (1.0 - F1) * SST_AK2) * nut;
        if (F.mixed) { F.gam32[c] = (float)F.gam[c]; F.gamk32[c] = (float)F.gamk[c]; }
    }
}
__global__ void k_turb_prep(Grid g, Params P, Fields F) {
    b_turb_prep(grid_pos(), g, P, F);
}

// P_ib in the log branch of bc cells: kappa nu y+ |n.grad u|^2 / ln^2(E y+)
__device__ __forceinline__ void b_bc_prod(Pos pos, const Grid& g, const BcList& bl, const Fields& F) {
    int q = pos.bid * blockDim.x + threadIdx.x;
    if (q >= bl.nbc) return;
    if (bl.lamb[q]) return;
    long long c = bl.cell[q];
    double dudn2 = 0.0;
    #pragma unroll
    for (int b = 0; b < 3 && b < g.dims; ++b) {
        double comp = 0.0;
        #pragma unroll
        for (int a = 0; a < 3 && a < g.dims; ++a) comp += bl.n[3 * q + a] * F.G[(long long)(3 * a + b) * g.N + c];
        dudn2 += comp * comp;
    }
    // y+ > y+_lam in the log branch; the max only matters for cells kept
    // there by the one-way switch option
    double yp = fmax(bl.yplus[q], YPLUS_LAM);
    double L = log(E_WF * yp);
    F.Pk[c] = KAPPA * g.nu * yp * dudn2 / (L * L);
}
__global__ void k_bc_prod(Grid g, BcList bl, Fields F) {
    b_bc_prod(grid_pos(), g, bl, F);
}

// ---------------------------------------------------------------- scalar rows
__device__ inline bool scal_row_fixed(const Grid& g, const Fields& F, int eq, long long c, double& v) {
    uint16_t f = F.flags[c];
    int tag = tag_of(f);
    if (eq == 0) {
        if (tag == TAG_IC) { v = F.scal[SC_WMAX]; return true; }
        if (tag == TAG_BC) { v = F.wib[c]; return true; }
        return false;
    }
    if (tag == TAG_IC) { v = 0.0; return true; }
    if (f & F_AU) { v = F.kib[c]; return true; }
    return false;
}

template <typename T>
struct ScalRowT {
    T aP, bnd;
    T aPi;        // the interior-face part of aP (= -sum a)
    T a[6];
    long long nb[6];
    bool has[6];
};
using ScalRow = ScalRowT<double>;

// transport row of a turbulence scalar; T = double (operator) or float
// (FP32 smoother of the mixed path, from FP32 mirrors)
template <typename T>
__device__ void scal_row_t(const Grid& g, T* const* phi, const T* gam, double xin, long long c, int i, int j,
                           int k, uint16_t f, ScalRowT<T>& R) {
    T gP = gam[c];
    T aPi = T(0), aPb = T(0);
    R.bnd = T(0);
    #pragma unroll
    for (int d = 0; d < 3 && d < g.dims; ++d) {
        long long fl = face_lo(g, d, i, j, k);
        long long fs = face_stride(g, d);
        const T hSoD = (T)(0.5 * g.SoD[d]);
        for (int side = 0; side < 2; ++side) {
            int s = 2 * d + side;
            T Fb = phi[d][fl + side * fs];
            T Fout = side ? Fb : -Fb;
            if (interior_t(g, d, side, i, j, k)) {
                long long nc = side ? c + g.stride[d] : c - g.stride[d];
                // Dif = (gamma_P + gamma_N)/2 S/Delta; aP gains
                // max(-Fout, 0) + Dif = -a (five operations a face)
                T Dif = (gP + gam[nc]) * hSoD;
                R.a[s] = fmin(Fout, T(0)) - Dif;
                R.nb[s] = nc;
                R.has[s] = true;
                aPi -= R.a[s];
            } else {
                R.a[s] = T(0);
                R.nb[s] = c;
                R.has[s] = false;
                if (scal_fixed(g, f, s)) {
                    T coef = gP * (T)g.SoHD[d] + fmax(-Fout, T(0));
                    aPb += coef;
                    R.bnd += coef * (T)xin;
                }
            }
        }
    }
    R.aPi = aPi;
    R.aP = aPi + aPb;
}

__device__ inline void scal_row(const Grid& g, const Fields& F, const double* gam, double xin, long long c, int i,
                                int j, int k, uint16_t f, ScalRow& R) {
    scal_row_t<double>(g, F.phi, gam, xin, c, i, j, k, f, R);
}

__device__ __forceinline__ void b_scal_asm(Pos pos, const Grid& g, const Params& P, const Fields& F, int eq) {
    double red[3] = {0.0, 0.0, 0.0};
    double* x = eq == 0 ? F.w : F.k;
    const double* gam = eq == 0 ? F.gam : F.gamk;
    double xin = eq == 0 ? P.w_in : P.k_in;
    for (long long c = (long long)pos.bid * blockDim.x + threadIdx.x; c < g.N;
         c += (long long)pos.nblk * blockDim.x) {
        int i, j, k;
        cell_ijk(g, c, i, j, k);
        uint16_t f = F.flags[c];
        ScalRow R;
        scal_row(g, F, gam, xin, c, i, j, k, f, R);
        double aP = R.aP + F.sp[c];
        double b = R.bnd + F.src[c];
        double xold = x[c];
        F.bt[c] = b + P.rlx_t * aP * xold;
        F.diag[c] = aP * P.iurf_t;
        if (F.mixed) F.diag32[c] = (float)(aP * P.iurf_t);
        double fv;
        if (scal_row_fixed(g, F, eq, c, fv)) {
            // imposed rows start at their imposed values (only neighbours'
            // substituted values are read below, so this write is race-free)
            x[c] = fv;
            if (F.mixed) F.r32[0][c] = 0.0f;
        } else {
            double Ax = aP * xold;
            // row sum: aP + sum a = aP - aPi (the interior part cancels)
            const double A1 = aP - R.aPi;
            #pragma unroll
            for (int s = 0; s < 6 && s < 2 * g.dims; ++s) {
                if (!R.has[s]) continue;
                double xN;
                if (!scal_row_fixed(g, F, eq, R.nb[s], xN)) xN = x[R.nb[s]];
                Ax += R.a[s] * xN;
            }
            double xbar = F.scal[eq == 0 ? SC_SUM_W : SC_SUM_K] * g.iN;
            red[0] += fabs(b - Ax);
            red[1] += fabs(Ax - A1 * xbar);
            red[2] += fabs(b - A1 * xbar);
            // defect of the relaxed system at x_old (relaxation terms cancel)
            if (F.mixed) F.r32[0][c] = (float)(b - Ax);
        }
    }
    grid_reduce<3, false>(red, F.partials, F.counters + 7, F.scal + (eq == 0 ? SC_RES_W : SC_RES_K), pos);
}
__global__ void k_scal_asm(Grid g, Params P, Fields F, int eq) {
    b_scal_asm(grid_pos(), g, P, F, eq);
}

__device__ __forceinline__ void b_scal_smooth(Pos pos, const Grid& g, const Params& P, const Fields& F, int eq,
                                              int colour) {
    long long p = (long long)pos.bid * blockDim.x + threadIdx.x;
    if (p >= npairs(g)) return;
    long long c;
    int i, j, k;
    if (!pair_cell(g, p, colour, c, i, j, k)) return;
    double* x = eq == 0 ? F.w : F.k;
    double fv;
    if (scal_row_fixed(g, F, eq, c, fv)) {
        x[c] = fv;
        return;
    }
    const double* gam = eq == 0 ? F.gam : F.gamk;
    double xin = eq == 0 ? P.w_in : P.k_in;
    uint16_t f = F.flags[c];
    ScalRow R;
    scal_row(g, F, gam, xin, c, i, j, k, f, R);
    double acc = F.bt[c];
    #pragma unroll
    for (int s = 0; s < 6 && s < 2 * g.dims; ++s)
        if (R.has[s]) acc -= R.a[s] * x[R.nb[s]];
    x[c] = acc / F.diag[c];
}
__global__ void k_scal_smooth(Grid g, Params P, Fields F, int eq, int colour) {
    b_scal_smooth(grid_pos(), g, P, F, eq, colour);
}

// FP32 red-black sweep on the correction (mixed path): diag d_P + sum a_N d_N
// = r (FP64 defect rounded); d = 0 on imposed rows
__device__ __forceinline__ void b_scal_smooth32(Pos pos, const Grid& g, const Params& P, const Fields& F, int eq,
                                                int colour, int zero_init) {
    long long p = (long long)pos.bid * blockDim.x + threadIdx.x;
    if (p >= npairs(g)) return;
    long long c;
    int i, j, k;
    if (!pair_cell(g, p, colour, c, i, j, k)) return;
    double fv;
    if (scal_row_fixed(g, F, eq, c, fv)) {
        F.d32[0][c] = 0.0f;
        return;
    }
    const float* gam = eq == 0 ? F.gam32 : F.gamk32;
    double xin = eq == 0 ? P.w_in : P.k_in;
    uint16_t f = F.flags[c];
    ScalRowT<float> R;
    scal_row_t<float>(g, F.phi32, gam, xin, c, i, j, k, f, R);
    float acc = F.r32[0][c];
    if (!zero_init)
        #pragma unroll
        for (int s = 0; s < 6 && s < 2 * g.dims; ++s)
            if (R.has[s]) acc -= R.a[s] * F.d32[0][R.nb[s]];
    F.d32[0][c] = acc / F.diag32[c];
}
// six resident blocks per SM (40 registers): the half sweeps are bound by
// the latency of their global loads, so more warps in flight pay
__global__ void __launch_bounds__(BLOCK, 6) k_scal_smooth32(Grid g, Params P, Fields F, int eq, int colour, int zero_init) {
    b_scal_smooth32(grid_pos(), g, P, F, eq, colour, zero_init);
}

// after the eps/omega solve: bound it, set the k-equation sink and source
__device__ __forceinline__ void b_k_prep(Pos pos, const Grid& g, const Params& P, const Fields& F) {
    long long c = (long long)pos.bid * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    double w = F.w[c];
    if (F.mixed) w += (double)F.d32[0][c];   // apply the FP32 correction
    double wmin = eps_model(P.model) ? EPS_MIN : OMEGA_MIN;
    w = fmax(w, wmin);
    F.w[c] = w;
    double kold = F.k[c];
    if (eps_model(P.model)) {
        F.sp[c] = w / fmax(kold, K_MIN) * g.V;
        F.src[c] = F.Pk[c] * g.V;
    } else if (P.model == HFDIB_KOMEGA) {
        F.sp[c] = KW_BSTAR * w * g.V;
        F.src[c] = F.Pk[c] * g.V;
    } else {
        F.sp[c] = SST_BSTAR * w * g.V;
        F.src[c] = fmin(F.Pk[c], SST_C1 * SST_BSTAR * kold * w) * g.V;
    }
}
__global__ void k_k_prep(Grid g, Params P, Fields F) {
    b_k_prep(grid_pos(), g, P, F);
}

// bound k, apply the k correction (Eq. corru for k), update nu_t
__device__ __forceinline__ void b_turb_final(Pos pos, const Grid& g, const Params& P, const Fields& F) {
    long long c = (long long)pos.bid * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    uint16_t f = F.flags[c];
    double kx = F.k[c];
    if (F.mixed) kx += (double)F.d32[0][c];  // apply the FP32 correction
    double k = fmax(kx, K_MIN);
    if (tag_of(f) == TAG_IC) k = k + (0.0 - k);
    else if (f & F_AU) k = k + (F.kib[c] - k);
    F.k[c] = k;
    double w = F.w[c];
    double nut;
    if (P.model == HFDIB_KEPSILON) {
        nut = C_MU * k * k / w;
        F.w2[c] = w / (C_MU * fmax(k, K_MIN));
    } else if (P.model == HFDIB_REALIZABLE_KE) {
        // C_mu k^2/eps = k^2 / (A0 eps + A_s U* k)
        nut = k * k / (RKE_A0 * w + F.asus[c] * k);
        F.w2[c] = w / (C_MU * fmax(k, K_MIN));
    } else if (P.model == HFDIB_KOMEGA) {
        nut = k / w;
        F.w2[c] = C_MU * k * w;
    } else {
        double F2 = sst_F2(fmax(k, K_MIN), 1.0 / w, F.iyw[c], g.nu);
        nut = SST_A1 * k / fmax(SST_A1 * w, SST_BB1 * F2 * sqrt(F.S2[c]));
        F.w2[c] = C_MU * k * w;
    }
    F.nut[c] = nut;
    if (F.mixed) F.nut32[c] = (float)nut;
}
__global__ void k_turb_final(Grid g, Params P, Fields F) {
    b_turb_final(grid_pos(), g, P, F);
}

// ---------------------------------------------------------------- launchers
void launch_turb_prep(const Grid& g, const Params& P, const Fields& F, cudaStream_t s) {
    k_turb_prep<<<nblocks(g.N), BLOCK, 0, s>>>(g, P, F);
}
void launch_bc_prod(const Grid& g, const BcList& bl, const Fields& F, cudaStream_t s) {
    if (bl.nbc == 0) return;
    // one warp per block, as for the imposed fields (FP64 work per bc cell)
    k_bc_prod<<<(unsigned int)((bl.nbc + 31) / 32), 32, 0, s>>>(g, bl, F);
}
void launch_scal_asm(const Grid& g, const Params& P, const Fields& F, int eq, cudaStream_t s) {
    k_scal_asm<<<rblocks(g.N), BLOCK, 0, s>>>(g, P, F, eq);
}
void launch_scal_smooth(const Grid& g, const Params& P, const Fields& F, int eq, int colour,
                        cudaStream_t s) {
    k_scal_smooth<<<nblocks(npairs(g)), BLOCK, 0, s>>>(g, P, F, eq, colour);
}
void launch_scal_smooth32(const Grid& g, const Params& P, const Fields& F, int eq, int colour, int zero_init,
                          cudaStream_t s) {
    k_scal_smooth32<<<nblocks(npairs(g)), BLOCK, 0, s>>>(g, P, F, eq, colour, zero_init);
}
void launch_k_prep(const Grid& g, const Params& P, const Fields& F, cudaStream_t s) {
    k_k_prep<<<nblocks(g.N), BLOCK, 0, s>>>(g, P, F);
}
void launch_turb_final(const Grid& g, const Params& P, const Fields& F, cudaStream_t s) {
    k_turb_final<<<nblocks(g.N), BLOCK, 0, s>>>(g, P, F);
}

// ---------------------------------------------------------------- batched launches
struct OpTurbPrep {
    __device__ void operator()(Pos p, const SweepProblem& s) const { b_turb_prep(p, s.g, s.P, s.F); }
};
struct OpBcProd {
    __device__ void operator()(Pos p, const SweepProblem& s) const { b_bc_prod(p, s.g, s.bl, s.F); }
};
struct OpScalAsm {
    int eq;
    __device__ void operator()(Pos p, const SweepProblem& s) const { b_scal_asm(p, s.g, s.P, s.F, eq); }
};
struct OpScalSmooth {
    int eq, colour;
    __device__ void operator()(Pos p, const SweepProblem& s) const { b_scal_smooth(p, s.g, s.P, s.F, eq, colour); }
};
struct OpScalSmooth32 {
    int eq, colour, zero_init;
    __device__ void operator()(Pos p, const SweepProblem& s) const {
        b_scal_smooth32(p, s.g, s.P, s.F, eq, colour, zero_init);
    }
};
struct OpKPrep {
    __device__ void operator()(Pos p, const SweepProblem& s) const { b_k_prep(p, s.g, s.P, s.F); }
};
struct OpTurbFinal {
    __device__ void operator()(Pos p, const SweepProblem& s) const { b_turb_final(p, s.g, s.P, s.F); }
};
void launchb_turb_prep(const BatchTab& T, const int* tot, cudaStream_t s) {
    k_batched<BK_CELLS, OpTurbPrep><<<tot[BK_CELLS], BLOCK, 0, s>>>(T, OpTurbPrep{});
}
void launchb_bc_prod(const BatchTab& T, const int* tot, cudaStream_t s) {
    if (tot[BK_BC] > 0) k_batched<BK_BC, OpBcProd><<<tot[BK_BC], BLOCK, 0, s>>>(T, OpBcProd{});
}
void launchb_scal_asm(const BatchTab& T, const int* tot, int eq, cudaStream_t s) {
    k_batched<BK_REDUCE, OpScalAsm><<<tot[BK_REDUCE], BLOCK, 0, s>>>(T, OpScalAsm{eq});
}
void launchb_scal_smooth(const BatchTab& T, const int* tot, int eq, int colour, cudaStream_t s) {
    k_batched<BK_PAIRS, OpScalSmooth><<<tot[BK_PAIRS], BLOCK, 0, s>>>(T, OpScalSmooth{eq, colour});
}
void launchb_scal_smooth32(const BatchTab& T, const int* tot, int eq, int colour, int zero_init, cudaStream_t s) {
    k_batched<BK_PAIRS, OpScalSmooth32><<<tot[BK_PAIRS], BLOCK, 0, s>>>(T, OpScalSmooth32{eq, colour, zero_init});
}
void launchb_k_prep(const BatchTab& T, const int* tot, cudaStream_t s) {
    k_batched<BK_CELLS, OpKPrep><<<tot[BK_CELLS], BLOCK, 0, s>>>(T, OpKPrep{});
}
void launchb_turb_final(const BatchTab& T, const int* tot, cudaStream_t s) {
    k_batched<BK_CELLS, OpTurbFinal><<<tot[BK_CELLS], BLOCK, 0, s>>>(T, OpTurbFinal{});
}

}  // namespace hf
