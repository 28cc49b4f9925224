// common.cuh -- shared device definitions of the HFDIB SIMPLE kernels.
//
// Layout: cell arrays [nz][ny][nx], x fastest, cell index c = (k*ny + j)*nx + i.
// Face arrays (volumetric flux in the +d direction):
//   x faces [(nx+1) per row]: (k*ny + j)*(nx+1) + i is the face on the low-x side of cell i
//   y faces: (k*(ny+1) + j)*nx + i is the face on the low-y side of cell j
//   z faces: (k*ny + j)*nx + i     is the face on the low-z side of cell k
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hfdib.h"

namespace hf {

// wall-function constants (Sec. 2.5; standard published values)
constexpr double C_MU = 0.09;       // C_nu of Eq. (frictionvel)
constexpr double KAPPA = 0.41;
constexpr double E_WF = 9.8;
constexpr double BETA1_WF = 0.075;  // beta_1 of Eq. (omegaws)
constexpr double C_WF = 11.0;       // C of Eq. (kws)
constexpr double C_EPS2 = 1.9;      // C_eps2 of Eq. (kws)
constexpr double YPLUS_LAM = 11.0;  // Sec. 2.3

// standard k-epsilon
constexpr double KE_C1 = 1.44, KE_C2 = 1.92, KE_SIGK = 1.0, KE_SIGE = 1.3;
// k-omega SST (Menter) coefficients
constexpr double SST_AK1 = 0.85, SST_AK2 = 1.0, SST_AW1 = 0.5, SST_AW2 = 0.856;
constexpr double SST_G1 = 5.0 / 9.0, SST_G2 = 0.44, SST_B1 = 0.075, SST_B2 = 0.0828;
constexpr double SST_BSTAR = 0.09, SST_A1 = 0.31, SST_BB1 = 1.0, SST_C1 = 10.0;

// k-omega of Eq. (hfdibkomega): beta*, C_beta1, C_alpha1, 1/sigma_k1, 1/sigma_omega1
constexpr double KW_BSTAR = 0.09, KW_BETA = 0.072, KW_GAMMA = 0.52, KW_AK = 0.5, KW_AW = 0.5;
// realizable k-epsilon (Shih et al.)
constexpr double RKE_A0 = 4.0, RKE_C2 = 1.9, RKE_SIGK = 1.0, RKE_SIGE = 1.2;

constexpr double K_MIN = 1e-14, EPS_MIN = 1e-14, OMEGA_MIN = 1e-14;

// the second transported variable is eps (k-eps models) or omega (k-omega models)
__host__ __device__ inline bool eps_model(int model) {
    return model == HFDIB_KEPSILON || model == HFDIB_REALIZABLE_KE;
}

enum { TAG_FC = 0, TAG_BC = 1, TAG_IC = 2 };

// per-cell uint16 flags
constexpr uint16_t F_TAG = 3;           // bits 0-1: cell group
constexpr int F_CLOSED_SHIFT = 2;       // bits 2-7: closed boundary face on side s
constexpr uint16_t F_M = 1u << 8;       // lambda < 1: continuity enforced
constexpr uint16_t F_AU = 1u << 9;      // alpha_u = alpha_k = 1 (dynamic)

constexpr int BLOCK = 256;

struct Grid {
    int nx, ny, nz, dims;
    long long N;
    double iN;       // 1/N
    int n[3];
    double D[3];     // spacings
    double o[3];     // origin
    double S[3];     // face areas
    double SoD[3];   // S/Delta (interior face diffusion factor)
    double SoHD[3];  // S/(Delta/2) (boundary face diffusion factor)
    double iD[3];    // 1/Delta
    double V, h;     // cell volume, V^(1/3)
    int kind[6];     // hfdib_bc_kind per side
    double u_in[3], u_s[3], p_out;
    double nu;
    long long stride[3];
    long long nface[3];
    int mask_b;      // continuity mask: 0 reading A m = [lambda < 1], 1 reading B m = 1 - lambda
    int conv;        // momentum convection: 0 upwind, 1 linearUpwind, 2 vanLeer, 3 linearUpwind with a
                     // cell-limited gradient (deferred correction)
};

// m div(phiHbyA), the source of the pressure equation (Eq. hfdibrans_2 with
// its (1 - lambda) factor): reading A m = [lambda < 1] (flag F_M), reading B
// m = 1 - lambda
__device__ inline double masked_div(const Grid& g, const double* lam, uint16_t f, long long c, double div) {
    if (g.mask_b) return (1.0 - lam[c]) * div;
    return (f & F_M) ? div : 0.0;
}
__device__ inline double cont_mask(const Grid& g, const double* lam, uint16_t f, long long c) {
    if (g.mask_b) return 1.0 - lam[c];
    return (f & F_M) ? 1.0 : 0.0;
}

__host__ __device__ inline int tag_of(uint16_t f) { return f & F_TAG; }
__host__ __device__ inline bool closed_side(uint16_t f, int s) { return (f >> (F_CLOSED_SHIFT + s)) & 1u; }

// cell counts stay below 2^31 (checked at create), so 32-bit division suffices
__device__ inline void cell_ijk(const Grid& g, long long c, int& i, int& j, int& k) {
    unsigned int cc = (unsigned int)c, nx = (unsigned int)g.nx;
    unsigned int r = cc / nx;
    i = (int)(cc - r * nx);
    if (g.nz == 1) { j = (int)r; k = 0; return; }
    unsigned int ny = (unsigned int)g.ny;
    unsigned int kk = r / ny;
    j = (int)(r - kk * ny);
    k = (int)kk;
}

// Red-black passes launch one thread per x-pair of cells (cells 2p and 2p+1
// of a row, one of each colour; an odd row's last pair has one cell): the
// thread takes the cell of `colour`, so no lane of a warp is idle.
__host__ __device__ inline long long npairs(const Grid& g) { return (long long)((g.nx + 1) >> 1) * g.ny * g.nz; }
__device__ inline bool pair_cell(const Grid& g, long long p, int colour, long long& c, int& i, int& j, int& k) {
    unsigned int npx = (unsigned int)((g.nx + 1) >> 1);
    unsigned int pp = (unsigned int)p;
    unsigned int r = pp / npx;
    unsigned int pi = pp - r * npx;
    if (g.nz == 1) {
        j = (int)r;
        k = 0;
    } else {
        unsigned int ny = (unsigned int)g.ny;
        unsigned int kk = r / ny;
        j = (int)(r - kk * ny);
        k = (int)kk;
    }
    int i0 = 2 * (int)pi;
    i = i0 + ((i0 + j + k + colour) & 1);
    c = ((long long)k * g.ny + j) * g.nx + i;
    return i < g.nx;
}

// index of the low face of cell (i,j,k) in direction d; the high face is +fstride
__device__ inline long long face_lo(const Grid& g, int d, int i, int j, int k) {
    if (d == 0) return ((long long)k * g.ny + j) * (g.nx + 1) + i;
    if (d == 1) return ((long long)k * (g.ny + 1) + j) * g.nx + i;
    return ((long long)k * g.ny + j) * g.nx + i;
}
__device__ inline long long face_stride(const Grid& g, int d) {
    if (d == 0) return 1;
    if (d == 1) return g.nx;
    return (long long)g.nx * g.ny;
}

__device__ inline int coord(int d, int i, int j, int k) { return d == 0 ? i : (d == 1 ? j : k); }

// ---- boundary conditions -------------------------------------------------
// velocity component c on side s: true + value if the face is fixed-value
__device__ inline bool vel_fixed(const Grid& g, uint16_t f, int s, int c, double& val) {
    if (closed_side(f, s)) return false;
    int kind = g.kind[s];
    if (kind == HFDIB_BC_INLET) { val = g.u_in[c]; return true; }
    if (kind == HFDIB_BC_WALL) { val = 0.0; return true; }
    if (kind == HFDIB_BC_SLIP) { val = 0.0; return c == (s >> 1); }
    return false;
}
// scalar (k, eps, omega): fixed only on open inlet faces
__device__ inline bool scal_fixed(const Grid& g, uint16_t f, int s) {
    return !closed_side(f, s) && g.kind[s] == HFDIB_BC_INLET;
}
__device__ inline bool p_fixed(const Grid& g, int s) { return g.kind[s] == HFDIB_BC_OUTLET; }

// ---- block position -------------------------------------------------------
// The blocks that work on one problem: a plain launch gives the whole grid
// to one problem (block blockIdx.x of gridDim.x); a batched launch gives each
// problem its own consecutive range of blocks, and Pos is the block's place
// in its problem's range.  Kernel bodies index cells with Pos only, so a
// problem sees the same block partition, and reduces in the same order,
// alone or in a batch.
struct Pos {
    int bid;    // this block among its problem's blocks
    int nblk;   // the problem's blocks
};
__device__ __forceinline__ Pos grid_pos() { return Pos{(int)blockIdx.x, (int)gridDim.x}; }

// ---- deterministic grid reduction (last block finishes) -------------------
template <bool MAX>
__device__ inline double rop(double a, double b) { return MAX ? fmax(a, b) : a + b; }

// Reduce v[NV] over the problem's blocks.  Every block writes its partials;
// the block that finishes last combines all partials in a fixed order, so
// the result does not depend on scheduling.  blockDim.x must be BLOCK.
template <int NV, bool MAX>
__device__ void grid_reduce(double (&v)[NV], double* partials, unsigned int* counter, double* out,
                            Pos pos = grid_pos()) {
    __shared__ double sm[NV][BLOCK / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) x = rop<MAX>(x, __shfl_down_sync(0xffffffffu, x, o));
        if (lane == 0) sm[q][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double x = sm[q][0];
            for (int w = 1; w < BLOCK / 32; ++w) x = rop<MAX>(x, sm[q][w]);
            partials[(long long)q * pos.nblk + pos.bid] = x;
        }
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        last = (t == (unsigned int)pos.nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = MAX ? -1.0e308 : 0.0;
        for (int b = threadIdx.x; b < pos.nblk; b += BLOCK)
            x = rop<MAX>(x, __ldcg(&partials[(long long)q * pos.nblk + b]));
        for (int o = 16; o > 0; o >>= 1) x = rop<MAX>(x, __shfl_down_sync(0xffffffffu, x, o));
        if (lane == 0) sm[q][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double x = sm[q][0];
            for (int w = 1; w < BLOCK / 32; ++w) x = rop<MAX>(x, sm[q][w]);
            out[q] = x;
        }
        *counter = 0u;
    }
}

inline unsigned int nblocks(long long n) { return (unsigned int)((n + BLOCK - 1) / BLOCK); }

// Grid of the per-cell kernels that end in a grid-wide FP64 reduction: at most
// two blocks per SM, each thread looping over several cells, so the
// block-level shuffle tree (five FP64 adds per reduced value and thread, on a
// GPU with little FP64 throughput) is paid once per several cells.
inline unsigned int rblocks(long long n) {
    static int sms = 0;
    if (sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 1;
    }
    long long cap = 2LL * sms, b = nblocks(n);
    return (unsigned int)(b < cap ? b : cap);
}

}  // namespace hf
