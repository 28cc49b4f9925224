// krylov.cu -- restarted GMRES for the adjoint fixed point.
//
// The adjoint psi of the converged sweep solves (I - M) psi = b with
// M = G_x^T (one reverse pass of the sweep, adjoint.cu) and b = J_x^T.  The
// plain reverse fixed point psi <- M psi + b converges at the rate of the
// forward SIMPLE iteration; GMRES(m) on the same linear system reaches the
// same psi in far fewer passes.  Vectors are the flat adjoint state
// (u components, p, face fluxes).  Orthogonalisation is classical Gram-Schmidt
// applied twice (CGS2), so each Arnoldi step costs two multi-dot and two
// multi-axpy launches.  The small Hessenberg problem (Givens rotations,
// back substitution) runs in single-thread kernels; the host only reads the
// residual estimate.
#include "common.cuh"
#include "kernels.cuh"

namespace hf {

namespace {

__device__ inline double block_sum(double v, double* sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
    return t;  // valid in thread 0
}

}  // namespace

// out = a - b
__global__ void k_vsub(long long n, const double* __restrict__ a, const double* __restrict__ b, double* out) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        out[e] = a[e] - b[e];
}

// out = a - b + c
__global__ void k_vsub_add(long long n, const double* __restrict__ a, const double* __restrict__ b,
                           const double* __restrict__ c, double* out) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        out[e] = (a[e] - b[e]) + c[e];
}

// out[i] = <w, V_i>, i < k; per-block partials in fixed order, the last block
// to finish sums them (deterministic)
__global__ void k_mdot(long long n, const double* __restrict__ w, const double* __restrict__ V, long long ldv, int k,
                       double* partials, unsigned int* counter, double* out) {
    __shared__ double sm[32];
    __shared__ bool last;
    for (int i = 0; i < k; ++i) {
        const double* Vi = V + (long long)i * ldv;
        double s = 0.0;
        for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
            s += w[e] * Vi[e];
        double t = block_sum(s, sm);
        if (threadIdx.x == 0) partials[(long long)i * gridDim.x + blockIdx.x] = t;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int tk = atomicAdd(counter, 1u);
        last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        double t = 0.0;
        for (unsigned int b = 0; b < gridDim.x; ++b) t += __ldcg(&partials[(long long)i * gridDim.x + b]);
        out[i] = t;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// w += sgn * sum_{i<k} c_i V_i
__global__ void k_maxpy(long long n, double* w, const double* __restrict__ V, long long ldv, int k,
                        const double* __restrict__ c, double sgn) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < k; ++i) acc += c[i] * V[(long long)i * ldv + e];
        w[e] += sgn * acc;
    }
}

// dst = src / sqrt(*nrm2)  (nrm2 > 0), else 0
__global__ void k_vnormalize(long long n, const double* __restrict__ src, double* dst, const double* nrm2) {
    double s = *nrm2;
    double f = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        dst[e] = src[e] * f;
}

// Start of a cycle: g = (beta, 0, ...), beta = sqrt(*nrm2); st[0] = beta
__global__ void k_gmres_start(int m, const double* nrm2, double* gv, double* st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double beta = sqrt(fmax(*nrm2, 0.0));
    for (int i = 0; i <= m; ++i) gv[i] = 0.0;
    gv[0] = beta;
    st[0] = beta;
}

// Column j of the Hessenberg matrix (H column-major, leading dimension m+1):
// H[0..j, j] = h1 + h2 (both Gram-Schmidt passes), H[j+1, j] = |w|; the
// previous rotations are applied, a new one zeroes H[j+1, j], g is rotated.
// st[1] = |g[j+1]| (residual norm estimate), st[2] = H[j+1, j] before rotation.
__global__ void k_gmres_column(int j, int m, double* H, const double* h1, const double* h2, const double* nrm2,
                               double* cs, double* sn, double* gv, double* st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double* col = H + (long long)j * (m + 1);
    for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
    double hn = sqrt(fmax(*nrm2, 0.0));
    col[j + 1] = hn;
    st[2] = hn;
    for (int i = 0; i < j; ++i) {
        double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
    }
    double a = col[j], b = col[j + 1];
    double r = sqrt(a * a + b * b);
    double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
    cs[j] = c;
    sn[j] = s;
    col[j] = r;
    col[j + 1] = 0.0;
    double g0 = gv[j];
    gv[j] = c * g0;
    gv[j + 1] = -s * g0;
    st[1] = fabs(gv[j + 1]);
}

// y = R^{-1} g over the first k columns (back substitution)
__global__ void k_gmres_y(int k, int m, const double* H, const double* gv, double* y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double s = gv[i];
        for (int l = i + 1; l < k; ++l) s -= H[(long long)l * (m + 1) + i] * y[l];
        double d = H[(long long)i * (m + 1) + i];
        y[i] = d != 0.0 ? s / d : 0.0;
    }
}

// ---------------------------------------------------------------- launchers
namespace {
inline int vgrid(long long n) {
    long long b = (n + BLOCK - 1) / BLOCK;
    return (int)(b < 1024 ? (b < 1 ? 1 : b) : 1024);
}
}  // namespace

void launch_vsub(long long n, const double* a, const double* b, double* out, cudaStream_t s) {
    k_vsub<<<vgrid(n), BLOCK, 0, s>>>(n, a, b, out);
}
void launch_vsub_add(long long n, const double* a, const double* b, const double* c, double* out, cudaStream_t s) {
    k_vsub_add<<<vgrid(n), BLOCK, 0, s>>>(n, a, b, c, out);
}
int mdot_grid(long long n) { return vgrid(n); }
void launch_mdot(long long n, const double* w, const double* V, long long ldv, int k, double* partials,
                 unsigned int* counter, double* out, cudaStream_t s) {
    k_mdot<<<vgrid(n), BLOCK, 0, s>>>(n, w, V, ldv, k, partials, counter, out);
}
void launch_maxpy(long long n, double* w, const double* V, long long ldv, int k, const double* c, double sgn,
                  cudaStream_t s) {
    k_maxpy<<<vgrid(n), BLOCK, 0, s>>>(n, w, V, ldv, k, c, sgn);
}
void launch_vnormalize(long long n, const double* src, double* dst, const double* nrm2, cudaStream_t s) {
    k_vnormalize<<<vgrid(n), BLOCK, 0, s>>>(n, src, dst, nrm2);
}
void launch_gmres_start(int m, const double* nrm2, double* gv, double* st, cudaStream_t s) {
    k_gmres_start<<<1, 32, 0, s>>>(m, nrm2, gv, st);
}
void launch_gmres_column(int j, int m, double* H, const double* h1, const double* h2, const double* nrm2, double* cs,
                         double* sn, double* gv, double* st, cudaStream_t s) {
    k_gmres_column<<<1, 32, 0, s>>>(j, m, H, h1, h2, nrm2, cs, sn, gv, st);
}
void launch_gmres_y(int k, int m, const double* H, const double* gv, double* y, cudaStream_t s) {
    k_gmres_y<<<1, 32, 0, s>>>(k, m, H, gv, y);
}

}  // namespace hf
