// noalloc.cu -- allocation-free variant of the cell-group classification and
// the ordered boundary-cell compaction (the scratch-using part of a0).
//
// Some callers cannot allocate device memory at the moment they need the
// immersed-boundary cell groups: a process whose device memory is owned by
// another framework's pool (allocating behind its back would break its
// accounting), code that runs under a fixed memory budget, or a host thread
// that must not hit the driver's allocator (which can synchronise the
// device).  hfdib_classify_noalloc serves them: the caller passes the lambda
// field and the two output buffers, and the per-block counts that the ordered
// compaction needs live in a fixed array in this file's device memory.
//
// That array is a file-scope __device__ symbol of NOALLOC_SCRATCH_INTS ints
// (256 KB + 8 B: the block counts, the total and an invalid-lambda flag), so
// the limit is NOALLOC_MAX_CELLS = 2^24 cells.  Every GPU
// that loads the library holds it until the process exits.  The host cannot
// use the symbol's name as a device address; the first call on each device
// looks up its address with cudaGetSymbolAddress (with that device current)
// and caches it, so that first call should not be made inside a stream
// capture.  The stream must belong to the current device (checked).  All
// calls share the array and it keeps the last call's contents; each call
// clears the flag and rewrites every count it reads before reading it, and
// calls that overlap on the GPU (different streams, no ordering) race on it.
#include <mutex>

#include "common.cuh"

namespace {

using hf::BLOCK;

constexpr long long NOALLOC_MAX_CELLS = 1ll << 24;
constexpr int NOALLOC_MAX_BLOCKS = (int)(NOALLOC_MAX_CELLS / BLOCK);
// block counts (the total follows the last used one), then the flag slot
constexpr int NOALLOC_FLAG = NOALLOC_MAX_BLOCKS + 1;
constexpr int NOALLOC_SCRATCH_INTS = NOALLOC_MAX_BLOCKS + 2;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) int g_noalloc_scratch[NOALLOC_SCRATCH_INTS];

int* g_scratch_addr[NOALLOC_MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mu;

// device address of the scratch array on the current device (set-up once)
int scratch_address(int** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return HFDIB_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return HFDIB_ERR_CUDA;
        g_scratch_addr[dev] = (int*)p;
    }
    *out = g_scratch_addr[dev];
    return HFDIB_OK;
}

// cell groups of Sec. 2.3 written as bytes: 2 ic (lambda >= 0.5), 1 bc
// (0 < lambda < 0.5, or lambda = 0 with an ic vertex neighbour), 0 fc.  A
// lambda outside [0, 1] or NaN sets *bad (the call then fails, as
// hfdib_create does for such a field).
__global__ void k_na_classify(int nx, int ny, int nz, const double* __restrict__ lam, uint8_t* __restrict__ tags,
                              int* __restrict__ bad) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long N = (long long)nx * ny * nz;
    if (c >= N) return;
    int i = (int)(c % nx);
    long long r = c / nx;
    int j = (int)(r % ny);
    int k = (int)(r / ny);
    double l = lam[c];
    if (!(l >= 0.0 && l <= 1.0)) *bad = 1;
    uint8_t t;
    if (l >= 0.5) {
        t = 2;
    } else if (l > 0.0) {
        t = 1;
    } else {
        bool any = false;
        int z0 = nz > 1 ? -1 : 0, z1 = nz > 1 ? 1 : 0;
        for (int oz = z0; oz <= z1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    if (ox == 0 && oy == 0 && oz == 0) continue;
                    int ii = i + ox, jj = j + oy, kk = k + oz;
                    if (ii < 0 || jj < 0 || kk < 0 || ii >= nx || jj >= ny || kk >= nz) continue;
                    if (lam[((long long)kk * ny + jj) * nx + ii] >= 0.5) any = true;
                }
        t = any ? 1 : 0;
    }
    tags[c] = t;
}

__global__ void k_na_count(long long N, const uint8_t* __restrict__ tags, int* __restrict__ counts) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int v = (c < N && tags[c] == 1) ? 1 : 0;
    int s = __syncthreads_count(v);
    if (threadIdx.x == 0) counts[blockIdx.x] = s;
}

// exclusive scan of the block counts in one block; the total goes to counts[nb]
__global__ void k_na_scan(int nb, int* __restrict__ counts) {
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
        if (idx < nb) counts[idx] = carry + sm[threadIdx.x] - v;
        __syncthreads();
        carry += sm[BLOCK - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[nb] = carry;
}

__global__ void k_na_scatter(long long N, const uint8_t* __restrict__ tags, const int* __restrict__ offsets,
                             int32_t* __restrict__ cells, long long capacity) {
    __shared__ int sm[BLOCK];
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int v = (c < N && tags[c] == 1) ? 1 : 0;
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < BLOCK; o <<= 1) {
        int t = threadIdx.x >= o ? sm[threadIdx.x - o] : 0;
        __syncthreads();
        sm[threadIdx.x] += t;
        __syncthreads();
    }
    if (v) {
        long long pos = (long long)offsets[blockIdx.x] + sm[threadIdx.x] - 1;
        if (pos < capacity) cells[pos] = (int32_t)c;
    }
}

}  // namespace

extern "C" int hfdib_classify_noalloc(const hfdib_grid* grid, const double* lambda, uint8_t* tags,
                                      int32_t* bc_cells, int64_t bc_capacity, int64_t* n_bc, void* stream) {
    if (!grid || !lambda || !tags || !n_bc || bc_capacity < 0 || (bc_capacity > 0 && !bc_cells))
        return HFDIB_ERR_INVALID_ARG;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return HFDIB_ERR_INVALID_ARG;
    long long N = (long long)grid->nx * grid->ny * grid->nz;
    if (N > NOALLOC_MAX_CELLS) return HFDIB_ERR_TOO_LARGE;
    cudaStream_t s = (cudaStream_t)stream;
    // the scratch address below is the current device's: the stream must be on it
    int cur = -1, sdev = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return HFDIB_ERR_CUDA;
    if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) { cudaGetLastError(); return HFDIB_ERR_INVALID_ARG; }
    if (sdev != cur) return HFDIB_ERR_INVALID_ARG;
    int* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    int nb = (int)((N + BLOCK - 1) / BLOCK);
    if (cudaMemsetAsync(scratch + NOALLOC_FLAG, 0, sizeof(int), s) != cudaSuccess) return HFDIB_ERR_CUDA;
    k_na_classify<<<nb, BLOCK, 0, s>>>(grid->nx, grid->ny, grid->nz, lambda, tags, scratch + NOALLOC_FLAG);
    k_na_count<<<nb, BLOCK, 0, s>>>(N, tags, scratch);
    k_na_scan<<<1, BLOCK, 0, s>>>(nb, scratch);
    k_na_scatter<<<nb, BLOCK, 0, s>>>(N, tags, scratch, bc_cells, bc_capacity);
    // a launch failure is reported here, before the copy is issued (this also
    // consumes an error an earlier, unrelated launch may have left pending)
    if (cudaGetLastError() != cudaSuccess) return HFDIB_ERR_CUDA;
    int out[2] = {0, 0};
    if (cudaMemcpyAsync(&out[0], scratch + nb, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&out[1], scratch + NOALLOC_FLAG, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return HFDIB_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return HFDIB_ERR_CUDA;
    if (out[1]) { *n_bc = 0; return HFDIB_ERR_INVALID_ARG; }
    *n_bc = out[0];
    return out[0] > bc_capacity ? HFDIB_ERR_TOO_LARGE : HFDIB_OK;
}
