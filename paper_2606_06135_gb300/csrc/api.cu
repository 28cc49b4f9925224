// api.cu -- C ABI of the HFDIB SIMPLE solver: handle set-up, the sweep
// schedule (Fig. simplehfdibrans), steady solve, field access, checkpoints.
#include <math.h>
#include <stddef.h>
#include <cmath>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "batch.cuh"

using namespace hf;

namespace {

constexpr int HIST = 1024;

// ---------------------------------------------------------------- device memory
// Every device buffer of a handle or batch comes from the allocator that was
// current when the handle or batch was created: cudaMalloc / cudaFree, or
// the caller's hook set by hfdib_set_allocator (a framework's caching
// allocator, a fixed pool).  The handle keeps that allocator until it is
// destroyed, so each buffer goes back where it came from.
struct DevAlloc {
    hfdib_alloc_fn alloc = nullptr;
    hfdib_free_fn release = nullptr;
    void* ctx = nullptr;
};
struct DevBlock {
    void* p;
    size_t bytes;
};
std::mutex& alloc_mu() {
    static std::mutex m;
    return m;
}
DevAlloc& alloc_setting() {
    static DevAlloc a;
    return a;
}
DevAlloc current_alloc() {
    std::lock_guard<std::mutex> lock(alloc_mu());
    return alloc_setting();
}
// bytes > 0; HFDIB_ERR_OOM when the allocator has no memory, INVALID_ARG when
// a hook returns memory that is not 256-byte aligned
int dev_alloc(const DevAlloc& A, cudaStream_t s, size_t bytes, void** out) {
    *out = nullptr;
    if (A.alloc) {
        void* p = A.alloc(bytes, (void*)s, A.ctx);
        if (!p) return HFDIB_ERR_OOM;
        if ((uintptr_t)p & 255u) {
            A.release(p, bytes, (void*)s, A.ctx);
            return HFDIB_ERR_INVALID_ARG;
        }
        *out = p;
        return HFDIB_OK;
    }
    cudaError_t e = cudaMalloc(out, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return e == cudaErrorMemoryAllocation ? HFDIB_ERR_OOM : HFDIB_ERR_CUDA;
    }
    return HFDIB_OK;
}
void dev_free(const DevAlloc& A, cudaStream_t s, const DevBlock& b) {
    if (!b.p) return;
    if (A.release) A.release(b.p, b.bytes, (void*)s, A.ctx);
    else cudaFree(b.p);
}
constexpr uint64_t STATE_MAGIC = 0x48464449425354ull;  // "HFDIBST"

// Optional per-class kernel timing (host-driven sweeps only): an event pair
// around each launch, read back after the sweeps.
struct Prof {
    bool on = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> marks;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
};

// GMRES(m) workspace of the adjoint solve (device arrays)
struct AdjGmres {
    int m = 0;
    double *V = nullptr, *W = nullptr, *x = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr;
    double *gv = nullptr, *y = nullptr, *h1 = nullptr, *h2 = nullptr, *nrm2 = nullptr, *st = nullptr;
    double* part = nullptr;
    unsigned int* cnt = nullptr;
};

struct Ctx {
    Grid g;
    Params P;
    hfdib_options opt;
    hfdib_bc bc;
    int model = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Fields F;
    BcList bl;
    MgLevels mg;
    MgLevels32 mg32;
    int tail_from = 1;
    long long tail_cells = 0;   // persistent pressure solve: largest level of the one-block tail
    int coarse_sweeps = 20;
    int use_graph = 0;
    // F.G holds grad u of the current velocity (left by the last sweep's a9;
    // cleared by anything that writes the state)
    bool g_cur = false;
    int parity = 0;              // which of the two sweep graphs matches the p / pr buffers
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    long long graph_launches = 0, graph_body_launches = 0;
    Prof prof;
    int pblocks = 0;             // persistent pressure kernel grid (0: not used)
    double* ppart = nullptr;     // its block partials
    void* pdesc[2] = {nullptr, nullptr};  // its problem descriptor, per p / pr parity
    double* pbuf0 = nullptr;     // the buffer that is F.p at parity 0
    double* pbuf1 = nullptr;     // the buffer that is F.pr at parity 0
    size_t psmem = 0;            // its dynamic shared memory (the tail levels)
    unsigned int* pbar = nullptr;
    int* perr = nullptr;
    const int* err_src = nullptr;  // error word of the pressure kernel this handle's sweeps run
    long long spin_limit = BARRIER_POLLS;
    long long* trace = nullptr;    // set during hfdib_pressure_trace only
    int trace_cap = 0;
    double* lam = nullptr;
    double* hist = nullptr;      // device [HIST][HFDIB_NRES]
    double* res_dev = nullptr;   // device [HFDIB_NRES + 1]: residuals, then the barrier-timeout flag
    int* cnt_scratch = nullptr;  // compaction scratch
    std::vector<DevBlock> allocs;
    long long sweeps = 0;
    long long launches = 0;
    int last_piters = 0;
    double* pinned = nullptr;    // host pinned scratch (64 doubles)
    Adj adj;                     // adjoint work arrays (allocated by the first adjoint call)
    AdjGmres gm;                 // GMRES workspace of the adjoint
    cudaGraph_t adj_graph = nullptr;
    cudaGraphExec_t adj_gexec = nullptr;
    DevAlloc al;                 // the allocator of every block in `allocs`
    bool adj_ready = false;
    long long adj_tcap = 0;      // capacity of adj.tent
};

#define CK(x)                                         \
    do {                                              \
        cudaError_t e_ = (x);                         \
        if (e_ != cudaSuccess) return HFDIB_ERR_CUDA; \
    } while (0)

int dalloc(Ctx* h, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    int rc = dev_alloc(h->al, h->stream, bytes, p);
    if (rc) return rc;
    h->allocs.push_back({*p, bytes});
    if (cudaMemsetAsync(*p, 0, bytes, h->stream) != cudaSuccess) return HFDIB_ERR_CUDA;
    return HFDIB_OK;
}

template <typename T>
int dalloc_n(Ctx* h, T** p, long long n) {
    return dalloc(h, (void**)p, (size_t)n * sizeof(T));
}

void free_all(Ctx* h) {
    for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
    h->prof.pool.clear();
    for (int q = 0; q < 2; ++q) {
        if (h->gexec[q]) cudaGraphExecDestroy(h->gexec[q]);
        if (h->graph[q]) cudaGraphDestroy(h->graph[q]);
        h->gexec[q] = nullptr;
        h->graph[q] = nullptr;
    }
    if (h->adj_gexec) cudaGraphExecDestroy(h->adj_gexec);
    if (h->adj_graph) cudaGraphDestroy(h->adj_graph);
    h->adj_gexec = nullptr;
    h->adj_graph = nullptr;
    if (h->stream) cudaStreamSynchronize(h->stream);   // no pending work on blocks about to be released
    for (const DevBlock& b : h->allocs) dev_free(h->al, h->stream, b);
    h->allocs.clear();
    if (h->pinned) cudaFreeHost(h->pinned);
    h->pinned = nullptr;
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    h->stream = nullptr;
    h->own_stream = false;
}

__global__ void k_check_lambda(long long N, const double* lam, double* partials, unsigned int* counter,
                               double* out) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[1] = {0.0};
    if (c < N) {
        double l = lam[c];
        if (!(l >= 0.0 && l <= 1.0)) v[0] = 1.0;
    }
    grid_reduce<1, false>(v, partials, counter, out);
}

__global__ void k_to_f32(long long n, const double* __restrict__ a, float* __restrict__ b) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

__global__ void k_init_state(Grid g, Params P, Fields F, int model) {
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.N) return;
    bool ic = tag_of(F.flags[c]) == TAG_IC;
    for (int q = 0; q < 3; ++q) F.u[q][c] = ic ? g.u_s[q] : g.u_in[q];
    F.p[c] = 0.0;
    if (model != HFDIB_LAMINAR) {
        double k = ic ? 0.0 : P.k_in;
        F.k[c] = k;
        F.w[c] = P.w_in;
        // nu_t = C_mu k^2/eps = k/omega for the inlet pair
        double eps = eps_model(model) ? P.w_in : C_MU * P.k_in * P.w_in;
        F.nut[c] = ic ? 0.0 : C_MU * k * k / eps;
        F.w2[c] = eps_model(model) ? P.w_in / (C_MU * fmax(k, K_MIN)) : C_MU * k * P.w_in;
    }
}

int sync_read(Ctx* h, const double* dev, double* host, int n) {
    CK(cudaMemcpyAsync(h->pinned, dev, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    memcpy(host, h->pinned, n * sizeof(double));
    return HFDIB_OK;
}

// Residuals of the last sweep (HFDIB_NRES doubles).  HFDIB_ERR_TIMEOUT when a
// barrier wait of a persistent pressure kernel gave up since the last read
// (the flag is then cleared, so it is reported once).
int read_residuals(Ctx* h, double* res) {
    double tmp[HFDIB_NRES + 1];
    int rc = sync_read(h, h->res_dev, tmp, HFDIB_NRES + 1);
    if (rc) return rc;
    memcpy(res, tmp, HFDIB_NRES * sizeof(double));
    if (tmp[HFDIB_NRES] != 0.0) {
        CK(cudaMemsetAsync(h->F.scal + SC_TIMEOUT, 0, sizeof(double), h->stream));
        CK(cudaMemsetAsync(h->res_dev + HFDIB_NRES, 0, sizeof(double), h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return HFDIB_ERR_TIMEOUT;
    }
    return HFDIB_OK;
}

// FP32 mirrors of phi and nu_t (mixed path) after the FP64 fields changed
// outside a sweep (create, set_field, set_state)
void refresh_mirrors(Ctx* h) {
    if (!h->F.mixed) return;
    const Grid& g = h->g;
    for (int d = 0; d < g.dims; ++d)
        k_to_f32<<<nblocks(g.nface[d]), BLOCK, 0, h->stream>>>(g.nface[d], h->F.phi[d], h->F.phi32[d]);
    k_to_f32<<<nblocks(g.N), BLOCK, 0, h->stream>>>(g.N, h->F.nut, h->F.nut32);
}

// ---------------------------------------------------------------- profiling
cudaEvent_t prof_event(Prof& p) {
    if (p.used == p.pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        p.pool.push_back(e);
    }
    return p.pool[p.used++];
}

#define PROF(h, id, call)                                               \
    do {                                                                \
        if ((h)->prof.on) {                                             \
            cudaEvent_t a_ = prof_event((h)->prof), b_ = prof_event((h)->prof); \
            cudaEventRecord(a_, (h)->stream);                           \
            call;                                                       \
            cudaEventRecord(b_, (h)->stream);                           \
            (h)->prof.marks.push_back({(id), {a_, b_}});                \
        } else {                                                        \
            call;                                                       \
        }                                                               \
    } while (0)

// ---------------------------------------------------------------- sweep schedule
// grad u from the turbulence step (a9) of the previous sweep serves the
// next momentum assembly (a3) whenever that step runs
static bool grad_u_carried(const Ctx* h) { return h->model != HFDIB_LAMINAR && !h->opt.frozen_turbulence; }

// before a sweep: form grad u if no previous sweep left it for this state
static void ensure_grad_u(Ctx* h) {
    if (grad_u_carried(h) && !h->g_cur) {
        PROF(h, HFDIB_K_GRAD_U, launch_grad_u(h->g, h->F, h->stream));
        h->launches++;
    }
    h->g_cur = grad_u_carried(h);   // true again once the sweep's a9 has run
}

// Part A: a1-a6 of Fig. simplehfdibrans and (with_pressure) the pressure
// solve or its set-up.
void enqueue_part_a(Ctx* h, long long* L, bool with_pressure = true) {
    const Grid& g = h->g;
    const Params& P = h->P;
    Fields& F = h->F;
    cudaStream_t s = h->stream;
    bool turb = h->model != HFDIB_LAMINAR;
    // a1: omega_ib (eps_ib) of ic cells = max over bc u fc of the old field
    if (turb) { PROF(h, HFDIB_K_IMPOSED, launch_max_not_ic(g, F.flags, F.w, F.partials, F.counters + 0, F.scal + SC_WMAX, s)); (*L)++; }
    // a2: set alpha_u, compute u_ib, k_ib, omega_ib
    PROF(h, HFDIB_K_IMPOSED, launch_imposed(g, h->model, h->opt.freeze_switch, h->bl, F.flags, F.scal, F.u[0], F.u[1],
                                            F.u[2], F.k, F.uib[0], F.uib[1], F.uib[2], F.kib, F.wib, s));
    PROF(h, HFDIB_K_IMPOSED, launch_means(g, P, F, s));
    // a3: momentum assembly; a4: predictor; a5: correction (imposed rows).
    // With the turbulence step on, grad u of this velocity was formed by the
    // last sweep's a9 (the velocity does not change in between): the caller
    // makes sure of it (ensure_grad_u), so it is not formed again here.
    if (!grad_u_carried(h)) PROF(h, HFDIB_K_GRAD_U, launch_grad_u(g, F, s));
    if (g.conv == 3) { PROF(h, HFDIB_K_GRAD_U, launch_conv_limit(g, F, s)); (*L)++; }
    PROF(h, HFDIB_K_MOM_ASM, launch_mom_asm(g, P, F, s));
    *L += 4;
    for (int n = 0; n < h->opt.n_u; ++n) {
        if (F.mixed) {
            const int last = n == h->opt.n_u - 1;
            PROF(h, HFDIB_K_MOM_SMOOTH, launch_mom_smooth32(g, P, F, 0, n == 0, last, s));
            PROF(h, HFDIB_K_MOM_SMOOTH, launch_mom_smooth32(g, P, F, 1, 0, last, s));
        } else {
            PROF(h, HFDIB_K_MOM_SMOOTH, launch_mom_smooth(g, P, F, 0, s));
            PROF(h, HFDIB_K_MOM_SMOOTH, launch_mom_smooth(g, P, F, 1, s));
        }
        *L += 2;
    }
    // a6: rAU, HbyA, phiHbyA
    PROF(h, HFDIB_K_HBYA, launch_hbya(g, P, F, s));
    PROF(h, HFDIB_K_HBYA, launch_phiH(g, F, s));
    *L += 2;
    if (!with_pressure) return;
    // a7 set-up: operator, r0, initial preconditioning, loop state
    const MgLevels& M = h->mg;
    int jac = h->opt.precond == 0;
    if (h->pblocks > 0) {
        // the whole solve, operator hierarchy included, in one cooperative launch
        cudaMemsetAsync(h->pbar, 0, sizeof(unsigned int), s);
        cudaMemsetAsync(h->perr, 0, sizeof(int), s);
        PROF(h, HFDIB_K_PCG, launch_pressure_batched(F.mixed, g.dims, h->pdesc[h->parity], 1, M.nl, h->coarse_sweeps,
                                                     h->opt.p_reltol, h->opt.p_maxiter, h->pblocks, PT_THREADS,
                                                     h->psmem, h->pbar, h->perr, h->spin_limit, h->trace,
                                                     h->trace_cap, 0, s));
        (*L)++;
        return;
    }
    PROF(h, HFDIB_K_P_COEF, launch_p_coef(g, M, F.rAU, h->tail_from, s));
    *L += 1 + (h->tail_from - 1) + (h->tail_from < M.nl ? 1 : 0);
    PROF(h, HFDIB_K_PCG, launch_pcg_init(g, F, M, jac, s));
    (*L)++;
    if (!jac) {
        PROF(h, HFDIB_K_VCYCLE, launch_vcycle(g, M, h->tail_from, F, F.scal + SC_PCG_RZN, h->coarse_sweeps, s));
        *L += 5 * h->tail_from + 1;
    }
}

void enqueue_pcg_start(Ctx* h, cudaGraphConditionalHandle hc, int use_cond, long long* L) {
    launch_pcg_start(h->F, h->opt.precond == 0, h->opt.p_reltol, h->opt.p_maxiter, hc, use_cond, h->stream);
    (*L)++;
}

void enqueue_pcg_body(Ctx* h, cudaGraphConditionalHandle hc, int use_cond, long long* L) {
    int jac = h->opt.precond == 0;
    PROF(h, HFDIB_K_PCG, launch_pcg_body(h->g, h->F, h->mg, h->tail_from, jac, h->coarse_sweeps, h->opt.p_maxiter,
                                         hc, use_cond, h->stream));
    *L += 3 + (jac ? 0 : 5 * h->tail_from + 1);
}

// Part B: a8-a12 and the residual record.
void enqueue_part_b(Ctx* h, long long* L) {
    const Grid& g = h->g;
    const Params& P = h->P;
    Fields& F = h->F;
    cudaStream_t s = h->stream;
    bool turb = h->model != HFDIB_LAMINAR && !h->opt.frozen_turbulence;
    // a8: flux, pressure relaxation, velocity update (writes the relaxed p to pr)
    PROF(h, HFDIB_K_UPDATE, launch_update(g, P, F, h->mg.lv[0], s));
    (*L)++;
    if (turb) {
        // a9: production with the updated velocity, P_ib
        const Fields& G = F;
        PROF(h, HFDIB_K_GRAD_U, launch_grad_u(g, G, s));
        PROF(h, HFDIB_K_TURB_PREP, launch_turb_prep(g, P, G, s));
        PROF(h, HFDIB_K_TURB_PREP, launch_bc_prod(g, h->bl, G, s));
        // a10: eps / omega with imposed rows
        PROF(h, HFDIB_K_SCAL_ASM, launch_scal_asm(g, P, G, 0, s));
        *L += 4;
        for (int n = 0; n < h->opt.n_turb; ++n) {
            if (F.mixed) {
                PROF(h, HFDIB_K_SCAL_SMOOTH, launch_scal_smooth32(g, P, G, 0, 0, n == 0, s));
                PROF(h, HFDIB_K_SCAL_SMOOTH, launch_scal_smooth32(g, P, G, 0, 1, 0, s));
            } else {
                PROF(h, HFDIB_K_SCAL_SMOOTH, launch_scal_smooth(g, P, G, 0, 0, s));
                PROF(h, HFDIB_K_SCAL_SMOOTH, launch_scal_smooth(g, P, G, 0, 1, s));
            }
            *L += 2;
        }
        // a11: k with imposed rows, then the correction; a12 nu_t
        PROF(h, HFDIB_K_TURB_PREP, launch_k_prep(g, P, G, s));
        PROF(h, HFDIB_K_SCAL_ASM, launch_scal_asm(g, P, G, 1, s));
        *L += 2;
        for (int n = 0; n < h->opt.n_turb; ++n) {
            if (F.mixed) {
                PROF(h, HFDIB_K_SCAL_SMOOTH, launch_scal_smooth32(g, P, G, 1, 0, n == 0, s));
                PROF(h, HFDIB_K_SCAL_SMOOTH, launch_scal_smooth32(g, P, G, 1, 1, 0, s));
            } else {
                PROF(h, HFDIB_K_SCAL_SMOOTH, launch_scal_smooth(g, P, G, 1, 0, s));
                PROF(h, HFDIB_K_SCAL_SMOOTH, launch_scal_smooth(g, P, G, 1, 1, s));
            }
            *L += 2;
        }
        PROF(h, HFDIB_K_TURB_FINAL, launch_turb_final(g, P, G, s));
        (*L)++;
    }
    Params Pe = P;
    if (!turb) Pe.model = HFDIB_LAMINAR;  // frozen turbulence: no k / eps|omega residuals
    PROF(h, HFDIB_K_SWEEP_END, launch_sweep_end(Pe, F, g.dims, h->err_src, h->res_dev, h->hist, HIST, s));
    (*L)++;
}

// one iteration of the extended SIMPLE loop, host-driven
int run_sweep_host(Ctx* h) {
    long long L = 0;
    cudaGraphConditionalHandle none = 0;
    ensure_grad_u(h);
    enqueue_part_a(h, &L);
    if (h->pblocks == 0) PROF(h, HFDIB_K_PCG, enqueue_pcg_start(h, none, 0, &L));
    int check = h->opt.p_check;
    for (int it = 0; h->pblocks == 0 && it < h->opt.p_maxiter; ++it) {
        enqueue_pcg_body(h, none, 0, &L);
        if (check > 0 && (it + 1) % check == 0) {
            double done;
            int rc = sync_read(h, h->F.scal + SC_PCG_DONE, &done, 1);
            if (rc) return rc;
            if (done != 0.0) break;
        }
    }
    enqueue_part_b(h, &L);
    CK(cudaGetLastError());
    std::swap(h->F.p, h->F.pr);
    h->parity ^= 1;
    h->sweeps++;
    h->launches += L;
    return HFDIB_OK;
}

// The sweep as one CUDA graph: part A, a conditional while-node whose body is
// one PCG iteration (ended from the device when |r| <= p_reltol |r0| or at
// p_maxiter), part B.  Two graphs alternate the p / pr buffers.
int build_graph(Ctx* h, int which) {
    cudaStream_t s = h->stream;
    cudaGraph_t graph;
    CK(cudaGraphCreate(&graph, 0));
    if (h->pblocks > 0) {
        long long L = 0;
        CK(cudaStreamBeginCaptureToGraph(s, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        enqueue_part_a(h, &L);
        enqueue_part_b(h, &L);
        CK(cudaStreamEndCapture(s, &graph));
        cudaGraphExec_t exec;
        CK(cudaGraphInstantiate(&exec, graph, 0));
        h->graph[which] = graph;
        h->gexec[which] = exec;
        h->graph_launches = L;
        h->graph_body_launches = 0;
        return HFDIB_OK;
    }
    cudaGraphConditionalHandle hc;
    CK(cudaGraphConditionalHandleCreate(&hc, graph, 1, cudaGraphCondAssignDefault));
    long long L = 0;
    CK(cudaStreamBeginCaptureToGraph(s, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    enqueue_part_a(h, &L);
    enqueue_pcg_start(h, hc, 1, &L);
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &ndeps));
    std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
    CK(cudaStreamEndCapture(s, &graph));
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    CK(cudaGraphAddNode(&cnode, graph, dv.data(), nullptr, dv.size(), &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    long long Lb = 0;
    enqueue_pcg_body(h, hc, 1, &Lb);
    CK(cudaStreamEndCapture(s, &body));
    CK(cudaStreamBeginCaptureToGraph(s, graph, &cnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    enqueue_part_b(h, &L);
    CK(cudaStreamEndCapture(s, &graph));
    cudaGraphExec_t exec;
    CK(cudaGraphInstantiate(&exec, graph, 0));
    h->graph[which] = graph;
    h->gexec[which] = exec;
    h->graph_launches = L;
    h->graph_body_launches = Lb;
    return HFDIB_OK;
}

int run_sweep(Ctx* h) {
    if (!h->use_graph) return run_sweep_host(h);
    if (!h->gexec[h->parity]) {
        int rc = build_graph(h, h->parity);
        if (rc) {
            // capture not possible here: abandon it and run host-driven
            cudaStreamCaptureStatus st;
            if (cudaStreamIsCapturing(h->stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(h->stream, &g);
                if (g) cudaGraphDestroy(g);
            }
            cudaGetLastError();
            h->use_graph = 0;
            return run_sweep_host(h);
        }
    }
    ensure_grad_u(h);
    CK(cudaGraphLaunch(h->gexec[h->parity], h->stream));
    std::swap(h->F.p, h->F.pr);
    h->parity ^= 1;
    h->sweeps++;
    h->launches += h->graph_launches;
    return HFDIB_OK;
}

// ---------------------------------------------------------------- batches
// A batch holds B problems (each a full handle on the batch's stream) and
// advances them together, one launch per phase for all of them: every phase
// of the sweep (a1-a6, a8-a12) is a batched launch in which problem b owns a
// range of blocks (batch.cuh), and the pressure equations of all problems are
// solved by ONE persistent cooperative launch (pcgb.cu).  The problems'
// launch arguments live in two device tables (sweep phases, pressure solve);
// the p / pr buffers of a problem are swapped in both tables on the device at
// the end of each sweep it runs, so one captured graph serves every sweep.  A
// batch solve runs that sweep inside a device-controlled while loop: each
// problem's sweep end applies the stop test to its largest scaled residual,
// a problem that has stopped skips every later phase, and the loop ends when
// all have stopped or after max_iter sweeps.
struct BatchCtx {
    int B = 0;
    int mixed = 0;
    int dims = 2;
    std::vector<Ctx*> d;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevAlloc al;                          // the allocator of every block in `allocs`
    std::vector<DevBlock> allocs;
    std::vector<double*> parts;
    void* desc = nullptr;                 // device: pressure descriptors [B]
    SweepProblem* probs = nullptr;        // device: sweep-phase problem table [B]
    int* start = nullptr;                 // device: block offsets [BK_KINDS][B + 1]
    int tot[BK_KINDS] = {0, 0, 0, 0, 0};  // blocks of each launch kind
    unsigned int* bar = nullptr;
    int* err = nullptr;
    unsigned int* loop = nullptr;         // device: [0] sweeps of the running solve, [1] its max_iter
    int nblk = 0, threads = 1024, coarse_sweeps = 4, maxlev = 1;
    long long spin_limit = BARRIER_POLLS;
    long long tail_cells = PT_DEFAULT_TAIL_CELLS;
    size_t smem = 0;
    int use_graph = 1;
    cudaGraph_t graph = nullptr;          // one sweep
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t sgraph = nullptr;         // the solve loop
    cudaGraphExec_t sgexec = nullptr;
    long long sweeps = 0;
    double* pinned = nullptr;
    std::vector<SweepProblem> hprobs;
    bool described = false;               // the device tables hold the problems
    std::string key;
};

constexpr size_t BATCH_SMEM_BUDGET = PT_SMEM_BUDGET;

void batch_drop_graphs(BatchCtx* b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->sgexec) cudaGraphExecDestroy(b->sgexec);
    if (b->sgraph) cudaGraphDestroy(b->sgraph);
    b->gexec = nullptr;
    b->graph = nullptr;
    b->sgexec = nullptr;
    b->sgraph = nullptr;
}

BatchTab batch_tab(const BatchCtx* b, int skip) { return BatchTab{b->probs, b->start, b->B, skip}; }

// The host handles follow the device tables: their p / pr pointers, parity
// and sweep count (after every batch call, before any re-description).
int batch_sync_host(BatchCtx* b) {
    if (!b->probs || !b->described) return HFDIB_OK;
    CK(cudaMemcpyAsync(b->hprobs.data(), b->probs, sizeof(SweepProblem) * b->B, cudaMemcpyDeviceToHost, b->stream));
    for (int i = 0; i < b->B; ++i)
        CK(cudaMemcpyAsync(b->pinned + i, b->d[i]->F.scal + SC_NSWEEP, sizeof(double), cudaMemcpyDeviceToHost,
                           b->stream));
    CK(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->B; ++i) {
        Ctx* h = b->d[i];
        const double* p = b->hprobs[i].F.p;
        const double* pr = b->hprobs[i].F.pr;
        // the two pressure buffers of this problem, in either order
        if (!((p == h->pbuf0 && pr == h->pbuf1) || (p == h->pbuf1 && pr == h->pbuf0))) return HFDIB_ERR_CUDA;
        h->F.p = b->hprobs[i].F.p;
        h->F.pr = b->hprobs[i].F.pr;
        h->parity = h->F.p == h->pbuf0 ? 0 : 1;
        h->sweeps = (long long)b->pinned[i];
    }
    return HFDIB_OK;
}

// (re)build the problem table, the block offsets and the pressure
// descriptors for the current launch parameters and the current p / pr
int batch_describe(BatchCtx* b) {
    int rc = batch_sync_host(b);
    if (rc) return rc;
    batch_drop_graphs(b);
    const int B = b->B;
    size_t dsz = pcgb_desc_size(b->mixed);
    size_t foff = pcgb_fields_offset(b->mixed);
    std::vector<unsigned char> hdesc(dsz * B, 0);
    std::vector<int> st((size_t)BK_KINDS * (B + 1), 0);
    size_t smem = 0;
    for (int i = 0; i < B; ++i) {
        Ctx* h = b->d[i];
        void* dst = hdesc.data() + dsz * i;
        size_t by = b->mixed ? pcgb_describe32(dst, h->g, h->F, h->mg, h->mg32, b->parts[i], b->tail_cells,
                                               BATCH_SMEM_BUDGET)
                             : pcgb_describe64(dst, h->g, h->F, h->mg, b->parts[i], b->tail_cells, BATCH_SMEM_BUDGET);
        if (by > smem) smem = by;
        SweepProblem& sp = b->hprobs[i];
        memset((void*)&sp, 0, sizeof(sp));
        sp.g = h->g;
        sp.P = h->P;
        sp.F = h->F;
        sp.bl = h->bl;
        sp.L0 = h->mg.lv[0];
        sp.freeze = h->opt.freeze_switch;
        bool turb_b = h->model != HFDIB_LAMINAR && !h->opt.frozen_turbulence;
        sp.model_end = turb_b ? h->model : HFDIB_LAMINAR;
        sp.err = b->err;
        sp.res_out = h->res_dev;
        sp.hist = h->hist;
        sp.nhist = HIST;
        sp.done = h->F.scal + SC_DONE;
        char* pe = (char*)&b->probs[i];
        char* de = (char*)b->desc + dsz * i + foff;
        sp.swap_p[0] = (double**)(pe + offsetof(SweepProblem, F) + offsetof(Fields, p));
        sp.swap_pr[0] = (double**)(pe + offsetof(SweepProblem, F) + offsetof(Fields, pr));
        sp.swap_p[1] = (double**)(de + offsetof(Fields, p));
        sp.swap_pr[1] = (double**)(de + offsetof(Fields, pr));
        const long long n[BK_KINDS] = {nblocks(h->g.N), rblocks(h->g.N), nblocks(npairs(h->g)),
                                       h->bl.nbc > 0 ? nblocks(h->bl.nbc) : 0, 1};
        for (int k = 0; k < BK_KINDS; ++k) st[(size_t)k * (B + 1) + i + 1] = st[(size_t)k * (B + 1) + i] + (int)n[k];
    }
    for (int k = 0; k < BK_KINDS; ++k) b->tot[k] = st[(size_t)k * (B + 1) + B];
    CK(cudaMemcpyAsync(b->desc, hdesc.data(), dsz * B, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->probs, b->hprobs.data(), sizeof(SweepProblem) * B, cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->start, st.data(), st.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    b->described = true;
    int bps = 0;
    if (pcgb_fits(b->mixed, b->dims, b->threads, smem, &bps) != 0 || bps < 1) return HFDIB_ERR_INVALID_ARG;
    b->smem = smem;
    return HFDIB_OK;
}

// one sweep of every problem (skip: problems whose stop flag is set sit out)
void batch_enqueue(BatchCtx* b, int skip) {
    cudaStream_t s = b->stream;
    const BatchTab T = batch_tab(b, skip);
    const int* tot = b->tot;
    const Ctx* h0 = b->d[0];
    const bool turb = h0->model != HFDIB_LAMINAR;
    const bool turb_b = turb && !h0->opt.frozen_turbulence;
    const bool mixed = b->mixed != 0;
    // a1, a2, the residual means
    if (turb) launchb_max_not_ic(T, tot, s);
    launchb_imposed(T, tot, s);
    launchb_means(T, tot, s);
    // a3 assembly (grad u carried from the last sweep's a9 when that step
    // runs: batch_ensure_grad_u), a4/a5 predictor with the imposed rows
    if (!turb_b) launchb_grad_u(T, tot, s);
    if (h0->g.conv == 3) launchb_conv_limit(T, tot, s);
    launchb_mom_asm(T, tot, s);
    for (int n = 0; n < h0->opt.n_u; ++n) {
        if (mixed) {
            const int last = n == h0->opt.n_u - 1;
            launchb_mom_smooth32(T, tot, 0, n == 0, last, s);
            launchb_mom_smooth32(T, tot, 1, 0, last, s);
        } else {
            launchb_mom_smooth(T, tot, 0, s);
            launchb_mom_smooth(T, tot, 1, s);
        }
    }
    // a6
    launchb_hbya(T, tot, s);
    launchb_phiH(T, tot, s);
    // a7: every pressure equation in one persistent launch
    launch_pressure_reset(b->bar, b->err, s);
    launch_pressure_batched(b->mixed, b->dims, b->desc, b->B, b->maxlev, b->coarse_sweeps, h0->opt.p_reltol,
                            h0->opt.p_maxiter, b->nblk, b->threads, b->smem, b->bar, b->err, b->spin_limit, nullptr,
                            0, skip, s);
    // a8
    launchb_update(T, tot, s);
    if (turb_b) {
        // a9 production, P_ib; a10 eps / omega; a11 k; a12 nu_t
        launchb_grad_u(T, tot, s);
        launchb_turb_prep(T, tot, s);
        launchb_bc_prod(T, tot, s);
        launchb_scal_asm(T, tot, 0, s);
        for (int n = 0; n < h0->opt.n_turb; ++n) {
            if (mixed) {
                launchb_scal_smooth32(T, tot, 0, 0, n == 0, s);
                launchb_scal_smooth32(T, tot, 0, 1, 0, s);
            } else {
                launchb_scal_smooth(T, tot, 0, 0, s);
                launchb_scal_smooth(T, tot, 0, 1, s);
            }
        }
        launchb_k_prep(T, tot, s);
        launchb_scal_asm(T, tot, 1, s);
        for (int n = 0; n < h0->opt.n_turb; ++n) {
            if (mixed) {
                launchb_scal_smooth32(T, tot, 1, 0, n == 0, s);
                launchb_scal_smooth32(T, tot, 1, 1, 0, s);
            } else {
                launchb_scal_smooth(T, tot, 1, 0, s);
                launchb_scal_smooth(T, tot, 1, 1, s);
            }
        }
        launchb_turb_final(T, tot, s);
    }
    // residual record, stop test (solves), p / pr swap
    launchb_sweep_end(T, tot, s);
}

// before sweeps of a batch: form grad u for every problem unless each has it
// from its last sweep (problems that sat out keep theirs: their velocity did
// not change)
void batch_ensure_grad_u(BatchCtx* b) {
    const Ctx* h0 = b->d[0];
    const bool carried = grad_u_carried(h0);
    bool cur = true;
    for (const Ctx* h : b->d) cur = cur && h->g_cur;
    if (carried && !cur) launchb_grad_u(batch_tab(b, 0), b->tot, b->stream);
    for (Ctx* h : b->d) h->g_cur = carried;
}

int batch_sweep_once(BatchCtx* b) {
    if (b->use_graph && !b->gexec) {
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            batch_enqueue(b, 0);
            ok = cudaStreamEndCapture(b->stream, &g) == cudaSuccess;
        }
        cudaGraphExec_t ex = nullptr;
        if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
        if (!ok) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            b->use_graph = 0;
        } else {
            b->graph = g;
            b->gexec = ex;
        }
    }
    batch_ensure_grad_u(b);
    if (b->use_graph) CK(cudaGraphLaunch(b->gexec, b->stream));
    else batch_enqueue(b, 0);
    CK(cudaGetLastError());
    b->sweeps++;
    return HFDIB_OK;
}

// the solve loop as one graph: a device-controlled while node around one
// sweep (stop flags honoured) and the loop's end-of-sweep test
int batch_build_solve_graph(BatchCtx* b) {
    cudaStream_t s = b->stream;
    cudaGraph_t graph;
    CK(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle hc;
    CK(cudaGraphConditionalHandleCreate(&hc, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    CK(cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    batch_enqueue(b, 1);
    launchb_next(batch_tab(b, 1), b->loop, b->loop + 1, hc, s);
    CK(cudaStreamEndCapture(s, &body));
    cudaGraphExec_t exec;
    CK(cudaGraphInstantiate(&exec, graph, 0));
    b->sgraph = graph;
    b->sgexec = exec;
    return HFDIB_OK;
}

// residuals of every problem; HFDIB_ERR_TIMEOUT (after clearing the flags)
// when a barrier wait of the batched pressure kernel gave up since the last read
int batch_read_residuals(BatchCtx* b, double* out) {
    const size_t R = HFDIB_NRES + 1;
    for (int i = 0; i < b->B; ++i)
        CK(cudaMemcpyAsync(b->pinned + (size_t)i * R, b->d[i]->res_dev, R * sizeof(double),
                           cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    bool timeout = false;
    for (int i = 0; i < b->B; ++i) {
        memcpy(out + (size_t)i * HFDIB_NRES, b->pinned + (size_t)i * R, sizeof(double) * HFDIB_NRES);
        if (b->pinned[(size_t)i * R + HFDIB_NRES] != 0.0) timeout = true;
    }
    if (timeout) {
        for (Ctx* h : b->d) {
            CK(cudaMemsetAsync(h->F.scal + SC_TIMEOUT, 0, sizeof(double), b->stream));
            CK(cudaMemsetAsync(h->res_dev + HFDIB_NRES, 0, sizeof(double), b->stream));
        }
        CK(cudaStreamSynchronize(b->stream));
        return HFDIB_ERR_TIMEOUT;
    }
    return HFDIB_OK;
}

void batch_free(BatchCtx* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    for (Ctx* h : b->d)
        if (h) hfdib_destroy((hfdib_handle)h);
    for (const DevBlock& blk : b->allocs) dev_free(b->al, b->stream, blk);
    if (b->pinned) cudaFreeHost(b->pinned);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

// autotuner results, keyed by batch shape
std::map<std::string, hfdib_tune>& tune_cache() {
    static std::map<std::string, hfdib_tune> m;
    return m;
}
std::mutex& tune_mu() {
    static std::mutex m;
    return m;
}

double* field_ptr(Ctx* h, int field, long long* n) {
    *n = h->g.N;
    switch (field) {
        case HFDIB_FIELD_UX: return h->F.u[0];
        case HFDIB_FIELD_UY: return h->F.u[1];
        case HFDIB_FIELD_UZ: return h->g.dims == 3 ? h->F.u[2] : nullptr;
        case HFDIB_FIELD_P: return h->F.p;
        case HFDIB_FIELD_K: return h->model ? h->F.k : nullptr;
        case HFDIB_FIELD_EPS: return !h->model ? nullptr : (eps_model(h->model) ? h->F.w : h->F.w2);
        case HFDIB_FIELD_OMEGA: return !h->model ? nullptr : (eps_model(h->model) ? h->F.w2 : h->F.w);
        case HFDIB_FIELD_NUT: return h->F.nut;
        case HFDIB_FIELD_PHIX: *n = h->g.nface[0]; return h->F.phi[0];
        case HFDIB_FIELD_PHIY: *n = h->g.nface[1]; return h->F.phi[1];
        case HFDIB_FIELD_PHIZ: *n = h->g.nface[2]; return h->g.dims == 3 ? h->F.phi[2] : nullptr;
        default: return nullptr;
    }
}

// ---------------------------------------------------------------- adjoint
#define RC(x)                                  \
    do {                                       \
        int r_ = (x);                          \
        if (r_ != HFDIB_OK) return r_;         \
    } while (0)

int adj_alloc(Ctx* h) {
    if (h->adj_ready) return HFDIB_OK;
    const Grid& g = h->g;
    const long long N = g.N;
    Adj& A = h->adj;
    memset(&A, 0, sizeof(A));
    A.nu = h->opt.n_u;
    int rc = HFDIB_OK;
#define AL(p, n) \
    if (!rc) rc = dalloc_n(h, &(p), (long long)(n))
    AL(A.snap, (2LL * A.nu + 1) * 3 * N);
    AL(A.As, 6 * N); AL(A.AP, 3 * N); AL(A.aavg, N); AL(A.jw, N);
    for (int q = 0; q < 3; ++q) {
        AL(A.Hb[q], N); AL(A.b0b[q], N); AL(A.bmb[q], N);
        AL(A.aPb[q], N); AL(A.usb[0][q], N); AL(A.usb[1][q], N); AL(A.fixb[q], N); AL(A.fixs[q], N);
    }
    // flat adjoint state: u components, p, face fluxes of the active directions
    long long nv = (long long)(g.dims + 1) * N;
    for (int d = 0; d < g.dims; ++d) nv += g.nface[d];
    A.nvec = nv;
    AL(A.vpsi, nv); AL(A.vxb, nv); AL(A.vb, nv);
    AL(A.pnb, N); AL(A.ps, N); AL(A.rAUb, N);
    AL(A.asb, 6 * N); AL(A.Gb, 9 * N); AL(A.tptr, N + 1); AL(A.dlam, N);
#undef AL
    if (rc) return rc;
    {
        long long off = 0;
        for (int q = 0; q < g.dims; ++q, off += N) {
            A.psu[q] = A.vpsi + off; A.xbu[q] = A.vxb + off; A.vbu[q] = A.vb + off;
        }
        A.psp = A.vpsi + off;
        A.xbp = A.vxb + off;
        A.vbp = A.vb + off;
        off += N;
        for (int d = 0; d < g.dims; ++d) {
            A.psf[d] = A.vpsi + off;
            A.xbf[d] = A.vxb + off;
            A.vbf[d] = A.vb + off;
            off += g.nface[d];
        }
        for (int q = g.dims; q < 3; ++q) {  // not read in 2D; point at valid memory
            A.psu[q] = A.psu[0]; A.xbu[q] = A.xbu[0]; A.psf[q] = A.psf[0]; A.xbf[q] = A.xbf[0];
            A.vbu[q] = A.vbu[0]; A.vbf[q] = A.vbf[0];
        }
    }
    // objective weights from the closed-face flags (fixed for the handle's lambda)
    cudaStream_t s = h->stream;
    std::vector<uint16_t> flags(N);
    CK(cudaMemcpyAsync(flags.data(), h->F.flags, N * sizeof(uint16_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // objective: mean p over the cells of each open inlet side minus the mean over each outlet side
    std::vector<double> jw(N, 0.0);
    for (int sd = 0; sd < 2 * g.dims; ++sd) {
        int kind = g.kind[sd];
        if (kind != HFDIB_BC_INLET && kind != HFDIB_BC_OUTLET) continue;
        int d = sd >> 1, hi = sd & 1;
        std::vector<long long> cells;
        for (long long c = 0; c < N; ++c) {
            long long i = c % g.nx, j = (c / g.nx) % g.ny, k = c / ((long long)g.nx * g.ny);
            long long pos = d == 0 ? i : (d == 1 ? j : k);
            if (pos != (hi ? g.n[d] - 1 : 0)) continue;
            if (kind == HFDIB_BC_INLET && closed_side(flags[c], sd)) continue;
            cells.push_back(c);
        }
        if (cells.empty()) continue;
        double w = (kind == HFDIB_BC_INLET ? 1.0 : -1.0) / (double)cells.size();
        for (long long c : cells) jw[c] += w;
    }
    CK(cudaMemcpyAsync(A.jw, jw.data(), N * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    h->adj_ready = true;
    return HFDIB_OK;
}

// CG to a relative tolerance on the redirected Fields (the loop kernels are
// no-ops once the device flag says done; the host looks every 8 iterations)
int adj_pcg_run(Ctx* h, const Fields& Fa, double reltol, int maxit) {
    int jac = h->opt.precond == 0;
    launch_pcg_start(Fa, jac, reltol, maxit, 0, 0, h->stream);
    for (int it = 0; it < maxit; it += 8) {
        for (int r = 0; r < 8; ++r)
            launch_pcg_body(h->g, Fa, h->mg, h->tail_from, jac, h->coarse_sweeps, maxit, 0, 0, h->stream);
        double done = 0.0;
        RC(sync_read(h, Fa.scal + SC_PCG_DONE, &done, 1));
        if (done != 0.0) return HFDIB_OK;
    }
    return HFDIB_OK;
}

// The frozen-turbulence sweep at the converged state, kept for the reverse
// pass: imposed rows and u_ib, the predictor iterates, HbyA, rAU, phiHbyA,
// the exact pressure solution and the momentum-row coefficients.  The state
// (u, p, phi, turbulence) is not modified.  Host work: index bookkeeping only
// (objective cells, the per-cell entry list of the transposed interpolation).
int adj_setup(Ctx* h) {
    const Grid& g = h->g;
    Fields F = h->F;
    F.mixed = 0;  // the differentiated sweep is FP64
    const Params& P = h->P;
    cudaStream_t s = h->stream;
    Adj& A = h->adj;
    const long long N = g.N;
    int jac = h->opt.precond == 0;
    launch_imposed(g, h->model, h->opt.freeze_switch, h->bl, F.flags, F.scal, F.u[0], F.u[1], F.u[2], F.k,
                   F.uib[0], F.uib[1], F.uib[2], F.kib, F.wib, s);
    CK(cudaMemsetAsync(F.scal + SC_NLAM, 0, 2 * sizeof(double), s));
    launch_grad_u(g, F, s);
    launch_mom_asm(g, P, F, s);
    for (int n = 0; n < A.nu; ++n)
        for (int col = 0; col < 2; ++col) {
            for (int q = 0; q < g.dims; ++q)
                CK(cudaMemcpyAsync(A.snap + ((long long)(2 * n + col) * 3 + q) * N, F.us[q], N * sizeof(double),
                                   cudaMemcpyDeviceToDevice, s));
            launch_mom_smooth(g, P, F, col, s);
        }
    for (int q = 0; q < g.dims; ++q)
        CK(cudaMemcpyAsync(A.snap + ((long long)(2 * A.nu) * 3 + q) * N, F.us[q], N * sizeof(double),
                           cudaMemcpyDeviceToDevice, s));
    launch_hbya(g, P, F, s);
    launch_phiH(g, F, s);
    launch_p_coef(g, h->mg, F.rAU, h->tail_from, s);
    launch_pcg_init(g, F, h->mg, jac, s);
    if (!jac) launch_vcycle(g, h->mg, h->tail_from, F, F.scal + SC_PCG_RZN, h->coarse_sweeps, s);
    RC(adj_pcg_run(h, F, 1e-14, 4000));
    launch_adj_coef(g, P, F, A, s);
    CK(cudaGetLastError());
    // index bookkeeping on the host
    int nbc = h->bl.nbc;
    std::vector<uint16_t> flags(N);
    std::vector<int> cell(nbc > 0 ? nbc : 1), lamb(nbc > 0 ? nbc : 1), b1(3 * (nbc > 0 ? nbc : 1)),
        b2(3 * (nbc > 0 ? nbc : 1));
    CK(cudaMemcpyAsync(flags.data(), F.flags, N * sizeof(uint16_t), cudaMemcpyDeviceToHost, s));
    if (nbc > 0) {
        CK(cudaMemcpyAsync(cell.data(), h->bl.cell, nbc * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(lamb.data(), h->bl.lamb, nbc * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(b1.data(), h->bl.b1, 3 * nbc * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(b2.data(), h->bl.b2, 3 * nbc * sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    // transposed interpolation: for every cell, the (bc entry, stencil, corner) that read it
    std::vector<int> cnt(N + 1, 0);
    std::vector<std::pair<long long, int>> ent;
    for (int q = 0; q < nbc; ++q) {
        if (!lamb[q] || !(flags[cell[q]] & F_AU)) continue;
        for (int st = 0; st < 2; ++st) {
            const int* b = (st ? b2.data() : b1.data()) + 3 * q;
            for (int corner = 0; corner < 8; ++corner) {
                int id[3];
                bool skip = false;
                for (int d = 0; d < 3; ++d) {
                    int cc = (corner >> d) & 1;
                    if (g.n[d] == 1 && cc) skip = true;
                    id[d] = b[d] + (g.n[d] == 1 ? 0 : cc);
                }
                if (skip) continue;
                long long t = ((long long)id[2] * g.ny + id[1]) * g.nx + id[0];
                ent.push_back({t, q * 16 + st * 8 + corner});
            }
        }
    }
    for (auto& e : ent) cnt[e.first + 1]++;
    for (long long c = 0; c < N; ++c) cnt[c + 1] += cnt[c];
    std::vector<int> tent(ent.size() > 0 ? ent.size() : 1);
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (auto& e : ent) tent[fill[e.first]++] = e.second;
    if ((long long)tent.size() > h->adj_tcap) {
        RC(dalloc_n(h, &A.tent, (long long)tent.size()));
        h->adj_tcap = (long long)tent.size();
    }
    CK(cudaMemcpyAsync(A.tptr, cnt.data(), (N + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(A.tent, tent.data(), tent.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return HFDIB_OK;
}

// One reverse pass: x-bar = G_x^T psi (A.vxb from A.vpsi) and u_ib-bar (A.fixb),
// the part of G_lambda^T psi.  Part A ends with the set-up of the adjoint
// pressure solve (zero start, relative tolerance), part B follows it.
void adj_enqueue_a(Ctx* h, bool warm) {
    const Grid& g = h->g;
    Fields F = h->F;
    F.mixed = 0;
    cudaStream_t s = h->stream;
    Adj& A = h->adj;
    const Level& L0 = h->mg.lv[0];
    int jac = h->opt.precond == 0;
    launch_adj_update(g, h->P, F, L0, A, s);
    // the adjoint pressure solve starts from the previous pass's solution
    // (warm) and stops at tol |rhs| (see k_adj_pcg_init), or from zero
    if (!warm) cudaMemsetAsync(A.ps, 0, g.N * sizeof(double), s);
    Fields Fa = F;
    Fa.pn = A.ps;
    launch_adj_pcg_init(g, Fa, L0, A.pnb, jac, s);
    if (!jac) launch_vcycle(g, h->mg, h->tail_from, Fa, Fa.scal + SC_PCG_RZN, h->coarse_sweeps, s);
}

void adj_enqueue_b(Ctx* h) {
    const Grid& g = h->g;
    Fields F = h->F;
    F.mixed = 0;
    const Params& P = h->P;
    cudaStream_t s = h->stream;
    Adj& A = h->adj;
    launch_adj_pressure(g, F, h->mg.lv[0], A, s);
    launch_adj_hbya(g, P, F, A, s);
    int buf = 0;
    for (int hs = 2 * A.nu; hs >= 1; --hs) {
        const double* Sin = A.snap + (long long)(hs - 1) * 3 * g.N;
        const double* Sout = A.snap + (long long)hs * 3 * g.N;
        launch_adj_gs(g, P, F, A, (hs - 1) & 1, Sin, Sout, buf, s);
        buf = 1 - buf;
    }
    launch_adj_b0(g, P, F, A, buf, s);
    launch_adj_transpose(g, F, A, s);
    launch_adj_gradu(g, F, h->bl, A, s);
    launch_adj_phi(g, F, A, s);
}

Fields adj_pfields(Ctx* h) {
    Fields Fa = h->F;
    Fa.mixed = 0;
    Fa.pn = h->adj.ps;
    return Fa;
}

// the pass as one CUDA graph, the adjoint CG in a device-controlled while node
int adj_build_graph(Ctx* h, double ptol, bool warm) {
    cudaStream_t s = h->stream;
    int jac = h->opt.precond == 0;
    Fields Fa = adj_pfields(h);
    cudaGraph_t graph;
    CK(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle hc;
    CK(cudaGraphConditionalHandleCreate(&hc, graph, 1, cudaGraphCondAssignDefault));
    CK(cudaStreamBeginCaptureToGraph(s, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    adj_enqueue_a(h, warm);
    launch_pcg_start(Fa, jac, ptol, 4000, hc, 1, s);
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &ndeps));
    std::vector<cudaGraphNode_t> dv(deps, deps + ndeps);
    CK(cudaStreamEndCapture(s, &graph));
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    CK(cudaGraphAddNode(&cnode, graph, dv.data(), nullptr, dv.size(), &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch_pcg_body(h->g, Fa, h->mg, h->tail_from, jac, h->coarse_sweeps, 4000, hc, 1, s);
    CK(cudaStreamEndCapture(s, &body));
    CK(cudaStreamBeginCaptureToGraph(s, graph, &cnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    adj_enqueue_b(h);
    CK(cudaStreamEndCapture(s, &graph));
    cudaGraphExec_t exec;
    CK(cudaGraphInstantiate(&exec, graph, 0));
    h->adj_graph = graph;
    h->adj_gexec = exec;
    return HFDIB_OK;
}

void adj_drop_graph(Ctx* h) {
    if (h->adj_gexec) cudaGraphExecDestroy(h->adj_gexec);
    if (h->adj_graph) cudaGraphDestroy(h->adj_graph);
    h->adj_gexec = nullptr;
    h->adj_graph = nullptr;
}

int adj_pass(Ctx* h, double ptol, bool warm) {
    if (h->adj_gexec) {
        CK(cudaGraphLaunch(h->adj_gexec, h->stream));
        return HFDIB_OK;
    }
    adj_enqueue_a(h, warm);
    RC(adj_pcg_run(h, adj_pfields(h), ptol, 4000));
    adj_enqueue_b(h);
    CK(cudaGetLastError());
    return HFDIB_OK;
}

// GMRES(m) on (I - G_x^T) psi = J_x^T; psi ends in A.vpsi and the last pass
// (with that psi) leaves u_ib-bar in A.fixb.  mv counts reverse passes.
int adj_gmres_alloc(Ctx* h, int m) {
    AdjGmres& G = h->gm;
    if (G.m >= m && G.V) return HFDIB_OK;
    const long long n = h->adj.nvec;
    int rc = HFDIB_OK;
    G.m = m;
    int pg = mdot_grid(n);
#define AL(p, k) \
    if (!rc) rc = dalloc_n(h, &(p), (long long)(k))
    AL(G.V, (long long)(m + 1) * n); AL(G.W, n); AL(G.x, n);
    AL(G.H, (long long)(m + 1) * m); AL(G.cs, m + 1); AL(G.sn, m + 1); AL(G.gv, m + 1); AL(G.y, m + 1);
    AL(G.h1, m + 1); AL(G.h2, m + 1); AL(G.nrm2, 2); AL(G.st, 4);
    AL(G.part, (long long)(m + 1) * pg); AL(G.cnt, 1);
#undef AL
    return rc;
}

int adj_gmres(Ctx* h, int m, double tol, int max_mv, int* mv_out, double* rel_out) {
    Adj& A = h->adj;
    AdjGmres& G = h->gm;
    cudaStream_t s = h->stream;
    const long long n = A.nvec;
    const double ptol = 1e-12;
    RC(adj_gmres_alloc(h, m));
    launch_mdot(n, A.vb, A.vb, n, 1, G.part, G.cnt, G.nrm2 + 1, s);
    double bn2 = 0.0;
    RC(sync_read(h, G.nrm2 + 1, &bn2, 1));
    double bnorm = sqrt(bn2);
    CK(cudaMemsetAsync(G.x, 0, n * sizeof(double), s));
    int mv = 0;
    double relres = 1.0;
    bool first = true, done = bnorm == 0.0;
    while (!done && mv < max_mv) {
        // r0 = b - (x - M x)
        if (first) {
            CK(cudaMemcpyAsync(G.W, A.vb, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        } else {
            CK(cudaMemcpyAsync(A.vpsi, G.x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            RC(adj_pass(h, ptol, true));
            ++mv;
            launch_vsub_add(n, A.vb, G.x, A.vxb, G.W, s);
        }
        first = false;
        launch_mdot(n, G.W, G.W, n, 1, G.part, G.cnt, G.nrm2, s);
        launch_vnormalize(n, G.W, G.V, G.nrm2, s);
        launch_gmres_start(m, G.nrm2, G.gv, G.st, s);
        double beta = 0.0;
        RC(sync_read(h, G.st, &beta, 1));
        relres = beta / bnorm;
        if (!(beta > tol * bnorm)) break;
        int k = 0;
        for (int j = 0; j < m && mv < max_mv; ++j) {
            double* Vj = G.V + (long long)j * n;
            CK(cudaMemcpyAsync(A.vpsi, Vj, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            RC(adj_pass(h, ptol, true));
            ++mv;
            launch_vsub(n, Vj, A.vxb, G.W, s);  // w = (I - M) V_j
            launch_mdot(n, G.W, G.V, n, j + 1, G.part, G.cnt, G.h1, s);
            launch_maxpy(n, G.W, G.V, n, j + 1, G.h1, -1.0, s);
            launch_mdot(n, G.W, G.V, n, j + 1, G.part, G.cnt, G.h2, s);
            launch_maxpy(n, G.W, G.V, n, j + 1, G.h2, -1.0, s);
            launch_mdot(n, G.W, G.W, n, 1, G.part, G.cnt, G.nrm2, s);
            launch_gmres_column(j, m, G.H, G.h1, G.h2, G.nrm2, G.cs, G.sn, G.gv, G.st, s);
            launch_vnormalize(n, G.W, G.V + (long long)(j + 1) * n, G.nrm2, s);
            k = j + 1;
            double est = 0.0;
            RC(sync_read(h, G.st + 1, &est, 1));
            if (!std::isfinite(est)) return HFDIB_ERR_DIVERGED;
            relres = est / bnorm;
            if (est <= tol * bnorm) { done = true; break; }
        }
        if (k > 0) {
            launch_gmres_y(k, m, G.H, G.gv, G.y, s);
            launch_maxpy(n, G.x, G.V, n, k, G.y, 1.0, s);
        }
    }
    // the pass with the final psi: u_ib-bar for the gradient, and the true residual
    CK(cudaMemcpyAsync(A.vpsi, G.x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    RC(adj_pass(h, ptol, true));
    ++mv;
    launch_vsub_add(n, A.vb, G.x, A.vxb, G.W, s);
    launch_mdot(n, G.W, G.W, n, 1, G.part, G.cnt, G.nrm2, s);
    double r2 = 0.0;
    RC(sync_read(h, G.nrm2, &r2, 1));
    if (!std::isfinite(r2)) return HFDIB_ERR_DIVERGED;
    relres = bnorm > 0.0 ? sqrt(r2) / bnorm : 0.0;
    if (mv_out) *mv_out = mv;
    if (rel_out) *rel_out = relres;
    return relres <= tol ? HFDIB_OK : HFDIB_ERR_NOT_CONVERGED;
}

}  // namespace

extern "C" {

int hfdib_set_allocator(hfdib_alloc_fn alloc, hfdib_free_fn release, void* ctx) {
    if ((alloc == nullptr) != (release == nullptr)) return HFDIB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(alloc_mu());
    DevAlloc& a = alloc_setting();
    a.alloc = alloc;
    a.release = release;
    a.ctx = alloc ? ctx : nullptr;
    return HFDIB_OK;
}

void hfdib_default_options(hfdib_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->urf_u = 0.7;
    o->urf_p = 0.3;
    o->urf_turb = 0.85;
    o->n_u = 2;
    o->n_turb = 2;
    o->p_reltol = 0.1;
    o->p_maxiter = 50;
    o->precision = 0;
    o->precond = 1;
    o->p_check = 0;
    o->mg_coarse_sweeps = 4;
    o->graph = 1;
    o->p_persistent = 1;
    o->freeze_switch = 0;
}

const char* hfdib_error_string(int code) {
    switch (code) {
        case HFDIB_OK: return "ok";
        case HFDIB_ERR_INVALID_ARG: return "invalid argument";
        case HFDIB_ERR_CUDA: return "CUDA runtime error";
        case HFDIB_ERR_OOM: return "device out of memory";
        case HFDIB_ERR_NOT_CONVERGED: return "not converged";
        case HFDIB_ERR_DIVERGED: return "diverged (non-finite residual)";
        case HFDIB_ERR_STATE_MISMATCH: return "checkpoint does not match the handle";
        case HFDIB_ERR_TOO_LARGE: return "problem exceeds a fixed capacity of the call";
        case HFDIB_ERR_TIMEOUT: return "a device-wide barrier timed out";
        default: return "unknown error";
    }
}

int hfdib_create(const hfdib_grid* grid, const double* lambda, const double* ywall, int model, double Re,
                 const hfdib_bc* bc, const hfdib_options* opt, void* stream, hfdib_handle* out) {
    if (!out) return HFDIB_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grid || !lambda || !bc) return HFDIB_ERR_INVALID_ARG;
    if (grid->nx < 2 || grid->ny < 2 || grid->nz < 1) return HFDIB_ERR_INVALID_ARG;
    if (!(grid->dx > 0 && grid->dy > 0 && grid->dz > 0)) return HFDIB_ERR_INVALID_ARG;
    if (model < HFDIB_LAMINAR || model > HFDIB_REALIZABLE_KE) return HFDIB_ERR_INVALID_ARG;
    if (model == HFDIB_KOMEGA_SST && !ywall) return HFDIB_ERR_INVALID_ARG;
    if (!(Re > 0) || !(bc->u_ref > 0) || !(bc->l_ref > 0)) return HFDIB_ERR_INVALID_ARG;
    long long N = (long long)grid->nx * grid->ny * grid->nz;
    if (N > (1ll << 31) - 1) return HFDIB_ERR_INVALID_ARG;
    for (int s = 0; s < 6; ++s)
        if (bc->face[s] < HFDIB_BC_INLET || bc->face[s] > HFDIB_BC_EMPTY) return HFDIB_ERR_INVALID_ARG;
    if (grid->nz == 1) {
        if (bc->face[4] != HFDIB_BC_EMPTY || bc->face[5] != HFDIB_BC_EMPTY) return HFDIB_ERR_INVALID_ARG;
    }
    hfdib_options o;
    if (opt) o = *opt; else hfdib_default_options(&o);
    if (!(o.urf_u > 0 && o.urf_u <= 1) || !(o.urf_p > 0 && o.urf_p <= 1) || !(o.urf_turb > 0 && o.urf_turb <= 1))
        return HFDIB_ERR_INVALID_ARG;
    if (o.n_u < 1 || o.n_turb < 1 || o.p_maxiter < 0 || !(o.p_reltol >= 0)) return HFDIB_ERR_INVALID_ARG;
    if (o.precond < 0 || o.precond > 1 || o.p_check < 0 || o.mg_coarse_sweeps < 0) return HFDIB_ERR_INVALID_ARG;
    if (o.mg_tail_cells < 0 || o.mg_tail_cells > (1 << 20)) return HFDIB_ERR_INVALID_ARG;
    // the FP32 correction solve is a variant of the mixed persistent pressure solve
    if (o.p_cg32 < 0 || o.p_cg32 > 1 || (o.p_cg32 && o.precision != 1)) return HFDIB_ERR_INVALID_ARG;
    if (o.precision < 0 || o.precision > 1) return HFDIB_ERR_INVALID_ARG;
    if (o.wall_distance < 0 || o.wall_distance > 1) return HFDIB_ERR_INVALID_ARG;
    if (o.continuity_mask < 0 || o.continuity_mask > 1) return HFDIB_ERR_INVALID_ARG;
    if (o.convection < 0 || o.convection > 3) return HFDIB_ERR_INVALID_ARG;
    // the mixed path runs its FP32 V-cycle inside the persistent CG kernel
    if (o.precision == 1 && (o.p_persistent == 0 || o.precond != 1)) return HFDIB_ERR_INVALID_ARG;
    // the persistent solve is multigrid-preconditioned; Jacobi-PCG runs one launch per step
    if (o.precond == 0) o.p_persistent = 0;
    if (o.p_maxiter > 100000 || o.freeze_switch < 0) return HFDIB_ERR_INVALID_ARG;
    if (o.frozen_turbulence < 0 || o.frozen_turbulence > 1) return HFDIB_ERR_INVALID_ARG;

    Ctx* h = new (std::nothrow) Ctx();
    if (!h) return HFDIB_ERR_OOM;
    h->al = current_alloc();
    h->stream = (cudaStream_t)stream;
    if (!h->stream) {
        // graph capture needs a real stream: own a non-blocking one
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) { delete h; return HFDIB_ERR_CUDA; }
        h->own_stream = true;
    }
    h->opt = o;
    h->bc = *bc;
    h->coarse_sweeps = o.mg_coarse_sweeps > 0 ? o.mg_coarse_sweeps : 4;
    h->tail_cells = o.mg_tail_cells > 0 ? o.mg_tail_cells : PT_DEFAULT_TAIL_CELLS;
    h->use_graph = (o.graph != 0 && o.p_check == 0) ? 1 : 0;
    h->model = model;
    Grid& g = h->g;
    g.nx = grid->nx; g.ny = grid->ny; g.nz = grid->nz;
    g.dims = grid->nz == 1 ? 2 : 3;
    g.N = N;
    g.iN = 1.0 / (double)N;
    g.n[0] = g.nx; g.n[1] = g.ny; g.n[2] = g.nz;
    g.D[0] = grid->dx; g.D[1] = grid->dy; g.D[2] = grid->dz;
    g.o[0] = grid->x0; g.o[1] = grid->y0; g.o[2] = grid->z0;
    g.S[0] = g.D[1] * g.D[2]; g.S[1] = g.D[0] * g.D[2]; g.S[2] = g.D[0] * g.D[1];
    g.V = g.D[0] * g.D[1] * g.D[2];
    for (int d = 0; d < 3; ++d) {
        g.SoD[d] = g.S[d] / g.D[d];
        g.SoHD[d] = g.S[d] / (0.5 * g.D[d]);
        g.iD[d] = 1.0 / g.D[d];
    }
    // V^(1/3): sqrt(dx*dy) on one-cell-thick 2D grids
    g.h = g.dims == 2 ? sqrt(g.D[0] * g.D[1]) : pow(g.D[0] * g.D[1] * g.D[2], 1.0 / 3.0);
    for (int s = 0; s < 6; ++s) g.kind[s] = bc->face[s];
    for (int q = 0; q < 3; ++q) { g.u_in[q] = bc->u_in[q]; g.u_s[q] = bc->u_s[q]; }
    g.p_out = bc->p_out;
    g.nu = bc->u_ref * bc->l_ref / Re;
    g.stride[0] = 1; g.stride[1] = g.nx; g.stride[2] = (long long)g.nx * g.ny;
    g.nface[0] = (long long)(g.nx + 1) * g.ny * g.nz;
    g.nface[1] = (long long)g.nx * (g.ny + 1) * g.nz;
    g.nface[2] = (long long)g.nx * g.ny * (g.nz + 1);
    g.mask_b = o.continuity_mask;
    g.conv = o.convection;
    Params& P = h->P;
    P.model = model;
    P.urf_u = o.urf_u; P.urf_p = o.urf_p; P.urf_turb = o.urf_turb;
    P.iurf_u = 1.0 / o.urf_u; P.iurf_t = 1.0 / o.urf_turb;
    P.rlx_u = (1.0 - o.urf_u) / o.urf_u; P.rlx_t = (1.0 - o.urf_turb) / o.urf_turb;
    // inlet turbulence, Eq. (bcspkoein): k = 1.5 (U I)^2, eps = C_nu k^1.5 / l_t, omega = eps/(C_nu k)
    double U = sqrt(bc->u_in[0] * bc->u_in[0] + bc->u_in[1] * bc->u_in[1] + bc->u_in[2] * bc->u_in[2]);
    double kin = 1.5 * (U * bc->I_in) * (U * bc->I_in);
    double ein = C_MU * pow(kin, 1.5) / bc->lt_in;
    double win = ein / (C_MU * kin);
    P.k_in = kin;
    P.w_in = eps_model(model) ? ein : win;
    if (model != HFDIB_LAMINAR && !(kin > 0 && bc->lt_in > 0)) { delete h; return HFDIB_ERR_INVALID_ARG; }

    int rc = HFDIB_OK;
    Fields& F = h->F;
    memset(&F, 0, sizeof(F));
    unsigned int nb = nblocks(N);
    long long maxf = g.nface[0] > g.nface[1] ? g.nface[0] : g.nface[1];
    if (g.nface[2] > maxf) maxf = g.nface[2];
#define A(ptr, n) if (!rc) rc = dalloc_n(h, &(ptr), (n))
    A(h->lam, N);
    for (int q = 0; q < 3; ++q) {
        A(F.u[q], N); A(F.us[q], N); A(F.HbyA[q], N); A(F.bm[q], N); A(F.uib[q], N);
        A(F.phi[q], g.nface[q]); A(F.phiH[q], g.nface[q]);
    }
    A(F.p, N); A(F.pn, N); A(F.pr, N); A(F.rAU, N);
    A(F.k, N); A(F.w, N); A(F.w2, N); A(F.nut, N); A(F.kib, N); A(F.wib, N);
    A(F.G, 9 * N); A(F.mrow, 9 * N);
    if (o.convection == 3) A(F.Glim, 9 * N); A(F.Pk, N); A(F.S2, N); A(F.gam, N); A(F.gamk, N); A(F.sp, N); A(F.src, N); A(F.asus, N);
    A(F.bt, N); A(F.diag, N); A(F.ywall, N); A(F.flags, N);
    if (model == HFDIB_KOMEGA_SST) A(F.iyw, N);
    A(F.prhs, N); A(F.pdiag, N); A(F.r, N); A(F.z, N); A(F.d[0], N); A(F.d[1], N); A(F.q, N);
    A(F.scal, SC_NSCAL); A(F.partials, 16 * (long long)nb + 64); A(F.counters, 64);
    A(h->hist, HIST * HFDIB_NRES); A(h->res_dev, HFDIB_NRES + 1);
    A(h->cnt_scratch, (long long)nb + 2);
    // multigrid hierarchy of the pressure operator: level 0 is the grid
    // itself (x = z, b = r); coarsen by 2 while every dimension is >= 4
    if (!rc) {
        MgLevels& M = h->mg;
        memset(&M, 0, sizeof(M));
        Level& l0 = M.lv[0];
        l0.nx = g.nx; l0.ny = g.ny; l0.nz = g.nz; l0.N = N;
        for (int d = 0; d < 3; ++d) A(l0.cf[d], g.nface[d]);
        A(l0.diag, N); A(l0.idg, N);
        l0.x = F.z;
        l0.b = F.r;
        M.nl = 1;
        while (!rc && M.nl < MAX_LEVELS) {
            const Level& f = M.lv[M.nl - 1];
            int mn = f.nx < f.ny ? f.nx : f.ny;
            if (g.dims == 3 && f.nz < mn) mn = f.nz;
            if (mn < 4) break;
            Level c;
            c.nx = (f.nx + 1) / 2; c.ny = (f.ny + 1) / 2; c.nz = g.dims == 3 ? (f.nz + 1) / 2 : 1;
            c.N = (long long)c.nx * c.ny * c.nz;
            A(c.cf[0], (long long)(c.nx + 1) * c.ny * c.nz);
            A(c.cf[1], (long long)c.nx * (c.ny + 1) * c.nz);
            A(c.cf[2], (long long)c.nx * c.ny * (c.nz + 1));
            A(c.diag, c.N); A(c.idg, c.N); A(c.x, c.N); A(c.b, c.N);
            M.lv[M.nl++] = c;
        }
        h->tail_from = M.nl;
        for (int l = 1; l < M.nl; ++l)
            if (M.lv[l].N <= TAIL_CELLS) { h->tail_from = l; break; }
    }
    F.mixed = o.precision == 1 ? 1 : 0;
    F.lam = h->lam;
    h->pbuf0 = F.p;
    h->pbuf1 = F.pr;
    if (!rc && !F.mixed) A(F.r_alt, N);
    if (!rc && F.mixed) {
        for (int d = 0; d < 3; ++d) { A(F.phi32[d], g.nface[d]); A(F.r32[d], N); A(F.d32[d], N); }
        A(F.nut32, N); A(F.gam32, N); A(F.gamk32, N); A(F.diag32, N); A(F.z32, N);
        A(F.pd32[0], N); A(F.pd32[1], N); A(F.pq32, N); A(F.px32, N); A(F.pr32, N);
        // FP32 preconditioner hierarchy, same shapes as the FP64 one
        MgLevels32& M32 = h->mg32;
        memset(&M32, 0, sizeof(M32));
        M32.nl = h->mg.nl;
        for (int l = 0; l < M32.nl && !rc; ++l) {
            const Level& Ld = h->mg.lv[l];
            Level32& Lf = M32.lv[l];
            Lf.nx = Ld.nx; Lf.ny = Ld.ny; Lf.nz = Ld.nz; Lf.N = Ld.N;
            A(Lf.cf[0], (long long)(Lf.nx + 1) * Lf.ny * Lf.nz);
            A(Lf.cf[1], (long long)Lf.nx * (Lf.ny + 1) * Lf.nz);
            A(Lf.cf[2], (long long)Lf.nx * Lf.ny * (Lf.nz + 1));
            A(Lf.diag, Lf.N); A(Lf.idg, Lf.N); A(Lf.b, Lf.N);
            if (l == 0) Lf.x = F.z32;
            else A(Lf.x, Lf.N);
        }
    }
    if (!rc && o.p_persistent) {
        int dev = 0, nbk = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nbk, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nbk <= 0)
            rc = HFDIB_ERR_CUDA;
        h->pblocks = nbk;   // one block per SM: fewer arrivals per grid barrier
        A(h->ppart, 8 * (long long)nbk + 8);
        A(h->pbar, 2);
        A(h->perr, 1);
        h->err_src = h->perr;
        size_t dsz = pcgb_desc_size(F.mixed);
        for (int q = 0; q < 2 && !rc; ++q) rc = dalloc(h, &h->pdesc[q], dsz);
        // the problem's descriptor of the persistent solve, one per parity of
        // the p / pr buffers (a batch of one).  The upload goes on the
        // handle's stream, after the zero fill that dalloc queued there: a
        // synchronous copy runs on the legacy default stream, which does not
        // wait for a non-blocking stream, so the fill could land after it and
        // leave a zero descriptor (null pointers in the pressure kernel).
        std::vector<unsigned char> hd(2 * dsz);
        for (int q = 0; q < 2 && !rc; ++q) {
            Fields Fq = F;
            if (q == 1) std::swap(Fq.p, Fq.pr);
            unsigned char* hq = hd.data() + q * dsz;
            size_t by = F.mixed ? pcgb_describe32(hq, g, Fq, h->mg, h->mg32, h->ppart, h->tail_cells, PT_SMEM_BUDGET)
                                : pcgb_describe64(hq, g, Fq, h->mg, h->ppart, h->tail_cells, PT_SMEM_BUDGET);
            h->psmem = by;
            if (cudaMemcpyAsync(h->pdesc[q], hq, dsz, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
                rc = HFDIB_ERR_CUDA;
        }
        // (hd must outlive the copies)
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) rc = HFDIB_ERR_CUDA;
        int bps = 0;
        if (!rc && (pcgb_fits(F.mixed, g.dims, PT_THREADS, h->psmem, &bps) != 0 || bps < 1)) rc = HFDIB_ERR_CUDA;
    }
#undef A
    if (!rc && cudaMallocHost((void**)&h->pinned, 64 * sizeof(double)) != cudaSuccess) rc = HFDIB_ERR_OOM;
    if (rc) { free_all(h); delete h; return rc; }
    cudaStream_t s = h->stream;
    if (cudaMemcpyAsync(h->lam, lambda, N * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        (ywall && cudaMemcpyAsync(F.ywall, ywall, N * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)) {
        free_all(h); delete h; return HFDIB_ERR_CUDA;
    }
    // lambda must be finite and in [0, 1]
    k_check_lambda<<<nb, BLOCK, 0, s>>>(N, h->lam, F.partials, F.counters + 8, F.scal + 63);
    double bad = 0.0;
    if (sync_read(h, F.scal + 63, &bad, 1) != HFDIB_OK) { free_all(h); delete h; return HFDIB_ERR_CUDA; }
    if (bad != 0.0) { free_all(h); delete h; return HFDIB_ERR_INVALID_ARG; }
    if (model == HFDIB_KOMEGA_SST) launch_inv_wall_distance(g, F, s);

    // a0: groups, boundary-cell list and geometry
    launch_classify(g, h->lam, F.flags, s);
    launch_compact_bc(g, F.flags, h->cnt_scratch, h->cnt_scratch + nb, (int*)F.bt, s);
    int nbc = 0;
    if (cudaMemcpyAsync(&nbc, h->cnt_scratch + nb, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        free_all(h); delete h; return HFDIB_ERR_CUDA;
    }
    BcList& bl = h->bl;
    bl.nbc = nbc;
#define A(ptr, n) if (!rc) rc = dalloc_n(h, &(ptr), (n))
    A(bl.cell, nbc); A(bl.nbr, nbc); A(bl.cas, nbc); A(bl.clamped, nbc); A(bl.b1, 3 * (long long)nbc);
    A(bl.b2, 3 * (long long)nbc); A(bl.lamb, nbc); A(bl.n, 3 * (long long)nbc); A(bl.yp, nbc);
    A(bl.ye, nbc); A(bl.wS, nbc); A(bl.w1, nbc); A(bl.w2, nbc); A(bl.t1, 3 * (long long)nbc);
    A(bl.t2, 3 * (long long)nbc); A(bl.yplus, nbc);
    bl.ywf = o.wall_distance ? bl.yp : bl.ye;
#undef A
    if (rc) { free_all(h); delete h; return rc; }
    if (nbc > 0 && cudaMemcpyAsync(bl.cell, F.bt, nbc * sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        free_all(h); delete h; return HFDIB_ERR_CUDA;
    }
    launch_bc_geometry(g, h->lam, F.flags, bl, s);
    // initial state and face fluxes
    k_init_state<<<nb, BLOCK, 0, s>>>(g, P, F, model);
    launch_init_flux(g, F, s);
    refresh_mirrors(h);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        free_all(h); delete h; return HFDIB_ERR_CUDA;
    }
    *out = (hfdib_handle)h;
    return HFDIB_OK;
}

int hfdib_simple_sweep(hfdib_handle hh, int n_sweeps, double* residuals) {
    Ctx* h = (Ctx*)hh;
    if (!h || n_sweeps < 0) return HFDIB_ERR_INVALID_ARG;
    h->launches = 0;
    for (int n = 0; n < n_sweeps; ++n) {
        int rc = run_sweep(h);
        if (rc) return rc;
    }
    if (residuals) {
        int rc = read_residuals(h, residuals);
        if (rc) return rc;
        for (int q = 0; q < HFDIB_NRES; ++q)
            if (!isfinite(residuals[q])) return HFDIB_ERR_DIVERGED;
    }
    return HFDIB_OK;
}

int hfdib_solve_steady(hfdib_handle hh, double tol, int max_iter, int check_every, int* iters_out,
                       double* final_res) {
    Ctx* h = (Ctx*)hh;
    if (!h || max_iter < 0 || !(tol >= 0)) return HFDIB_ERR_INVALID_ARG;
    if (check_every <= 0) check_every = 10;
    h->launches = 0;
    double res[HFDIB_NRES] = {0};
    int it = 0;
    int status = HFDIB_ERR_NOT_CONVERGED;
    while (it < max_iter) {
        int rc = run_sweep(h);
        if (rc) return rc;
        ++it;
        if (it % check_every == 0 || it == max_iter) {
            rc = read_residuals(h, res);
            if (rc) return rc;
            double mx = 0.0;
            bool bad = false;
            for (int q = 0; q <= HFDIB_RES_K; ++q) {
                if (!isfinite(res[q])) bad = true;
                mx = fmax(mx, res[q]);
            }
            if (bad) { status = HFDIB_ERR_DIVERGED; break; }
            if (mx <= tol) { status = HFDIB_OK; break; }
        }
    }
    if (iters_out) *iters_out = it;
    if (final_res) memcpy(final_res, res, sizeof(res));
    return status;
}

int hfdib_get_field(hfdib_handle hh, int field, double* dst) {
    Ctx* h = (Ctx*)hh;
    if (!h || !dst) return HFDIB_ERR_INVALID_ARG;
    long long n;
    double* src = field_ptr(h, field, &n);
    if (!src) return HFDIB_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    return HFDIB_OK;
}

int hfdib_set_field(hfdib_handle hh, int field, const double* srcp) {
    Ctx* h = (Ctx*)hh;
    if (!h || !srcp) return HFDIB_ERR_INVALID_ARG;
    long long n;
    double* dst = field_ptr(h, field, &n);
    if (!dst) return HFDIB_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(dst, srcp, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    refresh_mirrors(h);
    h->g_cur = false;
    return HFDIB_OK;
}

int hfdib_get_tags(hfdib_handle hh, uint8_t* tags, int64_t* n_bc) {
    Ctx* h = (Ctx*)hh;
    if (!h) return HFDIB_ERR_INVALID_ARG;
    if (n_bc) *n_bc = h->bl.nbc;
    if (tags) {
        // low byte of the flags holds the group in bits 0-1
        std::vector<uint16_t> f(h->g.N);
        CK(cudaMemcpyAsync(f.data(), h->F.flags, h->g.N * sizeof(uint16_t), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        std::vector<uint8_t> t(h->g.N);
        for (long long c = 0; c < h->g.N; ++c) t[c] = (uint8_t)(f[c] & F_TAG);
        CK(cudaMemcpyAsync(tags, t.data(), h->g.N, cudaMemcpyHostToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    return HFDIB_OK;
}

int hfdib_get_bc_list(hfdib_handle hh, int64_t* ints, int64_t* ints2, double* reals) {
    Ctx* h = (Ctx*)hh;
    if (!h) return HFDIB_ERR_INVALID_ARG;
    launch_export_bc(h->bl, (long long*)ints, (long long*)ints2, reals, h->stream);
    CK(cudaGetLastError());
    return HFDIB_OK;
}

int hfdib_get_history(hfdib_handle hh, int count, double* host, int* n_out) {
    Ctx* h = (Ctx*)hh;
    if (!h || !host || count < 0) return HFDIB_ERR_INVALID_ARG;
    long long avail = h->sweeps < HIST ? h->sweeps : HIST;
    int n = (int)(count < avail ? count : avail);
    std::vector<double> all(HIST * HFDIB_NRES);
    CK(cudaMemcpyAsync(all.data(), h->hist, all.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int r = 0; r < n; ++r) {
        long long sw = h->sweeps - n + r;
        memcpy(host + (size_t)r * HFDIB_NRES, all.data() + (sw % HIST) * HFDIB_NRES, HFDIB_NRES * sizeof(double));
    }
    if (n_out) *n_out = n;
    return HFDIB_OK;
}

// checkpoint layout: header (8 x int64) then the FP64 arrays in a fixed order
static void state_arrays(Ctx* h, std::vector<std::pair<double*, long long>>& v) {
    const Grid& g = h->g;
    for (int q = 0; q < g.dims; ++q) v.push_back({h->F.u[q], g.N});
    v.push_back({h->F.p, g.N});
    for (int q = 0; q < g.dims; ++q) v.push_back({h->F.phi[q], g.nface[q]});
    v.push_back({h->F.k, g.N});
    v.push_back({h->F.w, g.N});
    v.push_back({h->F.w2, g.N});
    v.push_back({h->F.nut, g.N});
}

int hfdib_get_state(hfdib_handle hh, void* buf, size_t* bytes) {
    Ctx* h = (Ctx*)hh;
    if (!h || !bytes) return HFDIB_ERR_INVALID_ARG;
    std::vector<std::pair<double*, long long>> v;
    state_arrays(h, v);
    size_t total = 8 * sizeof(int64_t);
    for (auto& a : v) total += a.second * sizeof(double);
    if (!buf) { *bytes = total; return HFDIB_OK; }
    if (*bytes < total) return HFDIB_ERR_INVALID_ARG;
    int64_t* hd = (int64_t*)buf;
    hd[0] = (int64_t)STATE_MAGIC; hd[1] = h->g.nx; hd[2] = h->g.ny; hd[3] = h->g.nz; hd[4] = h->model;
    hd[5] = h->sweeps; hd[6] = (int64_t)total; hd[7] = 0;
    char* p = (char*)buf + 8 * sizeof(int64_t);
    for (auto& a : v) {
        CK(cudaMemcpyAsync(p, a.first, a.second * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        p += a.second * sizeof(double);
    }
    CK(cudaStreamSynchronize(h->stream));
    *bytes = total;
    return HFDIB_OK;
}

int hfdib_set_state(hfdib_handle hh, const void* buf, size_t bytes) {
    Ctx* h = (Ctx*)hh;
    if (!h || !buf) return HFDIB_ERR_INVALID_ARG;
    std::vector<std::pair<double*, long long>> v;
    state_arrays(h, v);
    size_t total = 8 * sizeof(int64_t);
    for (auto& a : v) total += a.second * sizeof(double);
    if (bytes != total) return HFDIB_ERR_STATE_MISMATCH;
    const int64_t* hd = (const int64_t*)buf;
    if (hd[0] != (int64_t)STATE_MAGIC || hd[1] != h->g.nx || hd[2] != h->g.ny || hd[3] != h->g.nz ||
        hd[4] != h->model || hd[6] != (int64_t)total)
        return HFDIB_ERR_STATE_MISMATCH;
    const char* p = (const char*)buf + 8 * sizeof(int64_t);
    for (auto& a : v) {
        CK(cudaMemcpyAsync(a.first, p, a.second * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        p += a.second * sizeof(double);
    }
    refresh_mirrors(h);
    double ns = (double)hd[5];
    CK(cudaMemcpyAsync(h->F.scal + SC_NSWEEP, &ns, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->sweeps = hd[5];
    h->g_cur = false;
    return HFDIB_OK;
}

int hfdib_profile_sweeps(hfdib_handle hh, int n_sweeps, double* total_us, int64_t* calls, int n_classes) {
    Ctx* h = (Ctx*)hh;
    if (!h || n_sweeps < 0 || !total_us || !calls || n_classes < HFDIB_K_COUNT) return HFDIB_ERR_INVALID_ARG;
    for (int q = 0; q < n_classes; ++q) { total_us[q] = 0.0; calls[q] = 0; }
    h->prof.on = true;
    h->prof.used = 0;
    h->prof.marks.clear();
    int rc = HFDIB_OK;
    for (int n = 0; n < n_sweeps && rc == HFDIB_OK; ++n) rc = run_sweep_host(h);
    h->prof.on = false;
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    for (auto& m : h->prof.marks) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, m.second.first, m.second.second));
        total_us[m.first] += 1e3 * (double)ms;
        calls[m.first] += 1;
    }
    h->prof.marks.clear();
    return HFDIB_OK;
}

int hfdib_get_launch_counts(hfdib_handle hh, int64_t* per_sweep, int64_t* per_pcg_iteration) {
    Ctx* h = (Ctx*)hh;
    if (!h) return HFDIB_ERR_INVALID_ARG;
    long long La = 0, Lb = 0, Lp = 0;
    // count by enqueueing nothing: replicate the schedule's arithmetic
    bool turb = h->model != HFDIB_LAMINAR;
    int jac = h->opt.precond == 0;
    int tf = h->tail_from;
    La = (turb ? 1 : 0) + (grad_u_carried(h) ? 3 : 4) + (h->g.conv == 3 ? 1 : 0) + 2 * h->opt.n_u + 2 +
         (h->pblocks > 0 ? 1 : (1 + (tf - 1) + (tf < h->mg.nl ? 1 : 0)) + 1 + (jac ? 0 : 5 * tf + 1) + 1);
    bool turb_b = turb && !h->opt.frozen_turbulence;
    Lb = 1 + (turb_b ? 4 + 2 * h->opt.n_turb + 2 + 2 * h->opt.n_turb + 1 : 0) + 1;
    Lp = h->pblocks > 0 ? 0 : 3 + (jac ? 0 : 5 * tf + 1);
    if (per_sweep) *per_sweep = La + Lb;
    if (per_pcg_iteration) *per_pcg_iteration = Lp;
    return HFDIB_OK;
}

int hfdib_get_counters(hfdib_handle hh, int64_t* sweeps, int64_t* launches) {
    Ctx* h = (Ctx*)hh;
    if (!h) return HFDIB_ERR_INVALID_ARG;
    if (sweeps) *sweeps = h->sweeps;
    if (launches) *launches = h->launches;
    return HFDIB_OK;
}

int hfdib_ib_force(hfdib_handle hh, double* force) {
    Ctx* h = (Ctx*)hh;
    if (!h || !force) return HFDIB_ERR_INVALID_ARG;
    const Grid& g = h->g;
    Fields F = h->F;
    cudaStream_t s = h->stream;
    // the imposed fields and grad u of the current state, as the next sweep sets them
    launch_imposed(g, h->model, h->opt.freeze_switch, h->bl, F.flags, F.scal, F.u[0], F.u[1], F.u[2], F.k,
                   F.uib[0], F.uib[1], F.uib[2], F.kib, F.wib, s);
    CK(cudaMemsetAsync(F.scal + SC_NLAM, 0, 2 * sizeof(double), s));
    launch_grad_u(g, F, s);
    if (g.conv == 3) launch_conv_limit(g, F, s);
    launch_ib_force(g, F, s);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(force, F.scal + SC_FORCE, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return HFDIB_OK;
}

int hfdib_force_coefficients(hfdib_handle hh, double A_ref, double gamma, double* coeffs) {
    Ctx* h = (Ctx*)hh;
    if (!h || !coeffs || !isfinite(gamma) || !(A_ref >= 0.0)) return HFDIB_ERR_INVALID_ARG;
    const Grid& g = h->g;
    if (A_ref == 0.0) {
        // Eqs. dragcoeff, dlcoeffs: A_ref = l_ref dz on a one-cell-thick grid
        if (g.dims != 2) return HFDIB_ERR_INVALID_ARG;
        A_ref = h->bc.l_ref * g.D[2];
    }
    double U2 = g.u_in[0] * g.u_in[0] + g.u_in[1] * g.u_in[1] + g.u_in[2] * g.u_in[2];
    if (!(U2 > 0.0)) return HFDIB_ERR_INVALID_ARG;
    double force[6];
    int rc = hfdib_ib_force(hh, force);
    if (rc) return rc;
    launch_force_coefficients(h->F, A_ref, U2, gamma, h->stream);
    CK(cudaGetLastError());
    return sync_read(h, h->F.scal + SC_COEF, coeffs, 2);
}

int hfdib_wall_shear(hfdib_handle hh, int side, double* tau, int64_t* n_faces_out) {
    Ctx* h = (Ctx*)hh;
    if (!h || side < 0 || side > 5) return HFDIB_ERR_INVALID_ARG;
    const Grid& g = h->g;
    int d = side >> 1;
    if (d >= g.dims || g.kind[side] != HFDIB_BC_WALL) return HFDIB_ERR_INVALID_ARG;
    long long nf = 1;
    for (int a = 0; a < 3; ++a)
        if (a != d) nf *= g.n[a];
    if (n_faces_out) *n_faces_out = nf;
    if (!tau) return HFDIB_OK;
    launch_wall_shear(g, h->F, side, nf, tau, h->stream);
    CK(cudaGetLastError());
    return HFDIB_OK;
}

int hfdib_recirculation(hfdib_handle hh, double x_rear, double* out) {
    Ctx* h = (Ctx*)hh;
    if (!h || !out || !(x_rear == x_rear)) return HFDIB_ERR_INVALID_ARG;
    const Grid& g = h->g;
    const Fields& F = h->F;
    cudaStream_t s = h->stream;
    unsigned int* count = F.counters + 13;
    CK(cudaMemsetAsync(count, 0, sizeof(unsigned int), s));
    launch_recirc(g, F, x_rear, count, s);
    CK(cudaGetLastError());
    double len = 0.0;
    unsigned int n = 0;
    CK(cudaMemcpyAsync(&len, F.scal + SC_RECIRC, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&n, count, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    out[0] = n ? len : 0.0;
    out[1] = (double)n * g.V;
    out[2] = (double)n;
    return HFDIB_OK;
}

int hfdib_adjoint_grad(hfdib_handle hh, int objective, double tol, int max_iter, int gmres_restart,
                       double* dJ_dlambda, double* J_out, int* iters_out, double* change_out) {
    Ctx* h = (Ctx*)hh;
    if (iters_out) *iters_out = 0;
    if (change_out) *change_out = 0.0;
    if (!h) return HFDIB_ERR_INVALID_ARG;
    if (objective != HFDIB_OBJ_PRESSURE_DROP && objective != HFDIB_OBJ_DRAG) return HFDIB_ERR_INVALID_ARG;
    const bool drag = objective == HFDIB_OBJ_DRAG;
    if (h->g.conv != 0) return HFDIB_ERR_INVALID_ARG;
    if (!(tol > 0.0) || max_iter < 0 || (max_iter > 0 && !dJ_dlambda)) return HFDIB_ERR_INVALID_ARG;
    if (gmres_restart < 0 || gmres_restart > HFDIB_GMRES_MAX_RESTART) return HFDIB_ERR_INVALID_ARG;
    const Grid& g = h->g;
    cudaStream_t s = h->stream;
    RC(adj_alloc(h));
    Adj& A = h->adj;
    Fields F = h->F;
    F.mixed = 0;
    if (max_iter == 0 && !drag) {
        // the objective alone
        launch_adj_objective(g, F, A, s);
        CK(cudaGetLastError());
        double J = 0.0;
        RC(sync_read(h, F.scal + SC_ADJ_J, &J, 1));
        if (J_out) *J_out = J;
        return HFDIB_OK;
    }
    RC(adj_setup(h));
    if (max_iter == 0) {
        // the drag alone (it needs the rows and u_ib of the set-up)
        launch_adj_drag_value(g, F, A, s);
        CK(cudaGetLastError());
        double J = 0.0;
        RC(sync_read(h, F.scal + SC_ADJ_J, &J, 1));
        if (J_out) *J_out = J;
        return HFDIB_OK;
    }
    // right-hand side J_x^T of the adjoint
    CK(cudaMemsetAsync(A.vb, 0, A.nvec * sizeof(double), s));
    if (drag) {
        // the objective's own derivative through the reverse-pass tail; its
        // u_ib-bar (the explicit lambda dependence) is kept in fixs
        launch_adj_drag_seed(g, F, A, s);
        launch_adj_transpose(g, F, A, s);
        launch_adj_gradu(g, F, h->bl, A, s);
        launch_adj_phi(g, F, A, s);
        CK(cudaMemcpyAsync(A.vb, A.vxb, A.nvec * sizeof(double), cudaMemcpyDeviceToDevice, s));
        for (int q = 0; q < g.dims; ++q)
            CK(cudaMemcpyAsync(A.fixs[q], A.fixb[q], g.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
        CK(cudaMemcpyAsync(A.vbp, A.jw, g.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    const bool warm = true;
    const double ptol = 1e-12;
    CK(cudaMemsetAsync(A.ps, 0, g.N * sizeof(double), s));
    adj_drop_graph(h);
    if (adj_build_graph(h, ptol, warm) != HFDIB_OK) {
        // capture not possible here: abandon it and run the pass host-driven
        cudaStreamCaptureStatus st;
        if (cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
            cudaGraph_t gg = nullptr;
            cudaStreamEndCapture(s, &gg);
            if (gg) cudaGraphDestroy(gg);
        }
        cudaGetLastError();
        adj_drop_graph(h);
    }
    int rc = HFDIB_OK, it = 0;
    double change = 0.0;
    if (gmres_restart > 0) {
        rc = adj_gmres(h, gmres_restart, tol, max_iter, &it, &change);
        if (rc != HFDIB_OK && rc != HFDIB_ERR_NOT_CONVERGED) { adj_drop_graph(h); return rc; }
    } else {
        // plain reverse fixed point psi <- G_x^T psi + J_x^T
        CK(cudaMemsetAsync(A.vpsi, 0, A.nvec * sizeof(double), s));
        double ch[2] = {0.0, 0.0};
        rc = HFDIB_ERR_NOT_CONVERGED;
        for (it = 0; it < max_iter;) {
            int r = adj_pass(h, ptol, warm);
            if (r) { adj_drop_graph(h); return r; }
            launch_adj_next(g, F, A, it == 0, s);
            ++it;
            if (it % 10 == 0 || it == max_iter) {
                r = sync_read(h, F.scal + SC_ADJ_DIFF, ch, 2);
                if (r) { adj_drop_graph(h); return r; }
                if (!std::isfinite(ch[0]) || !std::isfinite(ch[1])) { adj_drop_graph(h); return HFDIB_ERR_DIVERGED; }
                if (ch[0] <= tol * ch[1]) { rc = HFDIB_OK; break; }
            }
        }
        change = ch[1] > 0.0 ? ch[0] / ch[1] : ch[0];
    }
    adj_drop_graph(h);
    if (iters_out) *iters_out = it;
    if (change_out) *change_out = change;
    CK(cudaMemsetAsync(A.dlam, 0, g.N * sizeof(double), s));
    launch_adj_dlambda(g, F, h->bl, h->lam, A, s);
    launch_adj_dlambda_mask(g, F, A, s);
    if (drag) {
        // plus the explicit dependence of the drag on lambda through u_ib
        Adj Ae = A;
        for (int q = 0; q < 3; ++q) Ae.fixb[q] = A.fixs[q];
        launch_adj_dlambda(g, F, h->bl, h->lam, Ae, s);
    }
    CK(cudaMemcpyAsync(dJ_dlambda, A.dlam, g.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (drag) launch_adj_drag_value(g, F, A, s);
    else launch_adj_objective(g, F, A, s);
    CK(cudaGetLastError());
    double J = 0.0;
    RC(sync_read(h, F.scal + SC_ADJ_J, &J, 1));
    if (J_out) *J_out = J;
    return rc;
}

int hfdib_pressure_trace(hfdib_handle hh, int64_t* out, int capacity, int* n_out) {
    Ctx* h = (Ctx*)hh;
    if (!h || !out || capacity < 1 || capacity > (1 << 20)) return HFDIB_ERR_INVALID_ARG;
    if (h->pblocks <= 0 || !h->pdesc[0]) return HFDIB_ERR_INVALID_ARG;    // needs the persistent pressure kernel
    long long* dev = nullptr;
    size_t bytes = (1 + 2 * (size_t)capacity) * sizeof(long long);
    int rc = dev_alloc(h->al, h->stream, bytes, (void**)&dev);
    if (rc) return rc;
    if (cudaMemsetAsync(dev, 0, bytes, h->stream) != cudaSuccess) rc = HFDIB_ERR_CUDA;
    std::vector<long long> host(1 + 2 * (size_t)capacity);
    if (!rc) {
        h->trace = dev;
        h->trace_cap = capacity;
        int ug = h->use_graph;
        h->use_graph = 0;       // one host-driven sweep: the trace pointer is a launch argument
        rc = run_sweep_host(h);
        h->use_graph = ug;
        h->trace = nullptr;
        h->trace_cap = 0;
    }
    if (!rc && (cudaMemcpyAsync(host.data(), dev, bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
                cudaStreamSynchronize(h->stream) != cudaSuccess))
        rc = HFDIB_ERR_CUDA;
    cudaStreamSynchronize(h->stream);
    dev_free(h->al, h->stream, DevBlock{dev, bytes});
    if (rc) return rc;
    int n = (int)host[0];
    for (int i = 0; i < 2 * n; ++i) out[i] = host[1 + i];
    if (n_out) *n_out = n;
    return HFDIB_OK;
}

int hfdib_set_barrier_polls(hfdib_handle hh, int64_t polls) {
    Ctx* h = (Ctx*)hh;
    if (!h || polls < 0) return HFDIB_ERR_INVALID_ARG;
    long long v = polls > 0 ? (long long)polls : BARRIER_POLLS;
    if (v != h->spin_limit) {
        h->spin_limit = v;
        // the limit is a launch argument of the captured sweep: recapture
        CK(cudaStreamSynchronize(h->stream));
        for (int q = 0; q < 2; ++q) {
            if (h->gexec[q]) cudaGraphExecDestroy(h->gexec[q]);
            if (h->graph[q]) cudaGraphDestroy(h->graph[q]);
            h->gexec[q] = nullptr;
            h->graph[q] = nullptr;
        }
    }
    return HFDIB_OK;
}

void hfdib_destroy(hfdib_handle hh) {
    Ctx* h = (Ctx*)hh;
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

int hfdib_create_batch(int B, const hfdib_grid* grids, const double* const* lambdas, const double* const* ywalls,
                       int model, const double* Re, const hfdib_bc* bcs, const hfdib_options* opt, void* stream,
                       hfdib_batch* out) {
    if (!out) return HFDIB_ERR_INVALID_ARG;
    *out = nullptr;
    if (B < 1 || B > pcgb_max_batch() || !grids || !lambdas || !Re || !bcs) return HFDIB_ERR_INVALID_ARG;
    hfdib_options o;
    if (opt) o = *opt; else hfdib_default_options(&o);
    if (o.precond != 1) return HFDIB_ERR_INVALID_ARG;   // batched solve: multigrid preconditioner
    if (o.p_cg32) return HFDIB_ERR_INVALID_ARG;         // the FP32 correction solve is single-problem
    o.p_persistent = 1;
    for (int i = 1; i < B; ++i)
        if ((grids[i].nz == 1) != (grids[0].nz == 1)) return HFDIB_ERR_INVALID_ARG;   // all 2D or all 3D
    BatchCtx* b = new (std::nothrow) BatchCtx();
    if (!b) return HFDIB_ERR_OOM;
    b->al = current_alloc();
    b->B = B;
    b->mixed = o.precision == 1 ? 1 : 0;
    b->stream = (cudaStream_t)stream;
    if (!b->stream) {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) { delete b; return HFDIB_ERR_CUDA; }
        b->own_stream = true;
    }
    int rc = HFDIB_OK;
    // every problem is a handle on the batch's stream
    for (int i = 0; i < B && !rc; ++i) {
        hfdib_handle h = nullptr;
        rc = hfdib_create(&grids[i], lambdas[i], ywalls ? ywalls[i] : nullptr, model, Re[i], &bcs[i], &o, b->stream,
                          &h);
        if (rc) break;
        b->d.push_back((Ctx*)h);
    }
    if (!rc) b->dims = b->d[0]->g.dims;
    int dev = 0, sms = 0;
    if (!rc && (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess))
        rc = HFDIB_ERR_CUDA;
    b->nblk = sms;
    if (!rc && B > sms) rc = HFDIB_ERR_TOO_LARGE;   // problem b's tail runs on block b
    auto balloc = [&](void** p, size_t by) {
        if (rc) return;
        rc = dev_alloc(b->al, b->stream, by, p);
        if (!rc) b->allocs.push_back({*p, by});
    };
    {
        void *pb = nullptr, *pe = nullptr, *pl = nullptr;
        balloc(&pb, 256);
        balloc(&pe, 256);
        balloc(&pl, 256);
        if (!rc) {
            b->bar = (unsigned int*)pb;
            b->err = (int*)pe;
            b->loop = (unsigned int*)pl;
            cudaMemsetAsync(b->bar, 0, 256, b->stream);
            cudaMemsetAsync(b->err, 0, 256, b->stream);
            cudaMemsetAsync(b->loop, 0, 256, b->stream);
            for (Ctx* h : b->d) h->err_src = b->err;
        }
    }
    for (int i = 0; i < B && !rc; ++i) {
        void* p = nullptr;
        balloc(&p, sizeof(double) * 8 * (size_t)sms);
        if (rc) break;
        b->parts.push_back((double*)p);
        if (b->d[i]->mg.nl > b->maxlev) b->maxlev = b->d[i]->mg.nl;
    }
    balloc(&b->desc, pcgb_desc_size(b->mixed) * B);
    {
        void* p = nullptr;
        balloc(&p, sizeof(SweepProblem) * B);
        b->probs = (SweepProblem*)p;
        void* q = nullptr;
        balloc(&q, sizeof(int) * BK_KINDS * (B + 1));
        b->start = (int*)q;
    }
    b->hprobs.resize(B);
    if (!rc && cudaMallocHost((void**)&b->pinned, sizeof(double) * (HFDIB_NRES + 1) * B) != cudaSuccess)
        rc = HFDIB_ERR_OOM;
    b->coarse_sweeps = o.mg_coarse_sweeps > 0 ? o.mg_coarse_sweeps : 4;
    b->tail_cells = o.mg_tail_cells > 0 ? o.mg_tail_cells : PT_DEFAULT_TAIL_CELLS;   // as a single problem
    b->use_graph = o.graph != 0;
    // shape key of the autotuner cache
    if (!rc) {
        std::string k = std::to_string(B) + (b->mixed ? "m" : "d") + std::to_string(model);
        for (int i = 0; i < B; ++i)
            k += ":" + std::to_string(grids[i].nx) + "x" + std::to_string(grids[i].ny) + "x" + std::to_string(grids[i].nz);
        b->key = k;
        std::lock_guard<std::mutex> lock(tune_mu());
        auto it = tune_cache().find(k);
        if (it != tune_cache().end()) {
            b->threads = it->second.threads;
            b->tail_cells = it->second.tail_cells;
            b->coarse_sweeps = it->second.coarse_sweeps;
        }
    }
    if (!rc) rc = batch_describe(b);
    if (rc) { batch_free(b); return rc; }
    *out = (hfdib_batch)b;
    return HFDIB_OK;
}

int hfdib_batch_sweep(hfdib_batch bb, int n_sweeps, double* residuals) {
    BatchCtx* b = (BatchCtx*)bb;
    if (!b || n_sweeps < 0) return HFDIB_ERR_INVALID_ARG;
    for (int n = 0; n < n_sweeps; ++n) {
        int rc = batch_sweep_once(b);
        if (rc) return rc;
    }
    int rs = batch_sync_host(b);
    if (rs) return rs;
    if (residuals) {
        int rc = batch_read_residuals(b, residuals);
        if (rc) return rc;
        for (int q = 0; q < HFDIB_NRES * b->B; ++q)
            if (!isfinite(residuals[q])) return HFDIB_ERR_DIVERGED;
    }
    return HFDIB_OK;
}

int hfdib_batch_solve_steady(hfdib_batch bb, double tol, int max_iter, int check_every, int* iters_out,
                             double* final_res) {
    BatchCtx* b = (BatchCtx*)bb;
    if (!b || max_iter < 0 || !(tol >= 0)) return HFDIB_ERR_INVALID_ARG;
    if (check_every <= 0) check_every = 10;
    const int B = b->B;
    std::vector<double> res((size_t)HFDIB_NRES * B, 0.0);
    std::vector<long long> start_sweeps(B);
    for (int i = 0; i < B; ++i) start_sweeps[i] = b->d[i]->sweeps;
    // arm each problem's stop test, zero the loop counter
    {
        double arm[4] = {tol, 1.0, 0.0, 0.0};   // SC_STOP_TOL, SC_STOP_ON, SC_DONE, SC_DONE_AT
        for (Ctx* h : b->d) CK(cudaMemcpyAsync(h->F.scal + SC_STOP_TOL, arm, sizeof(arm), cudaMemcpyHostToDevice,
                                               b->stream));
        unsigned int lp[2] = {0u, (unsigned int)max_iter};
        CK(cudaMemcpyAsync(b->loop, lp, sizeof(lp), cudaMemcpyHostToDevice, b->stream));
        CK(cudaStreamSynchronize(b->stream));
    }
    long long ran = 0;
    if (max_iter > 0) {
        batch_ensure_grad_u(b);
        if (b->use_graph && !b->sgexec) {
            if (batch_build_solve_graph(b) != HFDIB_OK) {
                cudaStreamCaptureStatus st;
                if (cudaStreamIsCapturing(b->stream, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
                    cudaGraph_t g = nullptr;
                    cudaStreamEndCapture(b->stream, &g);
                    if (g) cudaGraphDestroy(g);
                }
                cudaGetLastError();
                b->use_graph = 0;
            }
        }
        if (b->use_graph) {
            // the whole solve: one graph launch, the loop and its stop test on the device
            CK(cudaGraphLaunch(b->sgexec, b->stream));
            unsigned int lp[2];
            CK(cudaMemcpyAsync(lp, b->loop, sizeof(lp), cudaMemcpyDeviceToHost, b->stream));
            CK(cudaStreamSynchronize(b->stream));
            ran = lp[0];
        } else {
            // host-driven fallback: the same sweeps, the stop flags read every check_every sweeps
            std::vector<double> done(B);
            while (ran < max_iter) {
                batch_enqueue(b, 1);
                CK(cudaGetLastError());
                ++ran;
                if (ran % check_every == 0 || ran == max_iter) {
                    for (int i = 0; i < B; ++i)
                        CK(cudaMemcpyAsync(b->pinned + i, b->d[i]->F.scal + SC_DONE, sizeof(double),
                                           cudaMemcpyDeviceToHost, b->stream));
                    CK(cudaStreamSynchronize(b->stream));
                    bool all = true;
                    for (int i = 0; i < B; ++i) all = all && b->pinned[i] != 0.0;
                    if (all) break;
                }
            }
        }
        b->sweeps += ran;
    }
    // disarm, read back the stop flags, the sweep counts and the residuals
    std::vector<double> flags(2 * (size_t)B);
    for (int i = 0; i < B; ++i) {
        CK(cudaMemcpyAsync(b->pinned + 2 * i, b->d[i]->F.scal + SC_DONE, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                           b->stream));
        CK(cudaMemsetAsync(b->d[i]->F.scal + SC_STOP_ON, 0, sizeof(double), b->stream));
    }
    CK(cudaStreamSynchronize(b->stream));
    memcpy(flags.data(), b->pinned, flags.size() * sizeof(double));
    int rc = batch_sync_host(b);
    if (rc) return rc;
    rc = batch_read_residuals(b, res.data());
    if (rc) return rc;
    int status = HFDIB_OK;
    for (int i = 0; i < B; ++i) {
        if (flags[2 * i] == 2.0) status = HFDIB_ERR_DIVERGED;
        else if (flags[2 * i] == 0.0 && status == HFDIB_OK) status = HFDIB_ERR_NOT_CONVERGED;
    }
    if (max_iter == 0) status = HFDIB_ERR_NOT_CONVERGED;
    if (iters_out)
        for (int i = 0; i < B; ++i)
            iters_out[i] = flags[2 * i] != 0.0 ? (int)((long long)flags[2 * i + 1] - start_sweeps[i])
                                               : (int)(b->d[i]->sweeps - start_sweeps[i]);
    if (final_res) memcpy(final_res, res.data(), sizeof(double) * res.size());
    return status;
}

int hfdib_batch_handle(hfdib_batch bb, int i, hfdib_handle* out) {
    BatchCtx* b = (BatchCtx*)bb;
    if (!b || !out || i < 0 || i >= b->B) return HFDIB_ERR_INVALID_ARG;
    *out = (hfdib_handle)b->d[i];
    return HFDIB_OK;
}

int hfdib_batch_autotune(hfdib_batch bb, int trial_sweeps, hfdib_tune* best_out) {
    BatchCtx* b = (BatchCtx*)bb;
    if (!b || trial_sweeps < 1) return HFDIB_ERR_INVALID_ARG;
    const int threads_c[2] = {512, 1024};
    const long long tail_c[3] = {256, 1024, 4096};
    const int coarse_c[3] = {2, 4, 8};
    hfdib_tune best{b->threads, (int)b->tail_cells, b->coarse_sweeps, 1e300, 0};
    int saved_graph = b->use_graph;
    b->use_graph = 0;   // trials run host-driven: parameters change between them
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int tried = 0;
    for (int t : threads_c)
        for (long long tc : tail_c)
            for (int cs : coarse_c) {
                b->threads = t;
                b->tail_cells = tc;
                b->coarse_sweeps = cs;
                if (batch_describe(b) != HFDIB_OK) continue;
                // warm one sweep, time the rest (the trial sweeps are real sweeps)
                int rc = batch_sweep_once(b);
                if (rc) return rc;
                CK(cudaEventRecord(e0, b->stream));
                for (int n = 0; n < trial_sweeps; ++n) {
                    rc = batch_sweep_once(b);
                    if (rc) return rc;
                }
                CK(cudaEventRecord(e1, b->stream));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                double us = 1e3 * ms / trial_sweeps;
                ++tried;
                if (us < best.us_per_sweep) best = hfdib_tune{t, (int)tc, cs, us, 0};
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    best.candidates = tried;
    b->threads = best.threads;
    b->tail_cells = best.tail_cells;
    b->coarse_sweeps = best.coarse_sweeps;
    int rc = batch_describe(b);
    if (rc) return rc;
    batch_drop_graphs(b);
    b->use_graph = saved_graph;
    {
        std::lock_guard<std::mutex> lock(tune_mu());
        tune_cache()[b->key] = best;
    }
    if (best_out) *best_out = best;
    return HFDIB_OK;
}

int hfdib_batch_set_barrier_polls(hfdib_batch bb, int64_t polls) {
    BatchCtx* b = (BatchCtx*)bb;
    if (!b || polls < 0) return HFDIB_ERR_INVALID_ARG;
    long long v = polls > 0 ? (long long)polls : BARRIER_POLLS;
    if (v != b->spin_limit) {
        b->spin_limit = v;
        CK(cudaStreamSynchronize(b->stream));
        batch_drop_graphs(b);   // the limit is a launch argument of the captured kernel
    }
    return HFDIB_OK;
}

void hfdib_destroy_batch(hfdib_batch bb) { batch_free((BatchCtx*)bb); }

}  // extern "C"
