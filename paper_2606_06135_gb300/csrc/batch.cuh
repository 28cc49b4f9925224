// batch.cuh -- one launch per phase of the SIMPLE sweep for a whole batch of
// problems (design candidates, angles of attack; grid sizes may differ).
//
// A batched launch gives each problem its own consecutive range of thread
// blocks: problem b owns blocks start[b] .. start[b+1]-1, as many as its own
// plain launch of the same kernel would have, so its kernel body (which
// indexes cells by Pos, common.cuh) sees the same block partition and
// reduces in the same order as when it runs alone.  A block finds its
// problem by binary search in start[], copies the problem's description into
// shared memory and runs the body.  A problem whose convergence flag is set
// (batch solves with the stop test on the device) skips every phase.
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace hf {

// everything one problem's sweep kernels read: the per-problem launch arguments
struct SweepProblem {
    Grid g;
    Params P;
    Fields F;
    BcList bl;
    Level L0;            // level-0 pressure operator (flux correction of a8)
    int freeze;          // option freeze_switch
    int model_end;       // model whose residuals the sweep record reports (laminar: frozen turbulence)
    const int* err;      // error word of the batch's pressure kernel
    double* res_out;     // residual record (HFDIB_NRES + 1)
    double* hist;        // residual history
    int nhist;
    double* done;        // F.scal + SC_DONE (the batch solve's per-problem stop flag)
    // the p / pr buffer pointers in the two device tables (this problem's
    // SweepProblem and its pressure descriptor), swapped on the device at the
    // end of every sweep the problem runs
    double** swap_p[2];
    double** swap_pr[2];
};

// launch kinds: how many blocks problem b gets in a plain launch
enum { BK_CELLS = 0,    // nblocks(N): one thread per cell
       BK_REDUCE = 1,   // rblocks(N): kernels ending in a grid reduction
       BK_PAIRS = 2,    // nblocks(npairs): red-black passes
       BK_BC = 3,       // nblocks(n_bc): boundary-cell list
       BK_ONE = 4,      // one block (its thread 0 works)
       BK_KINDS = 5 };

struct BatchTab {
    SweepProblem* probs;         // device, B entries
    const int* start;            // device, [BK_KINDS][B + 1] block offsets per kind
    int B;
    int skip;                    // 1: problems with the stop flag set skip the phase
};

template <int KIND, class Op>
__global__ void __launch_bounds__(BLOCK) k_batched(BatchTab T, Op op) {
    __shared__ SweepProblem sp;
    __shared__ int s_b, s_run;
    const int* st = T.start + KIND * (T.B + 1);
    if (threadIdx.x == 0) {
        int lo = 0, hi = T.B - 1;   // the last b with st[b] <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (st[mid] <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        s_b = lo;
        s_run = !(T.skip && *T.probs[lo].done != 0.0);
    }
    __syncthreads();
    if (!s_run) return;
    const int b = s_b;
    const unsigned int* src = (const unsigned int*)&T.probs[b];
    unsigned int* dst = (unsigned int*)&sp;
    for (int w = threadIdx.x; w < (int)(sizeof(SweepProblem) / 4); w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    op(Pos{(int)blockIdx.x - st[b], st[b + 1] - st[b]}, sp);
}

// batched launches of the sweep's phases (ib.cu, flow.cu, turb.cu); tot[kind]
// is the launch's total block count of that kind
void launchb_max_not_ic(const BatchTab& T, const int* tot, cudaStream_t s);
void launchb_imposed(const BatchTab& T, const int* tot, cudaStream_t s);
void launchb_means(const BatchTab& T, const int* tot, cudaStream_t s);
void launchb_grad_u(const BatchTab& T, const int* tot, cudaStream_t s);
void launchb_conv_limit(const BatchTab& T, const int* tot, cudaStream_t s);
void launchb_mom_asm(const BatchTab& T, const int* tot, cudaStream_t s);
void launchb_mom_smooth(const BatchTab& T, const int* tot, int colour, cudaStream_t s);
void launchb_mom_smooth32(const BatchTab& T, const int* tot, int colour, int zero_init, int finalize,
                          cudaStream_t s);
void launchb_hbya(const BatchTab& T, const int* tot, cudaStream_t s);
void launchb_phiH(const BatchTab& T, const int* tot, cudaStream_t s);
void launchb_update(const BatchTab& T, const int* tot, cudaStream_t s);
void launchb_sweep_end(const BatchTab& T, const int* tot, cudaStream_t s);
void launchb_turb_prep(const BatchTab& T, const int* tot, cudaStream_t s);
void launchb_bc_prod(const BatchTab& T, const int* tot, cudaStream_t s);
void launchb_scal_asm(const BatchTab& T, const int* tot, int eq, cudaStream_t s);
void launchb_scal_smooth(const BatchTab& T, const int* tot, int eq, int colour, cudaStream_t s);
void launchb_scal_smooth32(const BatchTab& T, const int* tot, int eq, int colour, int zero_init, cudaStream_t s);
void launchb_k_prep(const BatchTab& T, const int* tot, cudaStream_t s);
void launchb_turb_final(const BatchTab& T, const int* tot, cudaStream_t s);
// end of a batched solve's sweep: count it, and keep looping (conditional
// handle) while a problem is still running and fewer than max_iter sweeps ran
void launchb_next(const BatchTab& T, unsigned int* count, const unsigned int* max_iter,
                  cudaGraphConditionalHandle h, cudaStream_t s);

}  // namespace hf
