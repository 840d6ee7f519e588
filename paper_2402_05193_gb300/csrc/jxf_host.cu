// jxf_host.cu -- the C interface (include/jxf.h): handle, buffers, argument
// checks, the captured step graph, reductions and status reporting.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "jxf.h"
#include "jxf_nvtx.cuh"
#include "jxf_ops.cuh"
#include "jxf_setup.cuh"

using namespace jxf;

struct jxf_ctx {
    int device = 0;
    jxf_grid grid{};
    jxf_eos eos{};
    jxf_scheme scheme{};
    int ndim = 0, nv = 0;
    long long ncell = 0;
    size_t esize = 8;
    int nblk = 0;
    const Ops *ops = nullptr;
    Dev base{};
    // device buffers
    void *Un = nullptr, *Us = nullptr, *W = nullptr, *Tt = nullptr;
    void *F[3] = {nullptr, nullptr, nullptr}, *UH[3] = {nullptr, nullptr, nullptr};
    void *G = nullptr;  // per-cell auxiliary arrays: velocity gradient (viscous) or THINC normal
    int naux = 0;       // their count
    // fused last-axis sweep (ndim >= 2, whole grids): the stage writes its
    // primitives and temperature to the next of three buffers and its state
    // to a buffer the stage does not read
    int fused = 0;
    void *W2 = nullptr, *W3 = nullptr, *T2 = nullptr, *T3 = nullptr, *Us2 = nullptr;
    int nblk_step = 0;  // partial records of the step's last update
    void *rU = nullptr, *rW = nullptr, *rT = nullptr, *rD = nullptr;  // jxf_rhs scratch
    void *rG = nullptr;
    void *adj[10] = {nullptr};                                          // reverse-mode scratch
    void *sbar = nullptr;  // stencil-slot adjoints of one axis's faces
    double *W64 = nullptr;                                             // jxf_set_primitive scratch
    double *scal = nullptr, *part = nullptr;
    int *status = nullptr;
    unsigned long long *counters = nullptr;
    // block of a decomposed grid (jxf_create_block): the cell arrays Un, Us,
    // W, Tt, G hold three halo planes before and after the owned cells along
    // the split axis; the pointers above point at the first owned cell
    int block = 0;
    int split = -1;            // split axis
    int nbr[2] = {0, 0};       // sides of the split axis shared with a neighbour
    size_t plane = 0;          // cells per plane of the split axis
    void *pad_base[10] = {nullptr};  // allocations of Un, Us, W, Tt, G, W2, W3, T2, T3, Us2
    const void *cur_state = nullptr;  // state the next stage reads (its halo is exchanged)
    int wcur = 0;  // which of W, W2, W3 (and Tt, T2, T3) holds the current primitives
    int npart_cur = 0;  // partial records written by the block's last epilogue
    double *record = nullptr;  // reduction record [3 + MAXV]
    double *gather = nullptr;  // records of a same-process all-reduce (this block leads)
    int gather_cap = 0;
    // host side
    double *h_pin = nullptr;  // pinned readback: [t, status, ...]
    cudaStream_t cap = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    cudaGraphExec_t vjp_exec = nullptr;  // jxf_step_vjp's kernels for the step size vjp_dt
    double vjp_dt = 0.0;
    cudaStream_t last = nullptr;
    std::string err;
};

namespace {

const char *kNoHandle = "jxf: null handle";

jxf_status fail(jxf_ctx *h, jxf_status s, const std::string &msg) {
    if (h) h->err = msg;
    return s;
}

jxf_status cuda_fail(jxf_ctx *h, cudaError_t e, const char *what) {
    std::string m = std::string("jxf: ") + what + ": " + cudaGetErrorString(e);
    if (h) h->err = m;
    return e == cudaErrorMemoryAllocation ? JXF_ERR_OOM : JXF_ERR_CUDA;
}

#define JXF_CUDA(h, call)                                   \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

__global__ void k_set_scalar(double *dst, double v) { *dst = v; }

// Block b folds its contiguous share of the records [0, npart) into record b
// of out.
__global__ void __launch_bounds__(kPartThreads) k_reduce_partials(const double *part, int npart, int nv,
                                                                   double *out) {
    const int per = (npart + gridDim.x - 1) / gridDim.x;
    const int begin = min(npart, blockIdx.x * per);
    const int end = min(npart, begin + per);
    double a[3 + MAXV];
    reduce_records(part, begin, end, nv, a);
    if (threadIdx.x == 0) {
        double *o = out + (size_t)blockIdx.x * (3 + MAXV);
#pragma unroll
        for (int k = 0; k < 3 + MAXV; ++k) o[k] = a[k];
    }
}

__global__ void __launch_bounds__(kFinalThreads) k_finalize(const Dev P, const double *part, int npart, int nv,
                                                             int mode) {
    finalize_block(P, part, npart, nv, mode);
}

// Fold the partial records [0, npart) into one record (one warp).
__global__ void __launch_bounds__(kPartThreads) k_fold_records(const double *part, int npart, int nv,
                                                                double *out) {
    double a[3 + MAXV];
    reduce_records(part, 0, npart, nv, a);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 3 + MAXV; ++k) out[k] = a[k];
}

__global__ void k_selftest_div(const double *a, const double *b, double *q, long long n) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) q[k] = jxf::fdiv(a[k], b[k]);
}

template <typename T> __global__ void __launch_bounds__(256) k_fma_probe(T *out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = x[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) s += x[k];
    if (s == T(-1.2345)) out[0] = s;  // keeps the chains alive
}

const Ops *select_ops(int prec, int model, int ndim) {
    if (prec == JXF_FP64) return model == JXF_SPM ? ops_f64_spm(ndim) : ops_f64_dim(ndim);
    return model == JXF_SPM ? ops_f32_spm(ndim) : ops_f32_dim(ndim);
}

jxf_status launch_check(jxf_ctx *h, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    return JXF_OK;
}

// Reduction of the update kernel's per-block partials and the time-step
// logic; many partials are first folded to kPartGroups records by as many
// blocks (the single finalising block would be bound by one SM's FP64 rate).
// Partial records of the last update kernel: after a step (mode 1) the
// fused sweep's blocks, else the cell kernels' blocks.
int npart_of(const jxf_ctx *h, int mode) { return mode == 1 && h->fused ? h->nblk_step : h->nblk; }

int finalize_kernels(const jxf_ctx *h, int mode) {
    return mode != 2 && npart_of(h, mode) > 4 * kPartGroups ? 2 : 1;
}

jxf_status finalize(jxf_ctx *h, int mode, cudaStream_t s) {
    const double *part = h->part;
    int npart = npart_of(h, mode);
    if (finalize_kernels(h, mode) == 2) {
        double *grp = h->part + (size_t)npart * (3 + MAXV);
        k_reduce_partials<<<kPartGroups, kPartThreads, 0, s>>>(h->part, npart, h->nv, grp);
        part = grp;
        npart = kPartGroups;
    }
    k_finalize<<<1, kFinalThreads, 0, s>>>(h->base, part, npart, h->nv, mode);
    return launch_check(h, "k_finalize");
}

jxf_status set_scalar(jxf_ctx *h, int slot, double v, cudaStream_t s) {
    k_set_scalar<<<1, 1, 0, s>>>(h->scal + slot, v);
    return launch_check(h, "k_set_scalar");
}

// Primitives, temperature and diagnostics of the state in Un, then dt.
jxf_status derive_state(jxf_ctx *h, cudaStream_t s) {
    Dev P = h->base;
    P.Us = h->Un;
    P.Wout = h->W;
    P.Tout = h->Tt;
    P.W = h->W;
    P.G = h->G;
    h->ops->prim(P, 1, s);
    if (h->block) {  // the rest follows the halo exchange (jxf_block_phase)
        h->cur_state = h->Un;
        h->wcur = 0;
        h->npart_cur = h->nblk;
        return launch_check(h, "k_prim");
    }
    if (h->G) h->ops->aux(P, s);  // P.W = P.G's input: the new primitives
    jxf_status st = launch_check(h, "k_prim");
    if (st != JXF_OK) return st;
    return finalize(h, 0, s);
}

// Copy nv rows of a state between the caller's contiguous layout and a
// handle array (a block's rows are its padded variable stride apart).
jxf_status copy_rows(jxf_ctx *h, void *dst, const void *src, bool to_handle, int rows, cudaStream_t s) {
    const size_t w = (size_t)h->ncell * h->esize;
    const size_t hp = h->block ? (size_t)h->base.vstride * h->esize : w;
    JXF_CUDA(h, cudaMemcpy2DAsync(dst, to_handle ? hp : w, src, to_handle ? w : hp, w, (size_t)rows,
                                  cudaMemcpyDefault, s));
    return JXF_OK;
}

jxf_status block_unsupported(jxf_ctx *h, const char *what) {
    return fail(h, JXF_ERR_UNSUPPORTED,
                std::string("jxf: ") + what + " is not available for a block of a decomposed grid "
                "(it steps through jxf_block_phase)");
}

// Optional per-kernel event timing of enqueue_step (profiling entry only):
// timed regions of one or more kernels (nk: the kernels a region launched).
// Event-timed regions of one step: 3 stages x (up to 3 face sweeps + the
// update / auxiliary pass) + the finalisation.
constexpr int kTimedRegionsPerStep = 3 * 4 + 1;
struct KernelTimer {
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind, nk;
    int n = 0;
    bool ok = true;
    explicit KernelTimer(int regions) : ev(2 * (size_t)regions), kind(regions), nk(regions) {
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                e = nullptr;
                ok = false;
            }
    }
    ~KernelTimer() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
    void begin(int k, cudaStream_t s) {
        static const char *names[5] = {"sweep x", "sweep y", "last-axis sweep (fused with the update in float)",
                                       "update / auxiliary pass", "finalise"};
        nvtxRangePushA(names[k]);  // a named range per kernel kind on a timeline
        if (n >= (int)kind.size()) return;  // more regions than sized for: left untimed
        kind[n] = k;
        cudaEventRecord(ev[2 * n], s);
    }
    void end(cudaStream_t s, int kernels = 1) {
        nvtxRangePop();
        if (n >= (int)kind.size()) return;
        cudaEventRecord(ev[2 * n + 1], s);
        nk[n] = kernels;
        ++n;
    }
};

// Stage `stage` of TVD-RK3 with the fused last-axis sweep (the auxiliary
// pass excluded): see enqueue_step for the buffer rotation.
void fused_stage(jxf_ctx *h, Dev &P, int stage, cudaStream_t s, KernelTimer *kt) {
    static const double coef[3][3] = {{0.0, 1.0, 1.0}, {0.75, 0.25, 0.25}, {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0}};
    void *Wr[3] = {h->W, h->W2, h->W3}, *Tr[3] = {h->Tt, h->T2, h->T3};
    const void *Uin[3] = {h->Un, h->Us, h->Us2};
    void *Uo[3] = {h->Us, h->Us2, h->Un};
    P.ca = coef[stage][0];
    P.cb = coef[stage][1];
    P.cc = coef[stage][2];
    P.ca32 = (float)P.ca;
    P.cb32 = (float)P.cb;
    P.stage0 = stage == 0 ? 1 : 0;
    P.Un = h->Un;
    P.W = Wr[stage];
    P.Tt = Tr[stage];
    P.Ucell = Uin[stage];
    P.Us = Uin[stage];
    P.Uout = Uo[stage];
    P.Wout = Wr[(stage + 1) % 3];
    P.Tout = Tr[(stage + 1) % 3];
    for (int d = 0; d < h->ndim - 1; ++d) {
        if (kt) kt->begin(d, s);
        h->ops->flux(P, d, s);
        if (kt) kt->end(s);
    }
    if (kt) kt->begin(2, s);
    h->ops->flux_update(P, stage == 2 ? 1 : 0, s);
    if (kt) kt->end(s);
}

// One full TVD-RK3 step (§3.4) on the handle's buffers.  With the fused
// last-axis sweep the stage inputs and outputs rotate: primitives and
// temperature through three buffers (W -> W2 -> W3 -> W), the state
// Un -> Us -> Us2 -> Un, so that no stage writes what its stencils read and
// the step ends in the buffers it started from (the captured graph replays).
jxf_status enqueue_step(jxf_ctx *h, cudaStream_t s, KernelTimer *kt = nullptr) {
    static const double coef[3][3] = {{0.0, 1.0, 1.0}, {0.75, 0.25, 0.25}, {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0}};
    Dev P = h->base;
    P.dtp = h->scal + SC_DT;
    P.skip_if_done = 1;
    P.G = h->G;
    for (int stage = 0; stage < 3; ++stage) {
        if (h->fused) {
            fused_stage(h, P, stage, s, kt);
            if (h->G) {
                P.W = P.Wout;  // gradient / interface normal of the new primitives
                if (kt) kt->begin(3, s);
                h->ops->aux(P, s);
                if (kt) kt->end(s);
            }
            continue;
        }
        P.ca = coef[stage][0];
        P.cb = coef[stage][1];
        P.cc = coef[stage][2];
        P.ca32 = (float)P.ca;
        P.cb32 = (float)P.cb;
        P.stage0 = stage == 0 ? 1 : 0;
        P.Un = h->Un;
        P.W = h->W;
        P.Tt = h->Tt;
        P.Ucell = stage == 0 ? h->Un : h->Us;
        for (int d = 0; d < h->ndim; ++d) {
            if (kt) kt->begin(d, s);
            h->ops->flux(P, d, s);
            if (kt) kt->end(s);
        }
        P.Us = stage == 0 ? h->Un : h->Us;
        P.Uout = stage == 2 ? h->Un : h->Us;
        P.Wout = h->W;
        P.Tout = h->Tt;
        if (kt) kt->begin(3, s);
        h->ops->update(P, 1, stage == 2 ? 1 : 0, s);
        if (h->G) h->ops->aux(P, s);  // gradient / interface normal of the new primitives (P.W)
        if (kt) kt->end(s, h->G ? 2 : 1);
    }
    jxf_status st = launch_check(h, "step kernels");
    if (st != JXF_OK) return st;
    if (kt) kt->begin(4, s);
    st = finalize(h, 1, s);
    if (kt) kt->end(s, finalize_kernels(h, 1));
    return st;
}

jxf_status check_status(jxf_ctx *h, cudaStream_t s) {
    JXF_CUDA(h, cudaMemcpyAsync(h->h_pin, h->scal + SC_T, sizeof(double), cudaMemcpyDeviceToHost, s));
    JXF_CUDA(h, cudaMemcpyAsync(h->h_pin + 1, h->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    JXF_CUDA(h, cudaStreamSynchronize(s));
    int st;
    std::memcpy(&st, h->h_pin + 1, sizeof(int));
    if (st & ST_NONPHYSICAL)
        return fail(h, JXF_ERR_NONPHYSICAL, "jxf: non-admissible state (density, rho c^2 or non-finite) after a step");
    if (st & ST_BAD_DT) return fail(h, JXF_ERR_NONPHYSICAL, "jxf: non-finite or negative time step");
    if (st & ST_BOUNDS) return fail(h, JXF_ERR_BOUNDS, "jxf: a stencil or face index left its array (checked build)");
    return JXF_OK;
}

size_t state_bytes(const jxf_ctx *h) { return (size_t)h->nv * h->ncell * h->esize; }

// Host-side fault injection for the allocation-failure tests: when armed
// with jxf_fail_allocation_after(k), the k-th following device allocation of
// a handle reports cudaErrorMemoryAllocation without calling cudaMalloc.
std::atomic<int> g_fail_alloc_after{-1};

template <typename P> jxf_status dalloc(jxf_ctx *h, P **p, size_t bytes) {
    void *q = nullptr;
    int k = g_fail_alloc_after.load();
    while (k >= 0 && !g_fail_alloc_after.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 0) return cuda_fail(h, cudaErrorMemoryAllocation, "cudaMalloc (injected failure)");
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMalloc");
    *p = static_cast<P *>(q);
    return JXF_OK;
}

void free_all(jxf_ctx *h) {
    if (h->block) {  // the cell arrays point into their padded allocations
        for (void *&b : h->pad_base)
            if (b) cudaFree(b);
        h->Un = h->Us = h->W = h->Tt = h->G = nullptr;
        h->W2 = h->W3 = h->T2 = h->T3 = h->Us2 = nullptr;
        if (h->record) cudaFree(h->record);
        if (h->gather) cudaFree(h->gather);
    }
    void *bufs[] = {h->Un, h->Us, h->W, h->Tt, h->F[0], h->F[1], h->F[2], h->UH[0], h->UH[1], h->UH[2],
                    h->rU, h->rW, h->rT, h->rD, h->W64, h->scal, h->part, h->status, h->counters,
                    h->G, h->rG, h->W2, h->W3, h->T2, h->T3, h->Us2};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (void *b : h->adj)
        if (b) cudaFree(b);
    if (h->sbar) cudaFree(h->sbar);
    if (h->h_pin) cudaFreeHost(h->h_pin);
    if (h->step_exec) cudaGraphExecDestroy(h->step_exec);
    if (h->vjp_exec) cudaGraphExecDestroy(h->vjp_exec);
    if (h->cap) cudaStreamDestroy(h->cap);
}

jxf_status ensure_rhs_scratch(jxf_ctx *h) {
    if (h->rU) return JXF_OK;
    const size_t sb = state_bytes(h);
    jxf_status st;
    if ((st = dalloc(h, &h->rU, sb)) != JXF_OK) return st;
    if ((st = dalloc(h, &h->rW, sb)) != JXF_OK) return st;
    if ((st = dalloc(h, &h->rD, sb)) != JXF_OK) return st;
    if ((st = dalloc(h, &h->rT, (size_t)h->ncell * h->esize)) != JXF_OK) return st;
    if (h->G && (st = dalloc(h, &h->rG, (size_t)h->naux * h->ncell * h->esize)) != JXF_OK)
        return st;
    return JXF_OK;
}

// Reverse-mode scratch: [0] U copy, [1] U1, [2] U2, [3] R / vjp temporary,
// [4] Wbar, [5] Ubar(n+1), [6] Ubar2, [7] Ubar1, [8] Ubar(n), [9] R_bar copy.
enum { A_U0, A_U1, A_U2, A_TMP, A_WB, A_B3, A_B2, A_B1, A_BN, A_RB };

jxf_status ensure_adj_scratch(jxf_ctx *h) {
    jxf_status st = ensure_rhs_scratch(h);
    if (st != JXF_OK) return st;
    for (void *&b : h->adj)
        if (!b && (st = dalloc(h, &b, state_bytes(h))) != JXF_OK) return st;
    if (!h->sbar) {  // six slots per face and variable, every axis
        const size_t n = sbar_offset(h->base, h->ndim, h->ndim, h->nv);
        if ((st = dalloc(h, &h->sbar, n * h->esize)) != JXF_OK) return st;
    }
    return JXF_OK;
}

jxf_status check_vjp_supported(jxf_ctx *h) {
    if (h->block) return block_unsupported(h, "reverse mode");
    if (!h->ops->flux_vjp || h->scheme.viscous || h->scheme.limiter || h->scheme.recon >= JXF_TENO6A_COMP)
        return fail(h, JXF_ERR_UNSUPPORTED,
                    "jxf: reverse mode covers the single-phase model with WENO5, without viscous fluxes "
                    "or limiters");
    return JXF_OK;
}

// dU = R(U) for device U (rhs scratch for primitives and temperature).
jxf_status rhs_device(jxf_ctx *h, const void *U, void *dU, cudaStream_t s) {
    Dev P = h->base;
    P.Us = U;
    P.Wout = h->rW;
    P.Tout = h->rT;
    P.G = h->rG;
    h->ops->prim(P, 0, s);
    P.W = h->rW;
    P.Ucell = U;
    P.Tt = h->rT;
    P.dtp = h->scal + SC_RHS_DT;
    P.skip_if_done = 0;
    if (h->rG) h->ops->aux(P, s);
    for (int d = 0; d < h->ndim; ++d) h->ops->flux(P, d, s);
    P.dU = dU;
    h->ops->update(P, 0, 0, s);
    return launch_check(h, "rhs kernels");
}

// Ubar = (dR/dU)^T Rbar for device arrays.
jxf_status rhs_vjp_device(jxf_ctx *h, const void *U, const void *Rbar, void *Ubar, cudaStream_t s) {
    Dev P = h->base;
    P.Us = U;
    P.Wout = h->rW;
    P.Tout = h->rT;
    h->ops->prim(P, 0, s);
    P.W = h->rW;
    P.Rbar = Rbar;
    P.Wbar = h->adj[A_WB];
    P.Sbar = h->sbar;
    for (int d = 0; d < h->ndim; ++d) h->ops->flux_vjp(P, d, s);
    h->ops->gather_vjp(P, s);
    P.Ubar = Ubar;
    h->ops->prim_vjp(P, s);
    return launch_check(h, "vjp kernels");
}

// One RK stage of a block: the face sweeps and the cell update of stage s,
// as in enqueue_step (the auxiliary pass follows the halo exchange).
jxf_status block_stage(jxf_ctx *h, int stage, cudaStream_t s) {
    static const double coef[3][3] = {{0.0, 1.0, 1.0}, {0.75, 0.25, 0.25}, {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0}};
    Dev P = h->base;
    P.dtp = h->scal + SC_DT;
    P.skip_if_done = 1;
    P.G = h->G;
    if (h->fused) {
        if (h->wcur != stage)
            return fail(h, JXF_ERR_ARG, "jxf_block_phase: stages must follow 0, 1, 2 after a state or a step");
        fused_stage(h, P, stage, s, nullptr);
        h->cur_state = P.Uout;
        h->wcur = (stage + 1) % 3;
        if (stage == 2) h->npart_cur = h->nblk_step;
        return launch_check(h, "block stage kernels");
    }
    P.W = h->W;
    P.Tt = h->Tt;
    P.Ucell = stage == 0 ? h->Un : h->Us;
    for (int d = 0; d < h->ndim; ++d) h->ops->flux(P, d, s);
    P.Un = h->Un;
    P.Us = stage == 0 ? h->Un : h->Us;
    P.Uout = stage == 2 ? h->Un : h->Us;
    P.Wout = h->W;
    P.Tout = h->Tt;
    P.ca = coef[stage][0];
    P.cb = coef[stage][1];
    P.cc = coef[stage][2];
    P.ca32 = (float)P.ca;
    P.cb32 = (float)P.cb;
    P.stage0 = stage == 0 ? 1 : 0;
    h->ops->update(P, 1, stage == 2 ? 1 : 0, s);
    h->cur_state = P.Uout;
    if (stage == 2) h->npart_cur = h->nblk;
    return launch_check(h, "block stage kernels");
}

// Halo regions of a block: (array base at the first owned cell, rows).
int halo_regions(const jxf_ctx *h, int kind, const void *base[4], int rows[4]) {
    int n = 0;
    const size_t vs = (size_t)h->base.vstride * h->esize;
    if (kind == JXF_HALO_STATE) {
        const void *Wr[3] = {h->W, h->W2, h->W3}, *Tr[3] = {h->Tt, h->T2, h->T3};
        base[n] = Wr[h->wcur], rows[n++] = h->nv;
        if (h->eos.model == JXF_SPM && h->scheme.viscous) base[n] = Tr[h->wcur], rows[n++] = 1;
        if (h->scheme.limiter) base[n] = h->cur_state, rows[n++] = h->nv;
        if (h->base.thinc)  // psi, the last auxiliary array
            base[n] = static_cast<const unsigned char *>(h->G) + (size_t)h->ndim * vs, rows[n++] = 1;
    } else if (kind == JXF_HALO_AUX && h->G) {
        base[n] = h->G, rows[n++] = h->base.thinc ? h->ndim : h->naux;
    }
    return n;
}

// Address of the three planes next to (send) or beyond (receive) a side.
unsigned char *halo_ptr(const jxf_ctx *h, const void *base, int side, int recv) {
    const long long nax = h->base.n[h->split];
    const long long first = side == 0 ? (recv ? -3 : 0) : (recv ? nax : nax - 3);
    return const_cast<unsigned char *>(static_cast<const unsigned char *>(base)) +
           first * (long long)h->plane * (long long)h->esize;
}

// The split axis of a block (the last active one) and the checks of
// jxf_create_block on the block's extents and neighbour sides.
jxf_status check_block(const jxf_grid *grid, const jxf_block *b) {
    const int ax = grid->ndim - 1;
    for (int e = 0; e < 3; ++e) {
        if (e == ax) continue;
        if (b->lo[e] != 0 || b->n[e] != grid->n[e] || b->nbr[e][0] || b->nbr[e][1]) return JXF_ERR_ARG;
    }
    const int N = grid->n[ax];
    if (b->lo[ax] < 0 || b->n[ax] < 3 || b->lo[ax] + b->n[ax] > N) return JXF_ERR_ARG;
    for (int s = 0; s < 2; ++s) {
        const int nb = b->nbr[ax][s];
        if (nb != 0 && nb != 1) return JXF_ERR_ARG;
        const bool on_boundary = s == 0 ? b->lo[ax] == 0 : b->lo[ax] + b->n[ax] == N;
        if (!nb && !on_boundary) return JXF_ERR_ARG;  // an inner side must face a block
        if (nb && on_boundary && grid->bc[ax][s] != JXF_BC_PERIODIC) return JXF_ERR_ARG;
    }
    return JXF_OK;
}

// The block's kernel parameters: those of the whole grid (cell size,
// materials, scheme), with the block's extents, index divisors, padded
// variable stride and neighbour sides.
void fill_block_dev(const jxf_grid *grid, const jxf_eos *eos, const jxf_scheme *scheme, const jxf_block *b,
                    long long ncell, size_t plane, Dev &P) {
    fill_dev(grid, eos, scheme, ncell, P);
    const int ax = grid->ndim - 1;
    P.n[ax] = b->n[ax];
    P.ncell = ncell;
    P.vstride = (long long)(b->n[ax] + 6) * (long long)plane;
    P.cell_lo = -3 * (long long)plane;  // the halo planes
    P.cell_hi = ncell + 3 * (long long)plane;
    P.fd_cell[0] = FastDiv((unsigned)P.n[0]);
    P.fd_cell[1] = FastDiv((unsigned)P.n[1]);
    for (int d = 0; d < 3; ++d) {
        P.fd_face[d][0] = FastDiv((unsigned)(P.n[0] + (d == 0 ? 1 : 0)));
        P.fd_face[d][1] = FastDiv((unsigned)(P.n[1] + (d == 1 ? 1 : 0)));
    }
    for (int s = 0; s < 2; ++s)
        if (b->nbr[ax][s]) P.bc[ax][s] = JXF_BC_NEIGHBOR;
    // a lower side inside the grid: its face belongs to the block below
    P.skip_face0_count = b->nbr[ax][0] && b->lo[ax] > 0 ? 1 : 0;
}

jxf_status create_handle(const jxf_grid *grid, const jxf_eos *eos, const jxf_scheme *scheme,
                         const jxf_block *blk, jxf_handle *out) {
    if (!out) return JXF_ERR_ARG;
    *out = nullptr;
    long long ncell = 0;
    {
        const jxf_status vs = validate_setup(grid, eos, scheme, &ncell);
        if (vs != JXF_OK) return vs;
    }
    size_t plane = 0;
    if (blk) {
        const jxf_status bs = check_block(grid, blk);
        if (bs != JXF_OK) return bs;
        plane = 1;
        for (int e = 0; e < grid->ndim - 1; ++e) plane *= (size_t)grid->n[e];
        ncell = (long long)plane * blk->n[grid->ndim - 1];
    }
    jxf_ctx *h = new (std::nothrow) jxf_ctx();
    if (!h) return JXF_ERR_OOM;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return JXF_ERR_CUDA;
    }
    h->grid = *grid;
    h->eos = *eos;
    h->scheme = *scheme;
    h->ndim = grid->ndim;
    h->nv = grid->ndim + (eos->model == JXF_DIM ? 4 : 2);
    h->ncell = ncell;
    h->esize = scheme->precision == JXF_FP64 ? 8 : 4;
    h->nblk = (int)((ncell + kCellThreads - 1) / kCellThreads);
    h->ops = select_ops(scheme->precision, eos->model, grid->ndim);

    Dev &P = h->base;
    if (blk) {
        h->block = 1;
        h->split = grid->ndim - 1;
        h->nbr[0] = blk->nbr[h->split][0];
        h->nbr[1] = blk->nbr[h->split][1];
        h->plane = plane;
        for (int e = 0; e < 3; ++e) h->grid.n[e] = e < grid->ndim ? blk->n[e] : 1;
        fill_block_dev(grid, eos, scheme, blk, ncell, plane, P);
    } else {
        fill_dev(grid, eos, scheme, ncell, P);
    }
    // buffers
    const size_t sb = state_bytes(h);
    jxf_status st = JXF_OK;
    auto chk = [&](jxf_status s) { if (st == JXF_OK) st = s; };
    h->naux = aux_arrays(h->ndim, eos, scheme);
    if (blk) {
        // cell arrays with three halo planes on each side of the split axis
        const size_t vs = (size_t)P.vstride * h->esize, off = 3 * plane * h->esize;
        h->fused = h->ndim >= 2 && h->esize == 4 ? 1 : 0;
        const size_t nvr = (size_t)h->nv, f = (size_t)h->fused;
        void **dst[10] = {&h->Un, &h->Us, &h->W, &h->Tt, &h->G, &h->W2, &h->W3, &h->T2, &h->T3, &h->Us2};
        const size_t rows[10] = {nvr, nvr, nvr, 1, (size_t)h->naux, f * nvr, f * nvr, f, f, f * nvr};
        if (h->fused) {
            const dim3 fg = fused_grid(P, h->ndim);
            h->nblk_step = (int)(fg.x * fg.y * fg.z);
        }
        for (int k = 0; k < 10 && st == JXF_OK; ++k) {
            if (!rows[k]) continue;
            chk(dalloc(h, &h->pad_base[k], rows[k] * vs));
            if (st == JXF_OK) {
                cudaMemset(h->pad_base[k], 0, rows[k] * vs);
                *dst[k] = static_cast<unsigned char *>(h->pad_base[k]) + off;
            }
        }
        chk(dalloc(h, &h->record, (3 + MAXV) * sizeof(double)));
    } else {
        chk(dalloc(h, &h->Un, sb));
        chk(dalloc(h, &h->Us, sb));
        chk(dalloc(h, &h->W, sb));
        chk(dalloc(h, &h->Tt, (size_t)ncell * h->esize));
        if (h->naux) chk(dalloc(h, &h->G, (size_t)h->naux * ncell * h->esize));
        if (h->ndim >= 2 && h->esize == 4) {  // the fused last-axis sweep's rotating buffers (float)
            h->fused = 1;
            chk(dalloc(h, &h->W2, sb));
            chk(dalloc(h, &h->W3, sb));
            chk(dalloc(h, &h->T2, (size_t)ncell * h->esize));
            chk(dalloc(h, &h->T3, (size_t)ncell * h->esize));
            chk(dalloc(h, &h->Us2, sb));
            const dim3 fg = fused_grid(P, h->ndim);
            h->nblk_step = (int)(fg.x * fg.y * fg.z);
        }
    }
    for (int d = 0; d < h->ndim && st == JXF_OK; ++d) {
        long long nf = 1;
        for (int e = 0; e < 3; ++e) nf *= P.n[e] + (e == d ? 1 : 0);
        chk(dalloc(h, &h->F[d], (size_t)h->nv * nf * h->esize));
        if (eos->model == JXF_DIM) chk(dalloc(h, &h->UH[d], (size_t)nf * h->esize));
    }
    chk(dalloc(h, &h->scal, SC_N * sizeof(double)));
    chk(dalloc(h, &h->part,
               ((size_t)(h->nblk > h->nblk_step ? h->nblk : h->nblk_step) + kPartGroups) * (3 + MAXV) *
                   sizeof(double)));
    chk(dalloc(h, &h->status, sizeof(int)));
    chk(dalloc(h, &h->counters, 2 * sizeof(unsigned long long)));
    if (st == JXF_OK) {
        cudaError_t e = cudaMallocHost(&h->h_pin, 8 * sizeof(double));
        if (e != cudaSuccess) st = cuda_fail(h, e, "cudaMallocHost");
    }
    if (st == JXF_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) st = cuda_fail(h, e, "cudaStreamCreate");
    }
    if (st == JXF_OK) {
        cudaError_t e = cudaMemset(h->Un, 0, sb);
        if (e == cudaSuccess) e = cudaMemset(h->scal, 0, SC_N * sizeof(double));
        if (e == cudaSuccess) e = cudaMemset(h->status, 0, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(h->counters, 0, 2 * sizeof(unsigned long long));
        if (e == cudaSuccess && h->record) e = cudaMemset(h->record, 0, (3 + MAXV) * sizeof(double));
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = cuda_fail(h, e, "initialise buffers");
    }
    if (st != JXF_OK) {
        free_all(h);
        delete h;
        return st;
    }
    for (int d = 0; d < 3; ++d) {
        P.F[d] = h->F[d];
        P.UH[d] = h->UH[d];
    }
    P.scal = h->scal;
    P.part = h->part;
    P.status = h->status;
    P.counters = h->counters;
    P.dtp = h->scal + SC_DT;
    h->cur_state = h->Un;
    *out = h;
    return JXF_OK;
}

// The kernels of jxf_step_vjp between its copies (inputs in adj[A_U0] and
// adj[A_B3], output in adj[A_BN]).
jxf_status enqueue_step_vjp(jxf_ctx *h, double dt, cudaStream_t s) {
    const long long n = (long long)h->nv * h->ncell;
    void **a = h->adj;
    const Ops *o = h->ops;
    jxf_status st;
    if ((st = set_scalar(h, SC_RHS_DT, dt, s)) != JXF_OK) return st;
    // stage states (§3.4): U1 = Un + dt R(Un), U2 = 3/4 Un + 1/4 U1 + 1/4 dt R(U1)
    if ((st = rhs_device(h, a[A_U0], a[A_TMP], s)) != JXF_OK) return st;
    o->axpbypcz(a[A_U1], n, 1.0, a[A_U0], dt, a[A_TMP], 0.0, nullptr, s);
    if ((st = rhs_device(h, a[A_U1], a[A_TMP], s)) != JXF_OK) return st;
    o->axpbypcz(a[A_U2], n, 0.75, a[A_U0], 0.25, a[A_U1], 0.25 * dt, a[A_TMP], s);
    // reverse: U^{n+1} = 1/3 Un + 2/3 U2 + 2/3 dt R(U2)
    if ((st = rhs_vjp_device(h, a[A_U2], a[A_B3], a[A_TMP], s)) != JXF_OK) return st;
    o->axpbypcz(a[A_B2], n, 2.0 / 3.0, a[A_B3], 2.0 / 3.0 * dt, a[A_TMP], 0.0, nullptr, s);
    o->axpbypcz(a[A_BN], n, 1.0 / 3.0, a[A_B3], 0.75, a[A_B2], 0.0, nullptr, s);
    if ((st = rhs_vjp_device(h, a[A_U1], a[A_B2], a[A_TMP], s)) != JXF_OK) return st;
    o->axpbypcz(a[A_B1], n, 0.25, a[A_B2], 0.25 * dt, a[A_TMP], 0.0, nullptr, s);
    if ((st = rhs_vjp_device(h, a[A_U0], a[A_B1], a[A_TMP], s)) != JXF_OK) return st;
    o->axpbypcz(a[A_BN], n, 1.0, a[A_BN], 1.0, a[A_B1], dt, a[A_TMP], s);
    return launch_check(h, "step vjp");
}

}  // namespace

extern "C" {

jxf_status jxf_create(const jxf_grid *grid, const jxf_eos *eos, const jxf_scheme *scheme,
                      jxf_handle *out) {
    JXF_RANGE("jxf_create");
    return create_handle(grid, eos, scheme, nullptr, out);
}

jxf_status jxf_create_block(const jxf_grid *grid, const jxf_eos *eos, const jxf_scheme *scheme,
                            const jxf_block *block, jxf_handle *out) {
    JXF_RANGE("jxf_create_block");
    if (!block) {
        if (out) *out = nullptr;
        return JXF_ERR_ARG;
    }
    return create_handle(grid, eos, scheme, block, out);
}

jxf_status jxf_destroy(jxf_handle h) {
    JXF_RANGE("jxf_destroy");
    if (!h) return JXF_ERR_ARG;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    free_all(h);
    delete h;
    return JXF_OK;
}

int jxf_nvar(jxf_handle h) { return h ? h->nv : -1; }
long long jxf_ncell(jxf_handle h) { return h ? h->ncell : -1; }

jxf_status jxf_set_state(jxf_handle h, const void *U, jxf_stream stream) {
    JXF_RANGE("jxf_set_state");
    if (!h) return JXF_ERR_ARG;
    if (!U) return fail(h, JXF_ERR_ARG, "jxf_set_state: null state");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    jxf_status st = copy_rows(h, h->Un, U, true, h->nv, s);
    if (st != JXF_OK) return st;
    JXF_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(int), s));  // a new state starts clean
    return derive_state(h, s);
}

jxf_status jxf_set_primitive(jxf_handle h, const double *W, jxf_stream stream) {
    JXF_RANGE("jxf_set_primitive");
    if (!h) return JXF_ERR_ARG;
    if (!W) return fail(h, JXF_ERR_ARG, "jxf_set_primitive: null state");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    const size_t b64 = (size_t)h->nv * h->ncell * sizeof(double);
    if (!h->W64) {
        jxf_status st = dalloc(h, &h->W64, b64);
        if (st != JXF_OK) return st;
    }
    JXF_CUDA(h, cudaMemcpyAsync(h->W64, W, b64, cudaMemcpyDefault, s));
    JXF_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(int), s));  // a new state starts clean
    Dev P = h->base;
    P.Uout = h->Un;
    h->ops->from_prim(P, h->W64, s);
    jxf_status st = launch_check(h, "k_from_prim");
    if (st != JXF_OK) return st;
    return derive_state(h, s);
}

jxf_status jxf_get_state(jxf_handle h, void *U, jxf_stream stream) {
    JXF_RANGE("jxf_get_state");
    if (!h) return JXF_ERR_ARG;
    if (!U) return fail(h, JXF_ERR_ARG, "jxf_get_state: null buffer");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    jxf_status st = copy_rows(h, U, h->Un, false, h->nv, s);
    if (st != JXF_OK) return st;
    return check_status(h, s);
}

jxf_status jxf_get_primitive(jxf_handle h, void *W, jxf_stream stream) {
    JXF_RANGE("jxf_get_primitive");
    if (!h) return JXF_ERR_ARG;
    if (!W) return fail(h, JXF_ERR_ARG, "jxf_get_primitive: null buffer");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    jxf_status st = copy_rows(h, W, h->W, false, h->nv, s);
    if (st != JXF_OK) return st;
    return check_status(h, s);
}

jxf_status jxf_set_time(jxf_handle h, double t, jxf_stream stream) {
    JXF_RANGE("jxf_set_time");
    if (!h) return JXF_ERR_ARG;
    if (h->block) return block_unsupported(h, "jxf_set_time");
    if (!std::isfinite(t)) return fail(h, JXF_ERR_ARG, "jxf_set_time: non-finite time");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    jxf_status st = set_scalar(h, SC_T, t, s);
    if (st != JXF_OK) return st;
    return finalize(h, 2, s);
}

jxf_status jxf_rhs(jxf_handle h, const void *U, void *dU, double dt, jxf_stream stream) {
    JXF_RANGE("jxf_rhs");
    if (!h) return JXF_ERR_ARG;
    if (h->block) return block_unsupported(h, "jxf_rhs");
    if (!U || !dU) return fail(h, JXF_ERR_ARG, "jxf_rhs: null buffer");
    if (!std::isfinite(dt) || dt < 0.0) return fail(h, JXF_ERR_ARG, "jxf_rhs: dt must be finite and >= 0");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    jxf_status st = ensure_rhs_scratch(h);
    if (st != JXF_OK) return st;
    JXF_CUDA(h, cudaMemcpyAsync(h->rU, U, state_bytes(h), cudaMemcpyDefault, s));
    if ((st = set_scalar(h, SC_RHS_DT, dt, s)) != JXF_OK) return st;
    Dev P = h->base;
    P.Us = h->rU;
    P.Wout = h->rW;
    P.Tout = h->rT;
    P.G = h->rG;  // the primitives' epilogue writes psi here (THINC)
    h->ops->prim(P, 0, s);
    P.W = h->rW;
    P.Ucell = h->rU;
    P.Tt = h->rT;
    P.dtp = h->scal + SC_RHS_DT;
    P.skip_if_done = 0;
    if (h->G) h->ops->aux(P, s);
    for (int d = 0; d < h->ndim; ++d) h->ops->flux(P, d, s);
    P.dU = h->rD;
    h->ops->update(P, 0, 0, s);
    if ((st = launch_check(h, "rhs kernels")) != JXF_OK) return st;
    JXF_CUDA(h, cudaMemcpyAsync(dU, h->rD, state_bytes(h), cudaMemcpyDefault, s));
    return JXF_OK;
}

jxf_status jxf_rhs_vjp(jxf_handle h, const void *U, const void *R_bar, void *U_bar, double dt,
                       jxf_stream stream) {
    JXF_RANGE("jxf_rhs_vjp");
    if (!h) return JXF_ERR_ARG;
    if (!U || !R_bar || !U_bar) return fail(h, JXF_ERR_ARG, "jxf_rhs_vjp: null buffer");
    if (!std::isfinite(dt) || dt < 0.0) return fail(h, JXF_ERR_ARG, "jxf_rhs_vjp: dt must be finite and >= 0");
    jxf_status st = check_vjp_supported(h);
    if (st != JXF_OK) return st;
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    if ((st = ensure_adj_scratch(h)) != JXF_OK) return st;
    const size_t sb = state_bytes(h);
    JXF_CUDA(h, cudaMemcpyAsync(h->adj[A_U0], U, sb, cudaMemcpyDefault, s));
    JXF_CUDA(h, cudaMemcpyAsync(h->adj[A_RB], R_bar, sb, cudaMemcpyDefault, s));
    if ((st = rhs_vjp_device(h, h->adj[A_U0], h->adj[A_RB], h->adj[A_BN], s)) != JXF_OK) return st;
    JXF_CUDA(h, cudaMemcpyAsync(U_bar, h->adj[A_BN], sb, cudaMemcpyDefault, s));
    return JXF_OK;
}

jxf_status jxf_step_vjp(jxf_handle h, const void *U_n, double dt, const void *U_bar_np1, void *U_bar_n,
                        jxf_stream stream) {
    JXF_RANGE("jxf_step_vjp");
    if (!h) return JXF_ERR_ARG;
    if (!U_n || !U_bar_np1 || !U_bar_n) return fail(h, JXF_ERR_ARG, "jxf_step_vjp: null buffer");
    if (!std::isfinite(dt) || dt < 0.0) return fail(h, JXF_ERR_ARG, "jxf_step_vjp: dt must be finite and >= 0");
    jxf_status st = check_vjp_supported(h);
    if (st != JXF_OK) return st;
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    if ((st = ensure_adj_scratch(h)) != JXF_OK) return st;
    const size_t sb = state_bytes(h);
    void **a = h->adj;
    JXF_CUDA(h, cudaMemcpyAsync(a[A_U0], U_n, sb, cudaMemcpyDefault, s));
    JXF_CUDA(h, cudaMemcpyAsync(a[A_B3], U_bar_np1, sb, cudaMemcpyDefault, s));
    // the kernels between the copies run as one CUDA graph, captured once per
    // step size (a rollout's backward pass replays it for every step)
    if (!h->vjp_exec || h->vjp_dt != dt) {
        if (h->vjp_exec) {
            cudaGraphExecDestroy(h->vjp_exec);
            h->vjp_exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        JXF_CUDA(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        st = enqueue_step_vjp(h, dt, h->cap);
        cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
        if (st != JXF_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&h->vjp_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            h->vjp_exec = nullptr;
            return cuda_fail(h, e, "cudaGraphInstantiate");
        }
        h->vjp_dt = dt;
    }
    JXF_CUDA(h, cudaGraphLaunch(h->vjp_exec, s));
    JXF_CUDA(h, cudaMemcpyAsync(U_bar_n, a[A_BN], sb, cudaMemcpyDefault, s));
    return JXF_OK;
}

jxf_status jxf_step(jxf_handle h, int n, double *t_out, jxf_stream stream) {
    JXF_RANGE("jxf_step");
    if (!h) return JXF_ERR_ARG;
    if (h->block) return block_unsupported(h, "jxf_step");
    if (n < 0) return fail(h, JXF_ERR_ARG, "jxf_step: n < 0");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    if (n > 0 && !h->step_exec) {
        cudaGraph_t graph = nullptr;
        JXF_CUDA(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        jxf_status st = enqueue_step(h, h->cap);
        cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
        if (st != JXF_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&h->step_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            h->step_exec = nullptr;
            return cuda_fail(h, e, "cudaGraphInstantiate");
        }
    }
    for (int k = 0; k < n; ++k) JXF_CUDA(h, cudaGraphLaunch(h->step_exec, s));
    if (!t_out) return JXF_OK;
    jxf_status st = check_status(h, s);
    *t_out = h->h_pin[0];
    return st;
}

jxf_status jxf_step_profiled(jxf_handle h, int n, float *ms, int *launches, jxf_stream stream) {
    JXF_RANGE("jxf_step_profiled");
    if (!h) return JXF_ERR_ARG;
    if (h->block) return block_unsupported(h, "jxf_step_profiled");
    if (n < 0 || !ms || !launches) return fail(h, JXF_ERR_ARG, "jxf_step_profiled: bad arguments");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    // all n steps queued back to back (the device never idles between
    // kernels, as in a plain step), one synchronisation at the end
    KernelTimer kt(kTimedRegionsPerStep * (n > 0 ? n : 1));
    if (!kt.ok) return fail(h, JXF_ERR_CUDA, "jxf_step_profiled: cudaEventCreate failed");
    for (int step = 0; step < n; ++step) {
        jxf_status st = enqueue_step(h, s, &kt);
        if (st != JXF_OK) return st;
    }
    JXF_CUDA(h, cudaStreamSynchronize(s));
    for (int k = 0; k < kt.n; ++k) {
        float t = 0.f;
        JXF_CUDA(h, cudaEventElapsedTime(&t, kt.ev[2 * k], kt.ev[2 * k + 1]));
        ms[kt.kind[k]] += t;
        launches[kt.kind[k]] += kt.nk[k];
    }
    return check_status(h, s);
}

jxf_status jxf_stats(jxf_handle h, double *sums, double *dt_last, long long *limited) {
    JXF_RANGE("jxf_stats");
    if (!h) return JXF_ERR_ARG;
    DeviceGuard g(h->device);
    JXF_CUDA(h, cudaStreamSynchronize(h->last));
    double sc[SC_N];
    unsigned long long cnt[2];
    JXF_CUDA(h, cudaMemcpy(sc, h->scal, sizeof(sc), cudaMemcpyDeviceToHost));
    JXF_CUDA(h, cudaMemcpy(cnt, h->counters, sizeof(cnt), cudaMemcpyDeviceToHost));
    if (sums)
        for (int v = 0; v < h->nv; ++v) sums[v] = sc[SC_SUMS + v];
    if (dt_last) *dt_last = sc[SC_DT_LAST];
    if (limited) {
        limited[0] = (long long)cnt[0];
        limited[1] = (long long)cnt[1];
    }
    return JXF_OK;
}

void jxf_fail_allocation_after(int k) { g_fail_alloc_after.store(k < 0 ? -1 : k); }

jxf_status jxf_selftest_div(const double *a, const double *b, double *q, long long n) {
    if (!a || !b || !q || n < 0) return JXF_ERR_ARG;
    if (n == 0) return JXF_OK;
    k_selftest_div<<<(unsigned)((n + 255) / 256), 256>>>(a, b, q, n);
    if (cudaGetLastError() != cudaSuccess) return JXF_ERR_CUDA;
    return cudaDeviceSynchronize() == cudaSuccess ? JXF_OK : JXF_ERR_CUDA;
}

jxf_status jxf_peak_probe(int precision, double *tflops) {
    if (!tflops || (precision != JXF_FP64 && precision != JXF_MIXED32)) return JXF_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return JXF_ERR_CUDA;
    void *out = nullptr;
    if (cudaMalloc(&out, 16) != cudaSuccess) return JXF_ERR_OOM;
    const int blocks = sms * 8, threads = 256;
    const int iters = precision == JXF_FP64 ? 2048 : 65536;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0);
        if (precision == JXF_FP64)
            k_fma_probe<double><<<blocks, threads>>>(static_cast<double *>(out), iters, 0.999999, 1e-7);
        else
            k_fma_probe<float><<<blocks, threads>>>(static_cast<float *>(out), iters, 0.9999f, 1e-4f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // first launch is a warm-up
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return JXF_ERR_CUDA;
    *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
    return JXF_OK;
}

const char *jxf_last_error(jxf_handle h) {
    if (!h) return kNoHandle;
    return h->err.c_str();
}

jxf_status jxf_block_phase(jxf_handle h, int phase, int arg, jxf_stream stream) {
    JXF_RANGE("jxf_block_phase");
    if (!h) return JXF_ERR_ARG;
    if (!h->block) return fail(h, JXF_ERR_ARG, "jxf_block_phase: not a block handle");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    h->last = s;
    switch (phase) {
    case JXF_PHASE_STAGE:
        if (arg < 0 || arg > 2) return fail(h, JXF_ERR_ARG, "jxf_block_phase: stage must be 0, 1 or 2");
        return block_stage(h, arg, s);
    case JXF_PHASE_AUX: {
        if (!h->G) return JXF_OK;
        Dev P = h->base;
        const void *Wr[3] = {h->W, h->W2, h->W3};
        P.W = Wr[h->wcur];
        P.G = h->G;
        h->ops->aux(P, s);
        return launch_check(h, "k_aux");
    }
    case JXF_PHASE_REDUCE: {
        const double *part = h->part;
        int npart = h->npart_cur;
        if (npart > 4 * kPartGroups) {
            double *grp = h->part + (size_t)npart * (3 + MAXV);
            k_reduce_partials<<<kPartGroups, kPartThreads, 0, s>>>(h->part, npart, h->nv, grp);
            part = grp;
            npart = kPartGroups;
        }
        k_fold_records<<<1, kPartThreads, 0, s>>>(part, npart, h->nv, h->record);
        return launch_check(h, "k_fold_records");
    }
    case JXF_PHASE_FINISH:
        if (arg != 0 && arg != 1) return fail(h, JXF_ERR_ARG, "jxf_block_phase: finish mode must be 0 or 1");
        k_finalize<<<1, kFinalThreads, 0, s>>>(h->base, h->record, 1, h->nv, arg);
        return launch_check(h, "k_finalize");
    default:
        return fail(h, JXF_ERR_ARG, "jxf_block_phase: unknown phase");
    }
}

int jxf_block_halo_count(jxf_handle h, int kind) {
    if (!h || !h->block || (kind != JXF_HALO_STATE && kind != JXF_HALO_AUX)) return -1;
    const void *b[4];
    int r[4];
    return halo_regions(h, kind, b, r);
}

jxf_status jxf_block_halo(jxf_handle h, int kind, int index, int side, int recv, void **ptr, size_t *pitch,
                          size_t *width, int *height) {
    if (!h) return JXF_ERR_ARG;
    if (!h->block || !ptr || !pitch || !width || !height || (side != 0 && side != 1) ||
        (recv != 0 && recv != 1) || (kind != JXF_HALO_STATE && kind != JXF_HALO_AUX))
        return fail(h, JXF_ERR_ARG, "jxf_block_halo: bad arguments");
    const void *b[4];
    int r[4];
    const int n = halo_regions(h, kind, b, r);
    if (index < 0 || index >= n) return fail(h, JXF_ERR_ARG, "jxf_block_halo: no such region");
    *ptr = halo_ptr(h, b[index], side, recv);
    *pitch = (size_t)h->base.vstride * h->esize;
    *width = 3 * h->plane * h->esize;
    *height = r[index];
    return JXF_OK;
}

jxf_status jxf_block_exchange(jxf_handle lo, jxf_handle hi, int kind, jxf_stream stream) {
    JXF_RANGE("jxf_block_exchange");
    if (!lo || !hi) return JXF_ERR_ARG;
    if (!lo->block || !hi->block || !lo->nbr[1] || !hi->nbr[0] || lo->plane != hi->plane ||
        lo->esize != hi->esize || lo->nv != hi->nv || lo->naux != hi->naux ||
        (kind != JXF_HALO_STATE && kind != JXF_HALO_AUX))
        return fail(lo, JXF_ERR_ARG, "jxf_block_exchange: not two neighbouring blocks of one grid");
    const void *bl[4], *bh[4];
    int rl[4], rh[4];
    const int n = halo_regions(lo, kind, bl, rl);
    if (halo_regions(hi, kind, bh, rh) != n) return fail(lo, JXF_ERR_ARG, "jxf_block_exchange: schemes differ");
    DeviceGuard g(lo->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t w = 3 * lo->plane * lo->esize;
    const size_t pl = (size_t)lo->base.vstride * lo->esize, ph = (size_t)hi->base.vstride * hi->esize;
    for (int k = 0; k < n; ++k) {
        JXF_CUDA(lo, cudaMemcpy2DAsync(halo_ptr(hi, bh[k], 0, 1), ph, halo_ptr(lo, bl[k], 1, 0), pl, w,
                                       (size_t)rl[k], cudaMemcpyDefault, s));
        JXF_CUDA(lo, cudaMemcpy2DAsync(halo_ptr(lo, bl[k], 1, 1), pl, halo_ptr(hi, bh[k], 0, 0), ph, w,
                                       (size_t)rh[k], cudaMemcpyDefault, s));
    }
    lo->last = hi->last = s;
    return JXF_OK;
}

jxf_status jxf_block_record(jxf_handle h, double **record) {
    if (!h) return JXF_ERR_ARG;
    if (!h->block || !record) return fail(h, JXF_ERR_ARG, "jxf_block_record: bad arguments");
    *record = h->record;
    return JXF_OK;
}

jxf_status jxf_block_allreduce(const jxf_handle *blocks, int n, jxf_stream stream) {
    JXF_RANGE("jxf_block_allreduce");
    if (!blocks || n < 1) return JXF_ERR_ARG;
    jxf_ctx *h0 = blocks[0];
    for (int k = 0; k < n; ++k)
        if (!blocks[k] || !blocks[k]->block || blocks[k]->nv != (h0 ? h0->nv : -1))
            return h0 ? fail(h0, JXF_ERR_ARG, "jxf_block_allreduce: not blocks of one grid") : JXF_ERR_ARG;
    DeviceGuard g(h0->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t rb = (3 + MAXV) * sizeof(double);
    if (h0->gather_cap < n + 1) {
        if (h0->gather) {
            JXF_CUDA(h0, cudaStreamSynchronize(s));
            cudaFree(h0->gather);
            h0->gather = nullptr;
            h0->gather_cap = 0;
        }
        jxf_status st = dalloc(h0, &h0->gather, (size_t)(n + 1) * rb);
        if (st != JXF_OK) return st;
        h0->gather_cap = n + 1;
    }
    for (int k = 0; k < n; ++k)
        JXF_CUDA(h0, cudaMemcpyAsync(h0->gather + (size_t)k * (3 + MAXV), blocks[k]->record, rb,
                                     cudaMemcpyDefault, s));
    double *res = h0->gather + (size_t)n * (3 + MAXV);
    k_fold_records<<<1, kPartThreads, 0, s>>>(h0->gather, n, h0->nv, res);
    jxf_status st = launch_check(h0, "k_fold_records");
    if (st != JXF_OK) return st;
    for (int k = 0; k < n; ++k) {
        JXF_CUDA(h0, cudaMemcpyAsync(blocks[k]->record, res, rb, cudaMemcpyDefault, s));
        blocks[k]->last = s;
    }
    return JXF_OK;
}

}  // extern "C"
