// jxf_batch.cu -- the batched form of the C interface: many independent
// simulations of uneven grid sizes (one material model and scheme) advanced
// together by persistent tile-queue kernels, n steps captured as one CUDA
// graph and replayed with one launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "jxf.h"
#include "jxf_nvtx.cuh"
#include "jxf_ops.cuh"
#include "jxf_setup.cuh"

using namespace jxf;

namespace {

__global__ void __launch_bounds__(kFinalThreads)
    k_finalize_batch(const Dev *__restrict__ devs, const double *part, const int *slot0,
                     const int *nslot, int nv, unsigned *tickets, int nticket) {
    const int sim = blockIdx.x;
    if (blockIdx.x == 0)
        for (int k = threadIdx.x; k < nticket; k += blockDim.x) tickets[k] = 0u;
    finalize_block(devs[sim], part + (size_t)slot0[sim] * (3 + MAXV), nslot[sim], nv, 1);
}

__global__ void __launch_bounds__(kFinalThreads) k_finalize_one(const Dev P, int npart, int nv) {
    finalize_block(P, P.part, npart, nv, 0);
}

}  // namespace

struct jxf_batch_ctx {
    int device = 0, nsim = 0, ndim = 0, nv = 0, sms = 0;
    size_t esize = 8;
    jxf_eos eos{};
    jxf_scheme scheme{};
    const Ops *ops = nullptr;
    std::vector<jxf_grid> grids;
    std::vector<long long> ncell, cell_off, nface[3], face_off[3];
    std::vector<int> slot0, nslot;
    int total_slots = 0;
    std::vector<Dev> hdev;  // [stage][sim]
    // device memory
    void *Un = nullptr, *Us = nullptr, *W = nullptr, *Tt = nullptr, *G = nullptr;
    int naux = 0;  // per-cell auxiliary arrays in G (viscous gradient or THINC normal)
    int vh = 0;    // viscous stencil half-width of the face sweeps (0: inviscid)
    void *F[3] = {nullptr, nullptr, nullptr}, *UH[3] = {nullptr, nullptr, nullptr};
    double *scal = nullptr, *part = nullptr, *W64 = nullptr;
    int *status = nullptr, *d_slot0 = nullptr, *d_nslot = nullptr;
    unsigned long long *counters = nullptr;
    unsigned *tickets = nullptr;
    int nticket = 0;
    Dev *devs = nullptr;
    Tile *ftiles[3] = {nullptr, nullptr, nullptr}, *ctiles = nullptr;
    int nft[3] = {0, 0, 0}, nct = 0;
    // tiling (autotuner knobs)
    int tile_faces = 1024, blocks_per_sm = 8;
    // graph of n steps
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    int exec_n = 0;
    cudaStream_t last = nullptr;
    std::string err;
};

namespace {

jxf_status bfail(jxf_batch_ctx *b, jxf_status s, const std::string &m) {
    if (b) b->err = m;
    return s;
}

jxf_status bcuda(jxf_batch_ctx *b, cudaError_t e, const char *what) {
    if (b) b->err = std::string("jxf_batch: ") + what + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? JXF_ERR_OOM : JXF_ERR_CUDA;
}

#define BCUDA(b, call)                                     \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return bcuda(b, e_, #call); \
    } while (0)

template <class P> jxf_status balloc(jxf_batch_ctx *b, P **p, size_t bytes) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) return bcuda(b, e, "cudaMalloc");
    *p = static_cast<P *>(q);
    return JXF_OK;
}

void bfree(jxf_batch_ctx *b) {
    void *bufs[] = {b->Un, b->Us, b->W, b->Tt, b->G, b->F[0], b->F[1], b->F[2], b->UH[0], b->UH[1], b->UH[2],
                    b->scal, b->part, b->W64, b->status, b->d_slot0, b->d_nslot, b->counters,
                    b->tickets, b->devs, b->ftiles[0], b->ftiles[1], b->ftiles[2], b->ctiles};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap) cudaStreamDestroy(b->cap);
}

char *at(void *base, long long elems, size_t es) { return static_cast<char *>(base) + elems * (long long)es; }

// Face tiles of the given length per axis, cell tiles of one block.
jxf_status build_tiles(jxf_batch_ctx *b) {
    for (int d = 0; d < b->ndim; ++d) {
        std::vector<Tile> t;
        for (int s = 0; s < b->nsim; ++s)
            for (long long st = 0; st < b->nface[d][s]; st += b->tile_faces)
                t.push_back(Tile{s, 0, st, std::min<long long>(b->tile_faces, b->nface[d][s] - st)});
        if (b->ftiles[d]) cudaFree(b->ftiles[d]);
        b->ftiles[d] = nullptr;
        jxf_status st = balloc(b, &b->ftiles[d], t.size() * sizeof(Tile));
        if (st != JXF_OK) return st;
        BCUDA(b, cudaMemcpy(b->ftiles[d], t.data(), t.size() * sizeof(Tile), cudaMemcpyHostToDevice));
        b->nft[d] = (int)t.size();
    }
    if (!b->ctiles) {
        std::vector<Tile> t;
        for (int s = 0; s < b->nsim; ++s)
            for (int j = 0; j < b->nslot[s]; ++j) {
                const long long st = (long long)j * kCellThreads;
                t.push_back(Tile{s, b->slot0[s] + j, st, std::min<long long>(kCellThreads, b->ncell[s] - st)});
            }
        jxf_status st = balloc(b, &b->ctiles, t.size() * sizeof(Tile));
        if (st != JXF_OK) return st;
        BCUDA(b, cudaMemcpy(b->ctiles, t.data(), t.size() * sizeof(Tile), cudaMemcpyHostToDevice));
        b->nct = (int)t.size();
    }
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
        b->exec_n = 0;
    }
    return JXF_OK;
}

// One step of every simulation: 3 stages x (ndim face sweeps + cell update)
// + per-simulation finalisation (which also re-arms the tile queues).
jxf_status enqueue_batch_step(jxf_batch_ctx *b, cudaStream_t s) {
    const int gf = b->blocks_per_sm > 0 ? std::min(b->blocks_per_sm * b->sms, 1 << 20) : 0;
    const int gc = std::min(b->nct, 8 * b->sms);
    int tk = 0;
    for (int stage = 0; stage < 3; ++stage) {
        const Dev *dv = b->devs + (size_t)stage * b->nsim;
        for (int d = 0; d < b->ndim; ++d)
            b->ops->flux_batch(dv, b->ftiles[d], b->nft[d], b->tickets + tk++, d, b->vh,
                               b->scheme.recon >= JXF_TENO6A_COMP ? 1 : 0,
                               gf > 0 ? std::min(gf, b->nft[d]) : b->nft[d], s);
        b->ops->update_batch(dv, b->ctiles, b->nct, b->tickets + tk++, b->part, stage == 2 ? 1 : 0, gc, s);
        if (b->G) b->ops->aux_batch(dv, b->ctiles, b->nct, b->tickets + tk++, gc, s);
    }
    k_finalize_batch<<<b->nsim, kFinalThreads, 0, s>>>(b->devs + 2 * (size_t)b->nsim, b->part, b->d_slot0,
                                                        b->d_nslot, b->nv, b->tickets, b->nticket);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bcuda(b, e, "batched step kernels");
    return JXF_OK;
}

jxf_status check_sim(jxf_batch_ctx *b, int sim) {
    if (sim < 0 || sim >= b->nsim) return bfail(b, JXF_ERR_ARG, "jxf_batch: simulation index out of range");
    return JXF_OK;
}

// Primitives, diagnostics and dt of simulation sim's state (single-grid kernels
// on that simulation's parameter block).
jxf_status derive_sim(jxf_batch_ctx *b, int sim, cudaStream_t s) {
    Dev P = b->hdev[sim];
    P.skip_if_done = 0;
    P.Us = P.Un;
    P.Wout = const_cast<void *>(P.W);
    P.Tout = const_cast<void *>(P.Tt);
    P.part = b->part + (size_t)b->slot0[sim] * (3 + MAXV);
    b->ops->prim(P, 1, s);
    if (b->G) b->ops->aux(P, s);
    k_finalize_one<<<1, kFinalThreads, 0, s>>>(P, b->nslot[sim], b->nv);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bcuda(b, e, "derive state");
    return JXF_OK;
}

}  // namespace

extern "C" {

jxf_status jxf_batch_create(int nsim, const jxf_grid *grids, const jxf_eos *eos, const jxf_scheme *scheme,
                            jxf_batch *out) {
    JXF_RANGE("jxf_batch_create");
    if (!out) return JXF_ERR_ARG;
    *out = nullptr;
    if (nsim < 1 || !grids || !eos || !scheme) return JXF_ERR_ARG;
    std::vector<long long> nc(nsim);
    for (int k = 0; k < nsim; ++k) {
        const jxf_status st = validate_setup(&grids[k], eos, scheme, &nc[k]);
        if (st != JXF_OK) return st;
        if (grids[k].ndim != grids[0].ndim) return JXF_ERR_ARG;
    }
    jxf_batch_ctx *b = new (std::nothrow) jxf_batch_ctx();
    if (!b) return JXF_ERR_OOM;
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
        delete b;
        return JXF_ERR_CUDA;
    }
    b->nsim = nsim;
    b->ndim = grids[0].ndim;
    b->nv = b->ndim + (eos->model == JXF_DIM ? 4 : 2);
    b->esize = scheme->precision == JXF_FP64 ? 8 : 4;
    b->eos = *eos;
    b->scheme = *scheme;
    b->grids.assign(grids, grids + nsim);
    b->ops = scheme->precision == JXF_FP64
                 ? (eos->model == JXF_SPM ? ops_f64_spm(b->ndim) : ops_f64_dim(b->ndim))
                 : (eos->model == JXF_SPM ? ops_f32_spm(b->ndim) : ops_f32_dim(b->ndim));
    // layout: per simulation, nv * ncell values per state array, nv * nface_d
    // per face-flux array, consecutive in the arenas
    long long cells = 0, faces[3] = {0, 0, 0};
    b->ncell = nc;
    for (int k = 0; k < nsim; ++k) {
        b->cell_off.push_back(cells);
        cells += nc[k];
        b->slot0.push_back(b->total_slots);
        b->nslot.push_back((int)((nc[k] + kCellThreads - 1) / kCellThreads));
        b->total_slots += b->nslot.back();
        for (int d = 0; d < 3; ++d) {
            long long nf = 0;
            if (d < b->ndim) {
                nf = 1;
                for (int e = 0; e < 3; ++e) nf *= (e < b->ndim ? grids[k].n[e] : 1) + (e == d ? 1 : 0);
            }
            b->face_off[d].push_back(faces[d]);
            b->nface[d].push_back(nf);
            faces[d] += nf;
        }
    }
    const size_t es = b->esize, nv = (size_t)b->nv;
    jxf_status st = JXF_OK;
    auto chk = [&](jxf_status x) { if (st == JXF_OK) st = x; };
    chk(balloc(b, &b->Un, nv * cells * es));
    chk(balloc(b, &b->Us, nv * cells * es));
    chk(balloc(b, &b->W, nv * cells * es));
    chk(balloc(b, &b->Tt, cells * es));
    b->naux = aux_arrays(b->ndim, eos, scheme);
    b->vh = scheme->viscous && eos->model == JXF_SPM
                ? (scheme->visc_order == 2 ? 1 : (scheme->visc_order == 6 ? 3 : 2))
                : 0;
    if (b->naux) chk(balloc(b, &b->G, (size_t)b->naux * cells * es));
    for (int d = 0; d < b->ndim; ++d) {
        chk(balloc(b, &b->F[d], nv * faces[d] * es));
        if (eos->model == JXF_DIM) chk(balloc(b, &b->UH[d], faces[d] * es));
    }
    long long maxc = *std::max_element(nc.begin(), nc.end());
    chk(balloc(b, &b->W64, nv * maxc * sizeof(double)));
    chk(balloc(b, &b->scal, (size_t)nsim * SC_N * sizeof(double)));
    chk(balloc(b, &b->part, (size_t)b->total_slots * (3 + MAXV) * sizeof(double)));
    chk(balloc(b, &b->status, nsim * sizeof(int)));
    chk(balloc(b, &b->d_slot0, nsim * sizeof(int)));
    chk(balloc(b, &b->d_nslot, nsim * sizeof(int)));
    chk(balloc(b, &b->counters, 2 * sizeof(unsigned long long)));
    b->nticket = 3 * (b->ndim + 2);
    chk(balloc(b, &b->tickets, b->nticket * sizeof(unsigned)));
    chk(balloc(b, &b->devs, 3 * (size_t)nsim * sizeof(Dev)));
    if (st == JXF_OK) {
        cudaError_t e = cudaMemset(b->Un, 0, nv * cells * es);
        if (e == cudaSuccess) e = cudaMemset(b->scal, 0, (size_t)nsim * SC_N * sizeof(double));
        if (e == cudaSuccess) e = cudaMemset(b->status, 0, nsim * sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(b->counters, 0, 2 * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMemset(b->tickets, 0, b->nticket * sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemcpy(b->d_slot0, b->slot0.data(), nsim * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_nslot, b->nslot.data(), nsim * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) st = bcuda(b, e, "initialise");
    }
    if (st == JXF_OK) {
        // parameter blocks: one per stage per simulation (stage buffer roles)
        static const double coef[3][3] = {{0.0, 1.0, 1.0}, {0.75, 0.25, 0.25}, {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0}};
        b->hdev.resize(3 * (size_t)nsim);
        for (int k = 0; k < nsim; ++k) {
            Dev P;
            fill_dev(&grids[k], eos, scheme, nc[k], P);
            const long long co = b->cell_off[k];
            void *Un = at(b->Un, co * b->nv, es), *Us = at(b->Us, co * b->nv, es);
            P.W = at(b->W, co * b->nv, es);
            P.Tt = at(b->Tt, co, es);
            if (b->G) P.G = at(b->G, co * b->naux, es);
            for (int d = 0; d < b->ndim; ++d) {
                P.F[d] = at(b->F[d], b->face_off[d][k] * b->nv, es);
                if (b->UH[d]) P.UH[d] = at(b->UH[d], b->face_off[d][k], es);
            }
            P.scal = b->scal + (size_t)k * SC_N;
            P.dtp = P.scal + SC_DT;
            P.status = b->status + k;
            P.counters = b->counters;
            P.part = b->part + (size_t)b->slot0[k] * (3 + MAXV);
            P.skip_if_done = 1;
            for (int s = 0; s < 3; ++s) {
                Dev Q = P;
                Q.Un = Un;
                Q.Us = s == 0 ? Un : Us;
                Q.Ucell = Q.Us;
                Q.Uout = s == 2 ? Un : Us;
                Q.Wout = const_cast<void *>(P.W);
                Q.Tout = const_cast<void *>(P.Tt);
                Q.ca = coef[s][0];
                Q.cb = coef[s][1];
                Q.cc = coef[s][2];
                Q.ca32 = (float)Q.ca;
                Q.cb32 = (float)Q.cb;
                Q.stage0 = s == 0 ? 1 : 0;
                b->hdev[(size_t)s * nsim + k] = Q;
            }
        }
        cudaError_t e = cudaMemcpy(b->devs, b->hdev.data(), b->hdev.size() * sizeof(Dev), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = bcuda(b, e, "upload parameter blocks");
    }
    if (st == JXF_OK) st = build_tiles(b);
    if (st != JXF_OK) {
        bfree(b);
        delete b;
        return st;
    }
    *out = b;
    return JXF_OK;
}

jxf_status jxf_batch_destroy(jxf_batch b) {
    JXF_RANGE("jxf_batch_destroy");
    if (!b) return JXF_ERR_ARG;
    cudaDeviceSynchronize();
    bfree(b);
    delete b;
    return JXF_OK;
}

int jxf_batch_nsim(jxf_batch b) { return b ? b->nsim : -1; }

jxf_status jxf_batch_set_primitive(jxf_batch b, int sim, const double *W, jxf_stream stream) {
    JXF_RANGE("jxf_batch_set_primitive");
    if (!b) return JXF_ERR_ARG;
    jxf_status st = check_sim(b, sim);
    if (st != JXF_OK) return st;
    if (!W) return bfail(b, JXF_ERR_ARG, "jxf_batch_set_primitive: null state");
    cudaStream_t s = (cudaStream_t)stream;
    b->last = s;
    BCUDA(b, cudaMemcpyAsync(b->W64, W, (size_t)b->nv * b->ncell[sim] * sizeof(double), cudaMemcpyDefault, s));
    Dev P = b->hdev[sim];
    P.Uout = const_cast<void *>(P.Un);
    b->ops->from_prim(P, b->W64, s);
    return derive_sim(b, sim, s);
}

jxf_status jxf_batch_set_state(jxf_batch b, int sim, const void *U, jxf_stream stream) {
    JXF_RANGE("jxf_batch_set_state");
    if (!b) return JXF_ERR_ARG;
    jxf_status st = check_sim(b, sim);
    if (st != JXF_OK) return st;
    if (!U) return bfail(b, JXF_ERR_ARG, "jxf_batch_set_state: null state");
    cudaStream_t s = (cudaStream_t)stream;
    b->last = s;
    BCUDA(b, cudaMemcpyAsync(const_cast<void *>(b->hdev[sim].Un), U, (size_t)b->nv * b->ncell[sim] * b->esize,
                             cudaMemcpyDefault, s));
    return derive_sim(b, sim, s);
}

jxf_status jxf_batch_set_time(jxf_batch b, int sim, double t, jxf_stream stream) {
    if (!b) return JXF_ERR_ARG;
    jxf_status st = check_sim(b, sim);
    if (st != JXF_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    b->last = s;
    BCUDA(b, cudaMemcpyAsync(b->scal + (size_t)sim * SC_N + SC_T, &t, sizeof(double), cudaMemcpyHostToDevice, s));
    BCUDA(b, cudaStreamSynchronize(s));
    return derive_sim(b, sim, s);
}

jxf_status jxf_batch_get_state(jxf_batch b, int sim, void *U, jxf_stream stream) {
    JXF_RANGE("jxf_batch_get_state");
    if (!b) return JXF_ERR_ARG;
    jxf_status st = check_sim(b, sim);
    if (st != JXF_OK) return st;
    if (!U) return bfail(b, JXF_ERR_ARG, "jxf_batch_get_state: null buffer");
    cudaStream_t s = (cudaStream_t)stream;
    b->last = s;
    BCUDA(b, cudaMemcpyAsync(U, b->hdev[sim].Un, (size_t)b->nv * b->ncell[sim] * b->esize, cudaMemcpyDefault, s));
    BCUDA(b, cudaStreamSynchronize(s));
    return JXF_OK;
}

jxf_status jxf_batch_set_tiling(jxf_batch b, int tile_faces, int blocks_per_sm) {
    if (!b) return JXF_ERR_ARG;
    if (tile_faces < kFluxThreads || tile_faces % kFluxThreads != 0 || blocks_per_sm < 0 || blocks_per_sm > 64)
        return bfail(b, JXF_ERR_ARG, "jxf_batch_set_tiling: tile_faces must be a positive multiple of 128, "
                                     "blocks_per_sm in [0, 64]");
    BCUDA(b, cudaDeviceSynchronize());
    b->tile_faces = tile_faces;
    b->blocks_per_sm = blocks_per_sm;
    return build_tiles(b);
}

jxf_status jxf_batch_step(jxf_batch b, int n, jxf_stream stream) {
    JXF_RANGE("jxf_batch_step");
    if (!b) return JXF_ERR_ARG;
    if (n < 0) return bfail(b, JXF_ERR_ARG, "jxf_batch_step: n < 0");
    if (n == 0) return JXF_OK;
    cudaStream_t s = (cudaStream_t)stream;
    b->last = s;
    if (!b->exec || b->exec_n != n) {
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        BCUDA(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        jxf_status st = JXF_OK;
        for (int k = 0; k < n && st == JXF_OK; ++k) st = enqueue_batch_step(b, b->cap);
        cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
        if (st != JXF_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return bcuda(b, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return bcuda(b, e, "cudaGraphInstantiate");
        }
        b->exec_n = n;
    }
    BCUDA(b, cudaGraphLaunch(b->exec, s));
    return JXF_OK;
}

jxf_status jxf_batch_stats(jxf_batch b, int sim, double *t, double *sums, double *dt_last, long long *limited) {
    JXF_RANGE("jxf_batch_stats");
    if (!b) return JXF_ERR_ARG;
    jxf_status st = check_sim(b, sim);
    if (st != JXF_OK) return st;
    BCUDA(b, cudaStreamSynchronize(b->last));
    double sc[SC_N];
    int status = 0;
    unsigned long long cnt[2];
    BCUDA(b, cudaMemcpy(sc, b->scal + (size_t)sim * SC_N, sizeof(sc), cudaMemcpyDeviceToHost));
    BCUDA(b, cudaMemcpy(&status, b->status + sim, sizeof(int), cudaMemcpyDeviceToHost));
    BCUDA(b, cudaMemcpy(cnt, b->counters, sizeof(cnt), cudaMemcpyDeviceToHost));
    if (t) *t = sc[SC_T];
    if (sums)
        for (int v = 0; v < b->nv; ++v) sums[v] = sc[SC_SUMS + v];
    if (dt_last) *dt_last = sc[SC_DT_LAST];
    if (limited) {
        limited[0] = (long long)cnt[0];
        limited[1] = (long long)cnt[1];
    }
    if (status & ST_NONPHYSICAL) return bfail(b, JXF_ERR_NONPHYSICAL, "jxf_batch: non-admissible state");
    if (status & ST_BAD_DT) return bfail(b, JXF_ERR_NONPHYSICAL, "jxf_batch: non-finite or negative dt");
    if (status & ST_BOUNDS) return bfail(b, JXF_ERR_BOUNDS, "jxf_batch: a stencil or face index left its array (checked build)");
    return JXF_OK;
}

const char *jxf_batch_last_error(jxf_batch b) { return b ? b->err.c_str() : "jxf_batch: null handle"; }

}  // extern "C"
