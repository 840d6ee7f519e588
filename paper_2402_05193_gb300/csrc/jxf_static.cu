// jxf_static.cu -- jxf_rhs_static: the right-hand side R(U) without any
// device allocation.
//
// For callers that cannot call cudaMalloc/cudaFree: code that runs while
// another runtime has reserved (nearly) all device memory for its own pool,
// code that must not trigger the implicit device synchronisation of
// cudaFree, and loops that forbid allocation after start-up.  Instead of a
// handle with its own buffers, the primitives, temperature, face fluxes and
// counters of one evaluation live in one file-scope device array of
// JXF_STATIC_SCRATCH_BYTES.  Every process that loads this library keeps
// that array on every GPU it uses until it exits.
//
// The scratch is shared by all calls: each call overwrites it (the counters
// it accumulates into are cleared at the start of every call), and two calls
// whose kernels overlap on the same GPU -- issued on different streams or
// from different host threads -- race on it.  The address of the array on a
// device is looked up once per device, by the first call made with that
// device current; that first call should come before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "jxf.h"
#include "jxf_nvtx.cuh"
#include "jxf_ops.cuh"
#include "jxf_setup.cuh"

using namespace jxf;

namespace {

static __device__ __align__(256) unsigned char g_scratch[JXF_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {nullptr};

void put_msg(char *msg, size_t len, const char *fmt, long long a = 0, long long b = 0) {
    if (msg && len) std::snprintf(msg, len, fmt, a, b);
}

__global__ void k_static_reset(double *dt_slot, double dt, unsigned long long *counters) {
    *dt_slot = dt;
    counters[0] = 0ull;
    counters[1] = 0ull;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" jxf_status jxf_rhs_static(const jxf_grid *grid, const jxf_eos *eos,
                                     const jxf_scheme *scheme, const void *U, void *dU, double dt,
                                     jxf_stream stream, char *msg, size_t msg_len) {
    JXF_RANGE("jxf_rhs_static");
    if (msg && msg_len) msg[0] = '\0';
    if (!grid || !eos || !scheme || !U || !dU) {
        put_msg(msg, msg_len, "jxf_rhs_static: null argument");
        return JXF_ERR_ARG;
    }
    if (!std::isfinite(dt) || dt < 0.0) {
        put_msg(msg, msg_len, "jxf_rhs_static: dt must be finite and >= 0");
        return JXF_ERR_ARG;
    }
    // the same checks as jxf_create (grid extents and boundaries, model,
    // materials, scheme options, viscous order and material), without the
    // time-step requirement
    long long ncell = 0;
    {
        const jxf_status vs = validate_setup(grid, eos, scheme, &ncell, false);
        if (vs != JXF_OK) {
            put_msg(msg, msg_len,
                    vs == JXF_ERR_UNSUPPORTED
                        ? "jxf_rhs_static: unsupported combination of model and scheme options"
                        : "jxf_rhs_static: invalid grid, material or scheme (the checks of jxf_create)");
            return vs;
        }
    }
    const int ndim = grid->ndim;

    // scratch plan: [dt, 2 counters] | W | T | G (viscous gradient or THINC
    // normal) | F_d ... | UH_d ...
    const int nv = ndim + (eos->model == JXF_DIM ? 4 : 2);
    const size_t es = scheme->precision == JXF_FP64 ? 8 : 4;
    long long nface[3] = {0, 0, 0};
    const int naux = aux_arrays(ndim, eos, scheme);
    const size_t gbytes = naux ? align256((size_t)naux * ncell * es) : 0;
    size_t need = 256 + align256((size_t)nv * ncell * es) + align256((size_t)ncell * es) + gbytes;
    for (int d = 0; d < ndim; ++d) {
        nface[d] = 1;
        for (int e = 0; e < 3; ++e) nface[d] *= (e < ndim ? grid->n[e] : 1) + (e == d ? 1 : 0);
        need += align256((size_t)nv * nface[d] * es);
        if (eos->model == JXF_DIM) need += align256((size_t)nface[d] * es);
    }
    if (need > (size_t)JXF_STATIC_SCRATCH_BYTES) {
        put_msg(msg, msg_len,
                "jxf_rhs_static: this grid needs %lld scratch bytes but the static scratch holds %lld",
                (long long)need, (long long)JXF_STATIC_SCRATCH_BYTES);
        return JXF_ERR_ARG;
    }

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        put_msg(msg, msg_len, "jxf_rhs_static: no usable current device");
        return JXF_ERR_CUDA;
    }
    cudaPointerAttributes a{};
    for (const void *p : {U, (const void *)dU}) {
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
            (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != dev) {
            cudaGetLastError();
            put_msg(msg, msg_len, "jxf_rhs_static: U and dU must be device memory of the current device");
            return JXF_ERR_ARG;
        }
    }
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess || !ptr) {
                put_msg(msg, msg_len, "jxf_rhs_static: cudaGetSymbolAddress failed");
                return JXF_ERR_CUDA;
            }
            g_addr[dev] = static_cast<unsigned char *>(ptr);
        }
        base = g_addr[dev];
    }

    // kernel parameters (same kernels as jxf_rhs)
    Dev P;
    fill_dev(grid, eos, scheme, ncell, P);

    double *dt_slot = reinterpret_cast<double *>(base);
    unsigned long long *counters = reinterpret_cast<unsigned long long *>(base + 64);
    size_t off = 256;
    void *W = base + off;
    off += align256((size_t)nv * ncell * es);
    void *Tt = base + off;
    off += align256((size_t)ncell * es);
    void *G = naux ? base + off : nullptr;
    off += gbytes;
    for (int d = 0; d < ndim; ++d) {
        P.F[d] = base + off;
        off += align256((size_t)nv * nface[d] * es);
        if (eos->model == JXF_DIM) {
            P.UH[d] = base + off;
            off += align256((size_t)nface[d] * es);
        }
    }
    P.counters = counters;
    P.dtp = dt_slot;
    P.skip_if_done = 0;

    const Ops *ops = scheme->precision == JXF_FP64
                         ? (eos->model == JXF_SPM ? ops_f64_spm(ndim) : ops_f64_dim(ndim))
                         : (eos->model == JXF_SPM ? ops_f32_spm(ndim) : ops_f32_dim(ndim));
    cudaStream_t s = (cudaStream_t)stream;
    k_static_reset<<<1, 1, 0, s>>>(dt_slot, dt, counters);
    P.Us = U;
    P.Wout = W;
    P.Tout = Tt;
    P.G = G;  // the primitives' epilogue writes psi here (THINC)
    ops->prim(P, 0, s);
    P.W = W;
    P.Ucell = U;
    P.Tt = Tt;
    if (G) ops->aux(P, s);
    for (int d = 0; d < ndim; ++d) ops->flux(P, d, s);
    P.dU = dU;
    ops->update(P, 0, 0, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        put_msg(msg, msg_len, "jxf_rhs_static: kernel launch failed");
        return JXF_ERR_CUDA;
    }
    return JXF_OK;
}
