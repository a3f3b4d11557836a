// extern "C" entry points of libllb: argument checking, device memory,
// host <-> device transfers and dispatch to the kernels.  Every step of the
// lattice Boltzmann update runs in the CUDA kernels of this library; the
// host code only validates, allocates, copies and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

namespace llb {

size_t elem_size(int dtype) {
    return dtype == LLB_F64 ? 8 : dtype == LLB_F32 ? 4 : (dtype == LLB_F16S || dtype == LLB_BF16S) ? 2 : 0;
}

int canonical_fields(const llb_ctx& c) { return c.ncomp == 2 ? 11 : 10; }

int fields_of(const llb_ctx& c) {
    if (c.scheme == LLB_SCHEME_MOMENT) return canonical_fields(c);
    return c.Q * c.ncomp;
}

}  // namespace llb

using namespace llb;

namespace {

// The moment-only state carries periodic ghosts (TMA tile boxes); its rows
// are 32-aligned for the one-component FP32 state (fields interleaved per 32
// nodes, FieldMap).  The population schemes keep dense populations and dense
// moment temporaries.
Layout layout_of(const llb_ctx& c) {
    const bool moment = c.scheme == LLB_SCHEME_MOMENT;
    const int align = (moment && c.ncomp == 1 && c.storage == LLB_F32) ? 32 : 8;
    return make_layout(c.nx, c.ny, c.nz, moment, c.ncomp == 2 ? 2 : 1, align);
}

// Bytes of one state copy.  A population state also holds the shifted
// moments of init and read-back (10 or 11 fields of stride lay.fs).
size_t state_bytes_of(const llb_ctx& c) {
    const size_t mom = (size_t)(c.ncomp == 2 ? 11 : 10) * c.lay.fs;
    if (c.scheme == LLB_SCHEME_MOMENT) return (size_t)c.nf * c.lay.fs * c.elem;
    return std::max((size_t)c.nf * c.N, mom) * c.elem;
}

int fail(llb_ctx* c, int code, const std::string& m) {
    if (c) {
        c->msg = m;
        if (code == LLB_ECUDA) c->sticky = LLB_ECUDA;
    }
    return code;
}

int cuda_fail(llb_ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, LLB_ECUDA, m);
}

#define LLB_CHECK_CTX(c)                         \
    do {                                         \
        if (!(c)) return LLB_EINVAL;             \
        if ((c)->sticky != LLB_OK) return LLB_ESTATE; \
    } while (0)

#define LLB_CUDA(c, expr, where)                              \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) return cuda_fail((c), e_, where); \
    } while (0)

bool dtype_ok(int dt) { return dt == LLB_F64 || dt == LLB_F32; }

// Validate shape and parameters; fill the shape-only fields of *c.
int validate(int nx, int ny, int nz, int lattice, double tau, const llb_params& p, llb_ctx* c, std::string* why) {
    if (nx < 1 || ny < 1 || nz < 1) { *why = "nx, ny, nz must be >= 1"; return LLB_EINVAL; }
    if (lattice != 19 && lattice != 27) { *why = "lattice must be 19 or 27"; return LLB_EINVAL; }
    if (!(tau > 0.5) || !std::isfinite(tau)) { *why = "tau must be finite and > 1/2 (nu = cs^2 (tau - 1/2) > 0)"; return LLB_EINVAL; }
    if (p.ncomp != 1 && p.ncomp != 2) { *why = "ncomp must be 1 or 2"; return LLB_EINVAL; }
    const bool narrow = p.storage == LLB_F16S || p.storage == LLB_BF16S;
    if (!dtype_ok(p.storage) && !narrow) { *why = "storage must be LLB_F32, LLB_F64, LLB_F16S or LLB_BF16S"; return LLB_EINVAL; }
    if (narrow && (p.ncomp != 1 || p.scheme != LLB_SCHEME_MOMENT)) {
        *why = "16-bit storage is for the one-component moment-only state"; return LLB_EINVAL;
    }
    if (p.scheme != LLB_SCHEME_MOMENT && p.scheme != LLB_SCHEME_POPULATION && p.scheme != LLB_SCHEME_POPULATION_BGK) {
        *why = "unknown scheme"; return LLB_EINVAL;
    }
    if (p.kernel != LLB_KERNEL_AUTO && p.kernel != LLB_KERNEL_DIRECT && p.kernel != LLB_KERNEL_TILED &&
        p.kernel != LLB_KERNEL_TMA) {
        *why = "unknown kernel"; return LLB_EINVAL;
    }
    if (p.variant < 0 || p.variant >= kTiledVariants32) { *why = "variant out of range"; return LLB_EINVAL; }
    if (p.ncomp == 2 && p.variant >= kCGVariants) { *why = "two-component variant out of range"; return LLB_EINVAL; }
    if (p.wait_budget_ms < 1 || p.wait_budget_ms > 600000) { *why = "wait_budget_ms must be in 1..600000"; return LLB_EINVAL; }
    if (p.debug_flags & ~3) { *why = "unknown debug flag"; return LLB_EINVAL; }
    if (!(p.grad_eps >= 0.0) || !std::isfinite(p.grad_eps)) { *why = "grad_eps must be finite and >= 0"; return LLB_EINVAL; }
    if (p.ncomp == 2) {
        if (nx < 4 || ny < 4 || nz < 4) { *why = "two components need nx, ny, nz >= 4"; return LLB_EINVAL; }
        if (p.scheme == LLB_SCHEME_MOMENT && (p.kernel == LLB_KERNEL_DIRECT || p.kernel == LLB_KERNEL_TMA)) {
            *why = "two components run the tiled kernel"; return LLB_EINVAL;
        }
        if (!(p.beta >= 0.0) || !std::isfinite(p.A_s) || !std::isfinite(p.A_h) || !(p.g_min > 0.0) || p.h_c < 0 ||
            p.h_c > 8) {
            *why = "bad two-component parameters"; return LLB_EINVAL;
        }
    }
    const double n = (double)nx * ny * nz;
    if (n > 4.0e9) { *why = "domain too large"; return LLB_EINVAL; }
    c->nx = nx; c->ny = ny; c->nz = nz;
    c->Q = lattice;
    c->tau = tau;
    c->omega = 1.0 / tau;
    c->ncomp = p.ncomp;
    c->storage = p.storage;
    c->scheme = p.scheme;
    c->kernel = p.kernel;
    c->variant = p.variant;
    c->params = p;
    c->N = (size_t)nx * ny * nz;
    c->nf = fields_of(*c);
    c->elem = elem_size(p.storage);
    c->lay = layout_of(*c);
    c->state_bytes = state_bytes_of(*c);
    return LLB_OK;
}

int ensure_staging(llb_ctx* c, size_t bytes) {
    if (c->staging_bytes >= bytes) return LLB_OK;
    if (c->staging) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->staging);
        c->staging = nullptr;
        c->staging_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&c->staging, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, LLB_ENOMEM, "cudaMalloc of the staging buffer failed");
    }
    c->staging_bytes = bytes;
    return LLB_OK;
}

// Shifted moments of the current state: the state itself (moment scheme), or
// the projection of the pulled populations into the spare flip-flop copy.
int current_moments(llb_ctx* c, const void** mom) {
    if (c->scheme == LLB_SCHEME_MOMENT) {
        *mom = c->buf[c->cur];
        return LLB_OK;
    }
    void* tmp = c->buf[1 - c->cur];
    LLB_CUDA(c, launch_moments_from_population(*c, c->buf[c->cur], tmp), "project populations");
    *mom = tmp;
    return LLB_OK;
}

// After shifted moments were written to `mom`, build the state from them.
int finish_init(llb_ctx* c, void* mom) {
    if (c->scheme != LLB_SCHEME_MOMENT)
        LLB_CUDA(c, launch_population_from_moments(*c, mom, c->buf[c->cur]), "reconstruct populations");
    c->t = 0;
    return LLB_OK;
}

// Where the init kernels write shifted moments before finish_init.
void* init_target(llb_ctx* c) {
    return c->scheme == LLB_SCHEME_MOMENT ? c->buf[c->cur] : c->buf[1 - c->cur];
}

// A kernel whose bounded wait gave up leaves a non-zero word at err_dev.
int check_kernel_error(llb_ctx* c) {
    int err = 0;
    LLB_CUDA(c, cudaMemcpyAsync(&err, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "error word copy");
    LLB_CUDA(c, cudaStreamSynchronize(c->stream), "synchronize");
    if (err) {
        c->sticky = LLB_ETIMEOUT;
        return fail(c, LLB_ETIMEOUT, "a device wait gave up (a TMA load or a plane barrier did not complete)");
    }
    return LLB_OK;
}

int check_bad_flag(llb_ctx* c) {
    int bad = 0;
    LLB_CUDA(c, cudaMemcpyAsync(&bad, c->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "flag copy");
    LLB_CUDA(c, cudaStreamSynchronize(c->stream), "synchronize");
    if (bad) return fail(c, LLB_EUNSTABLE, "input has rho <= 0 or a non-finite value");
    return LLB_OK;
}

// Launch one step from buffer `cur` into the other copy, without flipping.
cudaError_t launch_one(llb_ctx* c, int cur) {
    const void* in = c->buf[cur];
    void* out = c->buf[1 - cur];
    if (c->ncomp == 2 && c->scheme == LLB_SCHEME_MOMENT) return launch_cg_tiled(*c, in, out);
    if (c->scheme == LLB_SCHEME_MOMENT)
        return c->kernel == LLB_KERNEL_TMA     ? launch_moment_tma(*c, cur, out)
               : c->kernel == LLB_KERNEL_TILED ? launch_moment_tiled(*c, cur, in, out)
                                               : launch_moment_direct(*c, in, out);
    return launch_population_step(*c, in, out, c->scheme == LLB_SCHEME_POPULATION_BGK);
}

// Prepare the launch plan of (kernel, variant); false if it cannot run this shape.
bool configure(llb_ctx* c, int kernel, int variant) {
    c->kernel = kernel;
    c->variant = variant;
    if (c->ncomp == 2 && c->scheme == LLB_SCHEME_MOMENT) {
        c->tile_ctas = cg_tiled_ctas(*c);
        cudaGetLastError();
        return kernel == LLB_KERNEL_TILED && c->tile_ctas > 0;
    }
    if (kernel == LLB_KERNEL_TILED) {
        c->tile_ctas = moment_tiled_ctas(*c);
        c->pmap_ok = moment_tiled_encode(*c, c->buf[0], &c->pmap[0]) && moment_tiled_encode(*c, c->buf[1], &c->pmap[1]);
        cudaGetLastError();
        return c->tile_ctas > 0;
    }
    if (kernel == LLB_KERNEL_TMA) {
        c->tmap_ok = moment_tma_encode(*c, c->buf[0], &c->tmap[0]) && moment_tma_encode(*c, c->buf[1], &c->tmap[1]);
        c->tma_ctas = c->tmap_ok ? moment_tma_ctas(*c) : 0;
        cudaGetLastError();
        return c->tma_ctas > 0;
    }
    return kernel == LLB_KERNEL_DIRECT;
}

void drop_graphs(llb_ctx* c) {
    for (int k = 0; k < 2; ++k) {
        if (c->graph_exec[k]) cudaGraphExecDestroy(c->graph_exec[k]);
        c->graph_exec[k] = nullptr;
        c->graph_steps[k] = 0;
    }
}

}  // namespace

extern "C" {

void llb_params_default(llb_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->ncomp = 1;
    p->storage = LLB_F32;
    p->scheme = LLB_SCHEME_MOMENT;
    p->kernel = LLB_KERNEL_AUTO;
    p->beta = 0.7;
    p->A_s = 0.01;
    p->A_h = 0.0;
    p->g_min = 1e-6;
    p->h_c = 3;
    p->stream = nullptr;
    p->buffers[0] = p->buffers[1] = nullptr;
    p->wait_budget_ms = 2000;
    p->grad_eps = 0.0;
}

int llb_footprint_query(int nx, int ny, int nz, int lattice, const llb_params* p, llb_footprint* out) {
    if (!out) return LLB_EINVAL;
    llb_params d;
    llb_params_default(&d);
    llb_ctx c;
    std::string why;
    llb_params q = p ? *p : d;
    // the accounting does not depend on whether the two-component kernels are built
    const int ncomp = q.ncomp;
    if (ncomp == 2) q.ncomp = 1;
    int rc = validate(nx, ny, nz, lattice, 0.75, q, &c, &why);
    if (rc != LLB_OK) return rc;
    if (ncomp != 1 && ncomp != 2) return LLB_EINVAL;
    c.ncomp = ncomp;
    c.nf = fields_of(c);
    c.lay = layout_of(c);
    out->fields = c.nf;
    out->arrays = 2 * c.nf;
    out->bytes_per_node = 2 * (size_t)c.nf * c.elem;
    out->state_bytes = state_bytes_of(c);
    out->stream_bytes_per_node = 2 * (size_t)c.nf * c.elem;
    return LLB_OK;
}

int llb_state_bytes(int nx, int ny, int nz, int lattice, const llb_params* p, size_t* out) {
    if (!out) return LLB_EINVAL;
    llb_footprint f;
    int rc = llb_footprint_query(nx, ny, nz, lattice, p, &f);
    if (rc == LLB_OK) *out = f.state_bytes;
    return rc;
}

int llb_create(llb_ctx** out, int nx, int ny, int nz, int lattice, double tau, const llb_params* p) {
    if (!out) return LLB_EINVAL;
    *out = nullptr;
    llb_params d;
    llb_params_default(&d);
    const llb_params& prm = p ? *p : d;
    llb_ctx* c = new (std::nothrow) llb_ctx();
    if (!c) return LLB_ENOMEM;
    std::string why;
    int rc = validate(nx, ny, nz, lattice, tau, prm, c, &why);
    if (rc != LLB_OK) {
        delete c;
        return rc;
    }
    c->stream = static_cast<cudaStream_t>(prm.stream);
    auto bail = [&](int code) {
        llb_destroy(c);
        return code;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) { cudaGetLastError(); return bail(LLB_ECUDA); }
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        return bail(LLB_ECUDA);
    }
    const size_t bytes = c->state_bytes;
    for (int b = 0; b < 2; ++b) {
        if (prm.buffers[b]) {
            if (reinterpret_cast<uintptr_t>(prm.buffers[b]) % 256 != 0) return bail(LLB_EINVAL);
            c->buf[b] = prm.buffers[b];
            c->owns[b] = false;
        } else {
            if (cudaMalloc(&c->buf[b], bytes) != cudaSuccess) { cudaGetLastError(); c->buf[b] = nullptr; return bail(LLB_ENOMEM); }
            c->owns[b] = true;
        }
        if (cudaMemsetAsync(c->buf[b], 0, bytes, c->stream) != cudaSuccess) { cudaGetLastError(); return bail(LLB_ECUDA); }
    }
    c->diag_scratch_bytes = (size_t)diag_blocks(*c) * 16 * sizeof(double) + 256;
    if (cudaMalloc(&c->diag_scratch, c->diag_scratch_bytes + sizeof(llb_diag)) != cudaSuccess) { cudaGetLastError(); c->diag_scratch = nullptr; return bail(LLB_ENOMEM); }
    if (cudaMalloc(&c->flag_dev, 2 * sizeof(int)) != cudaSuccess) { cudaGetLastError(); c->flag_dev = nullptr; return bail(LLB_ENOMEM); }
    c->err_dev = static_cast<int*>(c->flag_dev) + 1;
    if (c->scheme != LLB_SCHEME_MOMENT && c->ncomp == 2 &&
        cudaMalloc(&c->phi_scratch, c->N * c->elem) != cudaSuccess) { cudaGetLastError(); c->phi_scratch = nullptr; return bail(LLB_ENOMEM); }
    if (cudaMemsetAsync(c->flag_dev, 0, 2 * sizeof(int), c->stream) != cudaSuccess) { cudaGetLastError(); return bail(LLB_ECUDA); }
    if (c->scheme == LLB_SCHEME_MOMENT && c->ncomp == 2) {
        c->tile_ctas = cg_tiled_ctas(*c);
        cudaGetLastError();
        if (c->tile_ctas <= 0) return bail(LLB_EINVAL);
        c->kernel = LLB_KERNEL_TILED;
    } else if (c->scheme == LLB_SCHEME_MOMENT) {
        c->tile_ctas = moment_tiled_ctas(*c);
        c->pmap_ok = moment_tiled_encode(*c, c->buf[0], &c->pmap[0]) && moment_tiled_encode(*c, c->buf[1], &c->pmap[1]);
        cudaGetLastError();
        c->tmap_ok = moment_tma_encode(*c, c->buf[0], &c->tmap[0]) && moment_tma_encode(*c, c->buf[1], &c->tmap[1]);
        c->tma_ctas = c->tmap_ok ? moment_tma_ctas(*c) : 0;
        cudaGetLastError();
        const int want = c->kernel;
        if (want == LLB_KERNEL_TMA && c->tma_ctas <= 0) return bail(LLB_EINVAL);
        if (want == LLB_KERNEL_TILED && c->tile_ctas <= 0) return bail(LLB_EINVAL);
        // measured on GB300: the plain-load tiled kernel is the fastest, the TMA-staged one next
        if (want == LLB_KERNEL_AUTO)
            c->kernel = c->tile_ctas > 0 ? LLB_KERNEL_TILED : c->tma_ctas > 0 ? LLB_KERNEL_TMA : LLB_KERNEL_DIRECT;
    } else {
        c->kernel = LLB_KERNEL_DIRECT;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) { cudaGetLastError(); return bail(LLB_ECUDA); }
    *out = c;
    return LLB_OK;
}

void llb_destroy(llb_ctx* c) {
    if (!c || c->in_batch) return;  // a box of a batch is released by llb_batch_destroy
    cudaStreamSynchronize(c->stream);
    for (int b = 0; b < 2; ++b)
        if (c->owns[b] && c->buf[b]) cudaFree(c->buf[b]);
    if (c->staging) cudaFree(c->staging);
    if (c->diag_scratch) cudaFree(c->diag_scratch);
    if (c->flag_dev) cudaFree(c->flag_dev);
    if (c->phi_scratch) cudaFree(c->phi_scratch);
    if (c->staging_out) cudaFree(c->staging_out);
    for (int k = 0; k < 3; ++k)
        if (c->pipe[k]) cudaStreamDestroy(c->pipe[k]);
    drop_graphs(c);
    cudaGetLastError();
    delete c;
}

int llb_init_moments(llb_ctx* c, const void* host_m, int host_dtype) {
    LLB_CHECK_CTX(c);
    if (!host_m || !dtype_ok(host_dtype)) return fail(c, LLB_EINVAL, "null buffer or bad dtype");
    const size_t bytes = (size_t)canonical_fields(*c) * c->N * elem_size(host_dtype);
    int rc = ensure_staging(c, bytes);
    if (rc != LLB_OK) return rc;
    LLB_CUDA(c, cudaMemsetAsync(c->flag_dev, 0, sizeof(int), c->stream), "flag reset");
    LLB_CUDA(c, cudaMemcpyAsync(c->staging, host_m, bytes, cudaMemcpyHostToDevice, c->stream), "H2D moments");
    void* mom = init_target(c);
    LLB_CUDA(c, launch_canonical_to_shifted(*c, c->staging, host_dtype, mom, static_cast<int*>(c->flag_dev)), "convert");
    rc = finish_init(c, mom);
    if (rc != LLB_OK) return rc;
    return check_bad_flag(c);
}

int llb_init_moments_device(llb_ctx* c, const void* dev_m, int dtype) {
    LLB_CHECK_CTX(c);
    if (!dev_m || !dtype_ok(dtype)) return fail(c, LLB_EINVAL, "null buffer or bad dtype");
    void* mom = init_target(c);
    LLB_CUDA(c, launch_canonical_to_shifted(*c, dev_m, dtype, mom, nullptr), "convert");
    return finish_init(c, mom);
}

int llb_init_equilibrium(llb_ctx* c, const void* host_rho, const void* host_u, int host_dtype) {
    LLB_CHECK_CTX(c);
    if (!host_rho || !host_u || !dtype_ok(host_dtype)) return fail(c, LLB_EINVAL, "null buffer or bad dtype");
    const size_t es = elem_size(host_dtype);
    const size_t rho_bytes = (size_t)c->ncomp * c->N * es, u_bytes = 3 * c->N * es;
    int rc = ensure_staging(c, rho_bytes + u_bytes);
    if (rc != LLB_OK) return rc;
    char* st = static_cast<char*>(c->staging);
    LLB_CUDA(c, cudaMemsetAsync(c->flag_dev, 0, sizeof(int), c->stream), "flag reset");
    LLB_CUDA(c, cudaMemcpyAsync(st, host_rho, rho_bytes, cudaMemcpyHostToDevice, c->stream), "H2D rho");
    LLB_CUDA(c, cudaMemcpyAsync(st + rho_bytes, host_u, u_bytes, cudaMemcpyHostToDevice, c->stream), "H2D u");
    void* mom = init_target(c);
    LLB_CUDA(c, launch_equilibrium(*c, st, st + rho_bytes, host_dtype, mom, static_cast<int*>(c->flag_dev)), "equilibrium");
    rc = finish_init(c, mom);
    if (rc != LLB_OK) return rc;
    return check_bad_flag(c);
}

int llb_step(llb_ctx* c, int nsteps) {
    LLB_CHECK_CTX(c);
    if (c->in_batch) return fail(c, LLB_EINVAL, "this box belongs to a batch: step it with llb_batch_step");
    if (nsteps < 0) return fail(c, LLB_EINVAL, "nsteps must be >= 0");
    for (int s = 0; s < nsteps; ++s) {
        const cudaError_t e = launch_one(c, c->cur);
        if (e != cudaSuccess) return cuda_fail(c, e, "step kernel");
        c->cur = 1 - c->cur;
        ++c->t;
    }
    return LLB_OK;
}

int llb_step_graph(llb_ctx* c, int nsteps) {
    LLB_CHECK_CTX(c);
    if (c->in_batch) return fail(c, LLB_EINVAL, "this box belongs to a batch: step it with llb_batch_step");
    if (nsteps < 0) return fail(c, LLB_EINVAL, "nsteps must be >= 0");
    if (nsteps == 0) return LLB_OK;
    const int k = c->cur;
    if (!c->graph_exec[k] || c->graph_steps[k] != nsteps) {
        if (c->graph_exec[k]) {
            cudaGraphExecDestroy(c->graph_exec[k]);
            c->graph_exec[k] = nullptr;
        }
        // capture on a private stream (the context stream may be the legacy default stream)
        cudaStream_t cap = nullptr;
        LLB_CUDA(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
        cudaStream_t saved = c->stream;
        c->stream = cap;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        int cur = k;
        for (int s = 0; s < nsteps && e == cudaSuccess; ++s) {
            e = launch_one(c, cur);
            cur = 1 - cur;
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        c->stream = saved;
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph_exec[k], g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            c->graph_exec[k] = nullptr;
            return cuda_fail(c, e, "graph capture");
        }
        c->graph_steps[k] = nsteps;
    }
    LLB_CUDA(c, cudaGraphLaunch(c->graph_exec[k], c->stream), "graph launch");
    if (nsteps % 2) c->cur = 1 - c->cur;
    c->t += nsteps;
    return LLB_OK;
}

int llb_autotune(llb_ctx* c, int trials, int* kernel, int* variant) {
    LLB_CHECK_CTX(c);
    if (c->in_batch) return fail(c, LLB_EINVAL, "this box belongs to a batch: step it with llb_batch_step");
    if (trials < 1) return fail(c, LLB_EINVAL, "trials must be >= 1");
    if (c->scheme != LLB_SCHEME_MOMENT) {
        if (kernel) *kernel = c->kernel;
        if (variant) *variant = c->variant;
        return LLB_OK;
    }
    struct Cand { int kernel, variant; };
    Cand cands[24];
    int nc = 0;
    const int nvar = c->ncomp == 2 ? kCGVariants : (c->storage == LLB_F32 ? kTiledVariants32 : 1);
    for (int v = 0; v < nvar; ++v) cands[nc++] = {LLB_KERNEL_TILED, v};
    if (c->ncomp == 1) {
        const int ntma = c->storage == LLB_F32 ? kTmaVariants : (c->storage == LLB_F64 ? 1 : 0);
        for (int v = 0; v < ntma; ++v) cands[nc++] = {LLB_KERNEL_TMA, v};
        cands[nc++] = {LLB_KERNEL_DIRECT, 0};
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LLB_CUDA(c, cudaEventCreate(&e0), "event");
    LLB_CUDA(c, cudaEventCreate(&e1), "event");
    const int keep_k = c->kernel, keep_v = c->variant;
    float best = -1.0f;
    Cand win = {keep_k, keep_v};
    for (int i = 0; i < nc; ++i) {
        if (!configure(c, cands[i].kernel, cands[i].variant)) continue;
        // every trial recomputes step t -> t+1 into the spare copy: the state does not move
        cudaError_t e = launch_one(c, c->cur);
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        for (int r = 0; r < trials && e == cudaSuccess; ++r) e = launch_one(c, c->cur);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(c, e, "autotune");
        }
        if (best < 0.0f || ms < best) {
            best = ms;
            win = cands[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!configure(c, win.kernel, win.variant)) configure(c, keep_k, keep_v);
    drop_graphs(c);
    if (kernel) *kernel = c->kernel;
    if (variant) *variant = c->variant;
    return LLB_OK;
}

int llb_get_moments(llb_ctx* c, void* host_out, int host_dtype) {
    LLB_CHECK_CTX(c);
    if (!host_out || !dtype_ok(host_dtype)) return fail(c, LLB_EINVAL, "null buffer or bad dtype");
    const size_t bytes = (size_t)canonical_fields(*c) * c->N * elem_size(host_dtype);
    int rc = ensure_staging(c, bytes);
    if (rc != LLB_OK) return rc;
    const void* mom = nullptr;
    rc = current_moments(c, &mom);
    if (rc != LLB_OK) return rc;
    LLB_CUDA(c, launch_shifted_to_canonical(*c, mom, c->staging, host_dtype), "convert");
    LLB_CUDA(c, cudaMemcpyAsync(host_out, c->staging, bytes, cudaMemcpyDeviceToHost, c->stream), "D2H moments");
    LLB_CUDA(c, cudaStreamSynchronize(c->stream), "synchronize");
    return check_kernel_error(c);
}

int llb_get_moments_device(llb_ctx* c, void* dev_out, int dtype) {
    LLB_CHECK_CTX(c);
    if (!dev_out || !dtype_ok(dtype)) return fail(c, LLB_EINVAL, "null buffer or bad dtype");
    const void* mom = nullptr;
    int rc = current_moments(c, &mom);
    if (rc != LLB_OK) return rc;
    LLB_CUDA(c, launch_shifted_to_canonical(*c, mom, dev_out, dtype), "convert");
    return LLB_OK;
}

int llb_diagnostics(llb_ctx* c, llb_diag* out) {
    LLB_CHECK_CTX(c);
    if (!out) return fail(c, LLB_EINVAL, "null output");
    const void* mom = nullptr;
    int rc = current_moments(c, &mom);
    if (rc != LLB_OK) return rc;
    llb_diag* dev_out = reinterpret_cast<llb_diag*>(static_cast<char*>(c->diag_scratch) + c->diag_scratch_bytes);
    LLB_CUDA(c, launch_diagnostics(*c, mom, c->diag_scratch, dev_out), "diagnostics");
    LLB_CUDA(c, cudaMemcpyAsync(out, dev_out, sizeof(llb_diag), cudaMemcpyDeviceToHost, c->stream), "D2H diag");
    LLB_CUDA(c, cudaStreamSynchronize(c->stream), "synchronize");
    return check_kernel_error(c);
}

int llb_synchronize(llb_ctx* c) {
    LLB_CHECK_CTX(c);
    LLB_CUDA(c, cudaStreamSynchronize(c->stream), "synchronize");
    return check_kernel_error(c);
}

int llb_steps_done(const llb_ctx* c, long long* out) {
    if (!c || !out) return LLB_EINVAL;
    *out = c->t;
    return LLB_OK;
}

int llb_state_device(const llb_ctx* c, void** dev_ptr, int* dtype, int* kernel) {
    if (!c) return LLB_EINVAL;
    if (dev_ptr) *dev_ptr = c->buf[c->cur];
    if (dtype) *dtype = c->storage;
    if (kernel) *kernel = c->kernel;
    return LLB_OK;
}

const char* llb_status_string(int s) {
    switch (s) {
        case LLB_OK: return "ok";
        case LLB_EINVAL: return "invalid argument";
        case LLB_ENOMEM: return "out of memory";
        case LLB_ECUDA: return "CUDA error";
        case LLB_EUNSTABLE: return "unstable state (rho <= 0 or non-finite)";
        case LLB_ETIMEOUT: return "device wait timed out";
        case LLB_ESTATE: return "context unusable after an earlier CUDA error";
        default: return "unknown status";
    }
}

const char* llb_last_error(const llb_ctx* c) {
    if (!c) return "no context";
    return c->msg.c_str();
}

int llb_checked_status(int* enabled, int* site, long long* index) {
#ifdef LLB_CHECKED
    const int on = 1;
#else
    const int on = 0;
#endif
    if (enabled) *enabled = on;
    if (site) *site = 0;
    if (index) *index = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return LLB_ECUDA;
    int (*const take[])(int*, long long*) = {llb::chk_take_tiled_f32, llb::chk_take_tiled_f64,
                                             llb::chk_take_tiled_f16, llb::chk_take_tiled_bf16,
                                             llb::chk_take_step,      llb::chk_take_tma,
                                             llb::chk_take_cg,        llb::chk_take_cg_batch,
                                             llb::chk_take_pop,       llb::chk_take_adjoint};
    int first = 0;
    long long first_i = 0;
    bool failed = false;
    for (auto f : take) {
        int s = 0;
        long long i = 0;
        if (f(&s, &i) != 0) failed = true;
        if (s && !first) {
            first = s;
            first_i = i;
        }
    }
    if (site) *site = first;
    if (index) *index = first_i;
    return failed ? LLB_ECUDA : LLB_OK;
}

}  // extern "C"
