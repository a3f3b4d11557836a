// Batched ensembles of independent boxes advanced by one persistent launch
// per step (two components; the ensemble workload of droplet collisions of
// different sizes).  Each box is an ordinary context (its own state copies,
// initialisation, read-back and diagnostics); the batch adds one device table
// of boxes per flip-flop parity and the launch that walks every box's work
// items in one grid.  The CTAs take items from a work queue (a counter zeroed
// before each launch), so that the items of boxes of different sizes, which
// differ in length, even out over the grid.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"

struct llb_batch {
    int n = 0;
    std::vector<llb_ctx*> ctx;
    llb::BatchDom* dev_doms[2] = {nullptr, nullptr};
    int* dev_next = nullptr;  // work queue: next item to take (zeroed before every launch)
    int total = 0;   // work items over all boxes
    int grid = 0;    // persistent CTAs
    int variant = 0;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int graph_steps[2] = {0, 0};
    long long nodes = 0;
    int sticky = LLB_OK;
};

namespace {

void drop_graphs(llb_batch* b) {
    for (int k = 0; k < 2; ++k) {
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
        b->graph[k] = nullptr;
        b->graph_steps[k] = 0;
    }
}

// (Re)build the box tables for the current variant: schedules, item offsets, grid.
int build_tables(llb_batch* b) {
    for (llb_ctx* c : b->ctx) c->variant = b->variant;
    const int grid = llb::cg_batch_ctas(*b->ctx[0]);
    if (grid <= 0) return LLB_EINVAL;
    std::vector<llb::BatchDom> h[2];
    h[0].resize(b->n);
    h[1].resize(b->n);
    int begin = 0;
    for (int d = 0; d < b->n; ++d) {
        llb_ctx* c = b->ctx[d];
        // each box is chunked as if it had its share of the grid, proportional to its nodes
        const double share = (double)c->N / (double)b->nodes;
        const int g = (int)std::fmax(1.0, std::floor(share * grid));
        llb::BatchDom dom;
        std::memset(&dom, 0, sizeof(dom));
        llb::cg_batch_plan(*c, g, &dom);
        dom.lay = c->lay;
        dom.item_begin = begin;
        begin += dom.nitems;
        for (int k = 0; k < 2; ++k) {
            h[k][d] = dom;
            h[k][d].in = c->buf[k];
            h[k][d].out = c->buf[1 - k];
        }
    }
    if (!b->dev_next && cudaMalloc(&b->dev_next, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        b->dev_next = nullptr;
        return LLB_ENOMEM;
    }
    for (int k = 0; k < 2; ++k) {
        if (!b->dev_doms[k] && cudaMalloc(&b->dev_doms[k], sizeof(llb::BatchDom) * b->n) != cudaSuccess) {
            cudaGetLastError();
            b->dev_doms[k] = nullptr;
            return LLB_ENOMEM;
        }
        if (cudaMemcpy(b->dev_doms[k], h[k].data(), sizeof(llb::BatchDom) * b->n, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
            cudaGetLastError();
            return LLB_ECUDA;
        }
    }
    b->total = begin;
    b->grid = grid < begin ? grid : begin;
    drop_graphs(b);
    return LLB_OK;
}

cudaError_t launch(llb_batch* b, int parity) {
    const cudaError_t e = cudaMemsetAsync(b->dev_next, 0, sizeof(int), b->ctx[0]->stream);
    if (e != cudaSuccess) return e;
    return llb::launch_cg_batch(*b->ctx[0], b->dev_doms[parity], b->n, b->total, b->grid, b->dev_next);
}

void advance(llb_batch* b, int nsteps) {
    for (llb_ctx* c : b->ctx) {
        if (nsteps % 2) c->cur = 1 - c->cur;
        c->t += nsteps;
    }
}

#define LLB_BATCH_CHECK(b)                          \
    do {                                            \
        if (!(b)) return LLB_EINVAL;                \
        if ((b)->sticky != LLB_OK) return LLB_ESTATE; \
    } while (0)

}  // namespace

extern "C" {

int llb_batch_create(llb_batch** out, int ndomains, const int* dims, int lattice, double tau, const llb_params* p) {
    if (!out) return LLB_EINVAL;
    *out = nullptr;
    if (ndomains < 1 || ndomains > 65536 || !dims || !p || p->ncomp != 2 || p->scheme != LLB_SCHEME_MOMENT)
        return LLB_EINVAL;
    llb_batch* b = new (std::nothrow) llb_batch();
    if (!b) return LLB_ENOMEM;
    b->n = ndomains;
    b->variant = p->variant;
    b->stream = static_cast<cudaStream_t>(p->stream);
    llb_params q = *p;
    q.buffers[0] = q.buffers[1] = nullptr;
    q.kernel = LLB_KERNEL_AUTO;
    for (int d = 0; d < ndomains; ++d) {
        llb_ctx* c = nullptr;
        const int rc = llb_create(&c, dims[3 * d], dims[3 * d + 1], dims[3 * d + 2], lattice, tau, &q);
        if (rc != LLB_OK) {
            llb_batch_destroy(b);
            return rc;
        }
        c->in_batch = true;
        b->ctx.push_back(c);
        b->nodes += (long long)c->N;
    }
    const int rc = build_tables(b);
    if (rc != LLB_OK) {
        llb_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LLB_OK;
}

void llb_batch_destroy(llb_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (int k = 0; k < 2; ++k)
        if (b->dev_doms[k]) cudaFree(b->dev_doms[k]);
    if (b->dev_next) cudaFree(b->dev_next);
    for (llb_ctx* c : b->ctx) {
        c->in_batch = false;
        llb_destroy(c);
    }
    cudaGetLastError();
    delete b;
}

int llb_batch_domain(llb_batch* b, int d, llb_ctx** ctx) {
    LLB_BATCH_CHECK(b);
    if (!ctx || d < 0 || d >= b->n) return LLB_EINVAL;
    *ctx = b->ctx[d];
    return LLB_OK;
}

int llb_batch_nodes(const llb_batch* b, long long* nodes) {
    if (!b || !nodes) return LLB_EINVAL;
    *nodes = b->nodes;
    return LLB_OK;
}

int llb_batch_step(llb_batch* b, int nsteps) {
    LLB_BATCH_CHECK(b);
    if (nsteps < 0) return LLB_EINVAL;
    for (int s = 0; s < nsteps; ++s) {
        if (launch(b, b->ctx[0]->cur) != cudaSuccess) {
            b->sticky = LLB_ECUDA;
            return LLB_ECUDA;
        }
        advance(b, 1);
    }
    return LLB_OK;
}

int llb_batch_step_graph(llb_batch* b, int nsteps) {
    LLB_BATCH_CHECK(b);
    if (nsteps < 0) return LLB_EINVAL;
    if (nsteps == 0) return LLB_OK;
    const int k = b->ctx[0]->cur;
    if (!b->graph[k] || b->graph_steps[k] != nsteps) {
        if (b->graph[k]) {
            cudaGraphExecDestroy(b->graph[k]);
            b->graph[k] = nullptr;
        }
        cudaStream_t cap = nullptr;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return LLB_ECUDA;
        }
        cudaStream_t saved = b->ctx[0]->stream;
        b->ctx[0]->stream = cap;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        int cur = k;
        for (int s = 0; s < nsteps && e == cudaSuccess; ++s) {
            e = launch(b, cur);
            cur = 1 - cur;
        }
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        b->ctx[0]->stream = saved;
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[k], g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cap);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b->graph[k] = nullptr;
            b->sticky = LLB_ECUDA;
            return LLB_ECUDA;
        }
        b->graph_steps[k] = nsteps;
    }
    if (cudaGraphLaunch(b->graph[k], b->stream) != cudaSuccess) {
        cudaGetLastError();
        b->sticky = LLB_ECUDA;
        return LLB_ECUDA;
    }
    advance(b, nsteps);
    return LLB_OK;
}

int llb_batch_autotune(llb_batch* b, int trials, int* variant) {
    LLB_BATCH_CHECK(b);
    if (trials < 1) return LLB_EINVAL;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return LLB_ECUDA;
    }
    const int keep = b->variant;
    float best = -1.0f;
    int win = keep;
    for (int v = 0; v < llb::kCGVariants; ++v) {
        b->variant = v;
        if (build_tables(b) != LLB_OK) continue;
        // each trial recomputes the current step into the spare copies: the state does not move
        const int par = b->ctx[0]->cur;
        cudaError_t e = launch(b, par);
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        for (int r = 0; r < trials && e == cudaSuccess; ++r) e = launch(b, par);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            b->sticky = LLB_ECUDA;
            return LLB_ECUDA;
        }
        if (best < 0.0f || ms < best) {
            best = ms;
            win = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->variant = win;
    const int rc = build_tables(b);
    if (rc != LLB_OK) {
        b->variant = keep;
        build_tables(b);
        return rc;
    }
    if (variant) *variant = win;
    return LLB_OK;
}

}  // extern "C"
