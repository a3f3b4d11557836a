// llb_step_host: moments in from host memory, time steps, moments out to host
// memory, with the host<->device copies overlapped with the device work.
//
// The box is cut into K slabs of whole z-planes.  Three streams of the
// context carry the work: the copy-in stream copies slab k of the canonical
// input (one copy per field) and converts it to the shifted state; the step
// stream runs the step for the output planes of slab k as soon as the input
// slabs k-1, k, k+1 have arrived (the pull reaches one plane across each
// slab boundary); the copy-out stream converts the finished output planes of
// slab k back to canonical moments and copies them to the host.  Events
// order the three streams; slab copies in, steps and copies out of
// different slabs run at the same time, so the call takes about as long as
// the larger of the two host copies.  Slabs are stepped in the order
// 1, 2, ..., K-1, 0: slab 0 needs the last slab of the box (periodic wrap).
//
// With nsteps > 1 the first step is pipelined with the copies in, the middle
// steps are ordinary launches and the last step is pipelined with the copies
// out.  One-component moment-only contexts on the tiled kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "internal.h"

namespace llb {
namespace {

constexpr int kMaxSlabs = 16;

int pipe_setup(llb_ctx* c, size_t out_bytes) {
    for (int k = 0; k < 3; ++k)
        if (!c->pipe[k] && cudaStreamCreateWithFlags(&c->pipe[k], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            c->pipe[k] = nullptr;
            return LLB_ECUDA;
        }
    if (c->staging_out_bytes < out_bytes) {
        if (c->staging_out) {
            cudaFree(c->staging_out);
            c->staging_out = nullptr;
            c->staging_out_bytes = 0;
        }
        if (cudaMalloc(&c->staging_out, out_bytes) != cudaSuccess) {
            cudaGetLastError();
            c->staging_out = nullptr;
            return LLB_ENOMEM;
        }
        c->staging_out_bytes = out_bytes;
    }
    return LLB_OK;
}

struct Events {
    cudaEvent_t ev[3 * kMaxSlabs + 2] = {};
    int n = 0;
    ~Events() {
        for (int i = 0; i < n; ++i) cudaEventDestroy(ev[i]);
    }
    cudaError_t make(int count) {
        for (; n < count; ++n)
            if (cudaError_t e = cudaEventCreateWithFlags(&ev[n], cudaEventDisableTiming); e != cudaSuccess) return e;
        return cudaSuccess;
    }
};

}  // namespace
}  // namespace llb

using namespace llb;

extern "C" int llb_step_host(llb_ctx* c, const void* host_in, void* host_out, int host_dtype, int nsteps) {
    if (!c) return LLB_EINVAL;
    if (c->sticky != LLB_OK) return LLB_ESTATE;
    if (c->in_batch || !host_in || !host_out || (host_dtype != LLB_F64 && host_dtype != LLB_F32) || nsteps < 1) {
        c->msg = "llb_step_host: bad argument";
        return LLB_EINVAL;
    }
    if (c->scheme != LLB_SCHEME_MOMENT || c->ncomp != 1 || c->kernel != LLB_KERNEL_TILED) {
        // other schemes and kernels: the same result without the overlap
        int rc = llb_init_moments(c, host_in, host_dtype);
        if (rc == LLB_OK) rc = llb_step(c, nsteps);
        if (rc == LLB_OK) rc = llb_get_moments(c, host_out, host_dtype);
        return rc;
    }
    const size_t es = elem_size(host_dtype), N = c->N, plane = (size_t)c->nx * c->ny;
    const size_t bytes = 10 * N * es;
    if (c->staging_bytes < bytes) {
        if (c->staging) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->staging);
            c->staging = nullptr;
            c->staging_bytes = 0;
        }
        if (cudaMalloc(&c->staging, bytes) != cudaSuccess) {
            cudaGetLastError();
            c->msg = "cudaMalloc of the staging buffer failed";
            return LLB_ENOMEM;
        }
        c->staging_bytes = bytes;
    }
    if (int rc = pipe_setup(c, bytes); rc != LLB_OK) {
        c->msg = "llb_step_host: stream or staging set-up failed";
        return rc;
    }
    const int K = std::max(1, std::min(kMaxSlabs, c->nz / 8));
    int zb[kMaxSlabs + 1];
    for (int k = 0; k <= K; ++k) zb[k] = (int)((long long)k * c->nz / K);
    Events E;
    cudaError_t e = E.make(3 * K + 2);
    cudaEvent_t* ev_in = E.ev;             // slab k converted into the state
    cudaEvent_t* ev_step = E.ev + K;       // output planes of slab k written
    cudaEvent_t* ev_out = E.ev + 2 * K;    // slab k copied to the host (unused but for ordering)
    cudaEvent_t ev_start = E.ev[3 * K], ev_mid = E.ev[3 * K + 1];
    cudaStream_t sin = c->pipe[0], scmp = c->pipe[1], sout = c->pipe[2];
    const char* host_i = static_cast<const char*>(host_in);
    char* host_o = static_cast<char*>(host_out);
    char* dev_i = static_cast<char*>(c->staging);
    char* dev_o = static_cast<char*>(c->staging_out);
    int* bad = static_cast<int*>(c->flag_dev);
    // the pipeline starts after all earlier work of the context stream
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev_start, c->stream);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(c->pipe[k], ev_start, 0);

    // copies in: slab by slab, one copy per field
    int cur = c->cur;
    for (int k = 0; k < K && e == cudaSuccess; ++k) {
        const size_t off = (size_t)zb[k] * plane * es, len = (size_t)(zb[k + 1] - zb[k]) * plane * es;
        for (int f = 0; f < 10 && e == cudaSuccess; ++f)
            e = cudaMemcpyAsync(dev_i + f * N * es + off, host_i + f * N * es + off, len, cudaMemcpyHostToDevice, sin);
        if (e == cudaSuccess)
            e = launch_canonical_to_shifted_range(*c, dev_i, host_dtype, c->buf[cur], bad, zb[k], zb[k + 1], sin);
        if (e == cudaSuccess) e = cudaEventRecord(ev_in[k], sin);
    }
    // one pipelined step (from buf[cur] to buf[1 - cur]); `wait_in`: slabs wait for their inputs,
    // `copy_out`: finished slabs go straight to the host
    auto pipelined_step = [&](bool wait_in, bool copy_out) {
        for (int i = 0; i < K && e == cudaSuccess; ++i) {
            const int k = K == 1 ? 0 : (i + 1) % K;   // 1, 2, ..., K-1, 0
            if (wait_in) {
                const int need = (k == K - 1 || k == 0) ? K - 1 : k + 1;  // highest input slab this slab reads
                e = cudaStreamWaitEvent(scmp, ev_in[need], 0);
            }
            if (e == cudaSuccess)
                e = launch_moment_tiled_range(*c, cur, c->buf[cur], c->buf[1 - cur], zb[k], zb[k + 1], scmp);
            if (e == cudaSuccess) e = cudaEventRecord(ev_step[k], scmp);
            if (copy_out && e == cudaSuccess) {
                e = cudaStreamWaitEvent(sout, ev_step[k], 0);
                if (e == cudaSuccess)
                    e = launch_shifted_to_canonical_range(*c, c->buf[1 - cur], dev_o, host_dtype, zb[k], zb[k + 1],
                                                          sout);
                const size_t off = (size_t)zb[k] * plane * es, len = (size_t)(zb[k + 1] - zb[k]) * plane * es;
                for (int f = 0; f < 10 && e == cudaSuccess; ++f)
                    e = cudaMemcpyAsync(host_o + f * N * es + off, dev_o + f * N * es + off, len,
                                        cudaMemcpyDeviceToHost, sout);
                if (e == cudaSuccess) e = cudaEventRecord(ev_out[k], sout);
            }
        }
        cur = 1 - cur;
    };
    pipelined_step(true, nsteps == 1);
    if (nsteps > 1 && e == cudaSuccess) {
        // middle steps on the step stream, then the last one with the copies out
        for (int s = 1; s < nsteps - 1 && e == cudaSuccess; ++s) {
            e = launch_moment_tiled_range(*c, cur, c->buf[cur], c->buf[1 - cur], 0, c->nz, scmp);
            cur = 1 - cur;
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_mid, scmp);
        if (e == cudaSuccess) pipelined_step(false, true);
    }
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaStreamSynchronize(c->pipe[k]);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->sticky = LLB_ECUDA;
        c->msg = std::string("llb_step_host: ") + cudaGetErrorString(e);
        return LLB_ECUDA;
    }
    c->cur = cur;
    c->t = nsteps;
    int flags[2] = {0, 0};
    if (cudaMemcpy(flags, c->flag_dev, 2 * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        c->sticky = LLB_ECUDA;
        return LLB_ECUDA;
    }
    if (flags[1]) {
        c->sticky = LLB_ETIMEOUT;
        c->msg = "a device wait gave up";
        return LLB_ETIMEOUT;
    }
    if (flags[0]) {
        c->msg = "input has rho <= 0 or a non-finite value";
        return LLB_EUNSTABLE;
    }
    return LLB_OK;
}
