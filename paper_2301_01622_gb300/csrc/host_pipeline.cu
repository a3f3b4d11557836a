// llb_step_host: moments in from host memory, time steps, moments out to host
// memory, with the host<->device copies overlapped with the device work.
//
// The box is cut into K slabs of whole z-planes (up to 32, at least 8 planes
// each).  Three streams of the context carry the work:
//   * copy-in: one 2D copy per slab (the ten fields of the slab, each a
//     contiguous run, strided by the field size) into a device staging buffer;
//   * step: converts each arrived slab to the shifted state, runs the step for
//     the output planes of slab k as soon as the input slabs k-1, k, k+1 are
//     converted (the pull reaches one plane across each slab boundary), and
//     converts the finished output planes back to canonical moments;
//   * copy-out: one 2D copy per finished slab to the host.
// The copy streams carry nothing but copies, so both directions of the host
// link stay busy; the conversions and steps (tens of microseconds per slab)
// run between them.  Events order the streams.  Slabs are stepped in the order
// 1, 2, ..., K-1, 0: slab 0 needs the last slab of the box (periodic wrap).
//
// With nsteps > 1 the first step is pipelined with the copies in, the middle
// steps are ordinary launches and the last step is pipelined with the copies
// out.  Moment-only contexts on the tiled kernels: one component (the pull
// reaches one plane) and two components (the phase-field gradient of a source
// node reaches two planes, the near-contact probes 1 + h_c); every slab is at
// least that thick, so a slab's inputs are still its own and its two
// neighbours'.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "internal.h"

namespace llb {
namespace {

constexpr int kMaxSlabs = 32;

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

// Copy the nf fields of planes [z0, z1) between host and device canonical
// arrays (field-major, field size N elements of es bytes): one 2D copy when
// the field stride is within the copy engine's pitch limit, else one copy per
// field.
cudaError_t copy_slab(void* dst, const void* src, size_t N, size_t es, int nf, size_t off, size_t len,
                      cudaMemcpyKind kind, cudaStream_t st) {
    static int max_pitch = -1;
    if (max_pitch < 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMaxPitch, dev) != cudaSuccess)
            v = 0;
        max_pitch = v;
    }
    char* d = static_cast<char*>(dst) + off;
    const char* s = static_cast<const char*>(src) + off;
    if (N * es <= (size_t)max_pitch) return cudaMemcpy2DAsync(d, N * es, s, N * es, len, nf, kind, st);
    for (int f = 0; f < nf; ++f)
        if (cudaError_t e = cudaMemcpyAsync(d + f * N * es, s + f * N * es, len, kind, st); e != cudaSuccess) return e;
    return cudaSuccess;
}

struct Events {
    cudaEvent_t ev[2 * kMaxSlabs + 1] = {};
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
    const bool two = c->ncomp == 2;
    if (c->scheme != LLB_SCHEME_MOMENT || (!two && c->kernel != LLB_KERNEL_TILED)) {
        // other schemes and kernels: the same result without the overlap
        int rc = llb_init_moments(c, host_in, host_dtype);
        if (rc == LLB_OK) rc = llb_step(c, nsteps);
        if (rc == LLB_OK) rc = llb_get_moments(c, host_out, host_dtype);
        return rc;
    }
    const size_t es = elem_size(host_dtype), N = c->N, plane = (size_t)c->nx * c->ny;
    const int nf = two ? 11 : 10;
    const size_t bytes = (size_t)nf * N * es;
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
    // planes a slab's step reaches beyond the slab: the pull (1); for two
    // components the gradient of phi at the source planes (2) and the
    // near-contact probes (1 + h_c)
    const int reach = two ? std::max(2, c->params.A_h != 0.0 ? 1 + c->params.h_c : 0) : 1;
    const int K = std::max(1, std::min(kMaxSlabs, c->nz / std::max(8, reach)));
    int zb[kMaxSlabs + 1];
    for (int k = 0; k <= K; ++k) zb[k] = (int)((long long)k * c->nz / K);
    Events E;
    cudaError_t e = E.make(2 * K + 1);
    cudaEvent_t* ev_copied = E.ev;         // slab k of the input is in the staging buffer
    cudaEvent_t* ev_ready = E.ev + K;      // output planes of slab k are canonical in the output staging buffer
    cudaEvent_t ev_start = E.ev[2 * K];
    cudaStream_t sin = c->pipe[0], scmp = c->pipe[1], sout = c->pipe[2];
    char* dev_i = static_cast<char*>(c->staging);
    char* dev_o = static_cast<char*>(c->staging_out);
    int* bad = static_cast<int*>(c->flag_dev);
    // the pipeline starts after all earlier work of the context stream
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev_start, c->stream);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(c->pipe[k], ev_start, 0);
    auto slab_off = [&](int k) { return (size_t)zb[k] * plane * es; };
    auto slab_len = [&](int k) { return (size_t)(zb[k + 1] - zb[k]) * plane * es; };

    // copies in: nothing but copies on this stream
    int cur = c->cur;
    for (int k = 0; k < K && e == cudaSuccess; ++k) {
        e = copy_slab(dev_i, host_in, N, es, nf, slab_off(k), slab_len(k), cudaMemcpyHostToDevice, sin);
        if (e == cudaSuccess) e = cudaEventRecord(ev_copied[k], sin);
    }
    int converted = 0;  // input slabs 0 .. converted-1 are in the shifted state
    // one pipelined step (from buf[cur] to buf[1 - cur]); `wait_in`: input slabs are
    // converted as they arrive, `copy_out`: finished slabs go straight to the host
    auto pipelined_step = [&](bool wait_in, bool copy_out) {
        for (int i = 0; i < K && e == cudaSuccess; ++i) {
            const int k = K == 1 ? 0 : (i + 1) % K;   // 1, 2, ..., K-1, 0
            if (wait_in) {
                const int need = (k == K - 1 || k == 0) ? K - 1 : k + 1;  // highest input slab this slab reads
                while (converted <= need && e == cudaSuccess) {
                    e = cudaStreamWaitEvent(scmp, ev_copied[converted], 0);
                    if (e == cudaSuccess)
                        e = launch_canonical_to_shifted_range(*c, dev_i, host_dtype, c->buf[cur], bad, zb[converted],
                                                              zb[converted + 1], scmp);
                    ++converted;
                }
            }
            if (e == cudaSuccess)
                e = two ? launch_cg_tiled_range(*c, c->buf[cur], c->buf[1 - cur], zb[k], zb[k + 1], scmp)
                        : launch_moment_tiled_range(*c, cur, c->buf[cur], c->buf[1 - cur], zb[k], zb[k + 1], scmp);
            if (copy_out && e == cudaSuccess) {
                e = launch_shifted_to_canonical_range(*c, c->buf[1 - cur], dev_o, host_dtype, zb[k], zb[k + 1], scmp);
                if (e == cudaSuccess) e = cudaEventRecord(ev_ready[k], scmp);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, ev_ready[k], 0);
                if (e == cudaSuccess)
                    e = copy_slab(host_out, dev_o, N, es, nf, slab_off(k), slab_len(k), cudaMemcpyDeviceToHost, sout);
            }
        }
        cur = 1 - cur;
    };
    pipelined_step(true, nsteps == 1);
    if (nsteps > 1 && e == cudaSuccess) {
        // middle steps on the step stream, then the last one with the copies out
        for (int s = 1; s < nsteps - 1 && e == cudaSuccess; ++s) {
            e = two ? launch_cg_tiled_range(*c, c->buf[cur], c->buf[1 - cur], 0, c->nz, scmp)
                    : launch_moment_tiled_range(*c, cur, c->buf[cur], c->buf[1 - cur], 0, c->nz, scmp);
            cur = 1 - cur;
        }
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
