// FP64 reductions over the shifted moments (validation diagnostics of
// Sec. IV: droplet density <rho>_{rho > 0.5} of Figs. 2, 5, 7; total mass and
// momentum, which BGK collision and periodic streaming conserve).
//
// Pass 1: a fixed grid of blocks walks the nodes with a grid-stride loop,
// reduces in registers, then warp shuffles, then across the block's warps
// through shared memory, and writes one row of partials per block to a
// scratch array.  Pass 2: one block reduces the rows in a fixed order.  The
// result is deterministic for a given grid.
#include <cuda_runtime.h>

#include <cfloat>
#include <mutex>

#include "internal.h"
#include "lattice.cuh"
#include "layout.cuh"
#include "storage.cuh"

namespace llb {
namespace {

constexpr int kDiagThreads = 256;
constexpr int kRow = 9;  // sum d, sum jx, sum jy, sum jz, sum rho_in, n_in, min rho, nonfinite, sum rho1

struct Part {
    double v[kRow];
};

__device__ __forceinline__ void part_init(Part& p) {
#pragma unroll
    for (int k = 0; k < kRow; ++k) p.v[k] = 0.0;
    p.v[6] = DBL_MAX;
}

__device__ __forceinline__ void part_merge(Part& a, const Part& b) {
#pragma unroll
    for (int k = 0; k < 6; ++k) a.v[k] += b.v[k];
    a.v[6] = fmin(a.v[6], b.v[6]);
    a.v[7] = fmax(a.v[7], b.v[7]);
    a.v[8] += b.v[8];
}

__device__ __forceinline__ Part warp_reduce(Part p) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Part o;
#pragma unroll
        for (int k = 0; k < kRow; ++k) o.v[k] = __shfl_down_sync(0xffffffffu, p.v[k], off);
        part_merge(p, o);
    }
    return p;
}

// Block-wide reduction; the result is valid in thread 0.
__device__ Part block_reduce(Part p) {
    __shared__ double sh[kDiagThreads / 32][kRow];
    p = warp_reduce(p);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < kRow; ++k) sh[wid][k] = p.v[k];
    __syncthreads();
    if (wid == 0) {
        Part q;
        part_init(q);
        if (lane < kDiagThreads / 32)
            for (int k = 0; k < kRow; ++k) q.v[k] = sh[lane][k];
        p = warp_reduce(q);
    }
    return p;
}

// Row of partial sums: (sum d, sum j, sum of the droplet density over nodes
// where it exceeds 0.5, their count, min rho, non-finite flag, sum rho1).
// The droplet density is rho for one component and rho1 for two (state
// rho1, d, j, A; rho2 = 1 + d - rho1 is recovered from the sums).
template <class T, int NC>
__global__ void __launch_bounds__(kDiagThreads) k_diag_partial(const T* __restrict__ m, Layout L,
                                                               double* __restrict__ rows) {
    Part p;
    part_init(p);
    const size_t N = (size_t)L.nx * L.ny * L.nz, F = L.fs;
    constexpr int o = NC == 2 ? 1 : 0;  // field offset of d
    for (size_t n = blockIdx.x * (size_t)kDiagThreads + threadIdx.x; n < N; n += (size_t)gridDim.x * kDiagThreads) {
        const int x = (int)(n % L.nx);
        const size_t r = n / L.nx;
        const size_t i = L.at(x, (int)(r % L.ny), (int)(r / L.ny));
        using FM = FieldMap<T, NC == 2 ? 11 : 10>;
        const double d = rd_field(m[FM::at(i, o, F)], 0);
        const double jx = rd_field(m[FM::at(i, o + 1, F)], 1), jy = rd_field(m[FM::at(i, o + 2, F)], 2),
                     jz = rd_field(m[FM::at(i, o + 3, F)], 3);
        const double rho = 1.0 + d;
        const double drop = NC == 2 ? rd_field(m[FM::at(i, 0, F)], 0) : rho;
        p.v[0] += d;
        p.v[1] += jx;
        p.v[2] += jy;
        p.v[3] += jz;
        if (drop > 0.5) {
            p.v[4] += drop;
            p.v[5] += 1.0;
        }
        p.v[6] = fmin(p.v[6], rho);
        if (NC == 2) p.v[8] += drop;
        bool finite = isfinite(d) && isfinite(jx) && isfinite(jy) && isfinite(jz) && isfinite(drop);
#pragma unroll
        for (int f = o + 4; f < o + 10; ++f) finite = finite && isfinite(rd_field(m[FM::at(i, f, F)], f - o));
        if (!finite) p.v[7] = 1.0;
    }
    p = block_reduce(p);
    if (threadIdx.x == 0)
        for (int k = 0; k < kRow; ++k) rows[(size_t)blockIdx.x * kRow + k] = p.v[k];
}

__global__ void __launch_bounds__(kDiagThreads) k_diag_final(const double* __restrict__ rows, int nrows, size_t N,
                                                             int ncomp, llb_diag* __restrict__ out) {
    Part p;
    part_init(p);
    for (int r = threadIdx.x; r < nrows; r += kDiagThreads) {
        Part q;
        for (int k = 0; k < kRow; ++k) q.v[k] = rows[(size_t)r * kRow + k];
        part_merge(p, q);
    }
    p = block_reduce(p);
    if (threadIdx.x == 0) {
        if (ncomp == 2) {
            out->mass[0] = p.v[8];
            out->mass[1] = (double)N + p.v[0] - p.v[8];
        } else {
            out->mass[0] = (double)N + p.v[0];
            out->mass[1] = 0.0;
        }
        out->momentum[0] = p.v[1];
        out->momentum[1] = p.v[2];
        out->momentum[2] = p.v[3];
        out->rho1_sum = p.v[4];
        out->n_in = (long long)p.v[5];
        out->rho1_avg = p.v[5] > 0.0 ? p.v[4] / p.v[5] : 0.0;
        const bool nonfinite = p.v[7] != 0.0;
        out->min_rho = nonfinite ? __longlong_as_double(0x7ff8000000000000ULL) : p.v[6];
        out->flags = (nonfinite ? LLB_FLAG_NONFINITE : 0) | (!nonfinite && p.v[6] <= 0.0 ? LLB_FLAG_NONPOSITIVE : 0);
        out->reserved = 0;
    }
}

}  // namespace

int diag_blocks(const llb_ctx& c) {
    const size_t want = (c.N + kDiagThreads - 1) / kDiagThreads;
    const size_t cap = (size_t)(c.num_sms > 0 ? c.num_sms : 148) * 4;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

cudaError_t launch_diagnostics(const llb_ctx& c, const void* mom, void* scratch, llb_diag* dev_out) {
    const int nb = diag_blocks(c);
    double* rows = static_cast<double*>(scratch);
    if (c.storage == LLB_F16S)
        k_diag_partial<__half, 1><<<nb, kDiagThreads, 0, c.stream>>>(static_cast<const __half*>(mom), c.lay, rows);
    else if (c.storage == LLB_BF16S)
        k_diag_partial<__nv_bfloat16, 1><<<nb, kDiagThreads, 0, c.stream>>>(static_cast<const __nv_bfloat16*>(mom),
                                                                             c.lay, rows);
    else if (c.ncomp == 2) {
        if (c.storage == LLB_F64)
            k_diag_partial<double, 2><<<nb, kDiagThreads, 0, c.stream>>>(static_cast<const double*>(mom), c.lay, rows);
        else
            k_diag_partial<float, 2><<<nb, kDiagThreads, 0, c.stream>>>(static_cast<const float*>(mom), c.lay, rows);
    } else {
        if (c.storage == LLB_F64)
            k_diag_partial<double, 1><<<nb, kDiagThreads, 0, c.stream>>>(static_cast<const double*>(mom), c.lay, rows);
        else
            k_diag_partial<float, 1><<<nb, kDiagThreads, 0, c.stream>>>(static_cast<const float*>(mom), c.lay, rows);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_diag_final<<<1, kDiagThreads, 0, c.stream>>>(rows, nb, c.N, c.ncomp, dev_out);
    return cudaGetLastError();
}

}  // namespace llb

// ---------------------------------------------------------------------------
// Diagnostics without allocation.
//
// Some callers cannot allocate device memory where they need the diagnostics:
// code running while a stream is being captured into a CUDA graph (a
// cudaMalloc there breaks the capture), allocator-owning frameworks and
// real-time loops that forbid allocation on the hot path, and embedders whose
// memory budget is fixed in advance.  For them the reduction below keeps its
// scratch (one row of partial sums per block plus the result) in a
// file-scope device array of fixed size, reserved when the library is loaded
// on a device and held until the process exits.
namespace llb {
namespace {

constexpr int kStaticRows = 4096;                       // partial-sum rows (one per block)
constexpr size_t kStaticNodesPerRow = (size_t)kDiagThreads * 64;
constexpr size_t kStaticMaxNodes = (size_t)kStaticRows * kStaticNodesPerRow;  // 67,108,864 nodes

struct StaticScratch {
    double rows[kStaticRows * kRow];
    llb_diag out;
};

// 288 KB of scratch per device.  Every call on a device reuses it: calls that
// overlap on the GPU (different streams, or different host threads without
// ordering) race on it.  Each call writes every row it later reads and the
// whole result, so no part of it has to be cleared between calls.
static __device__ __align__(256) StaticScratch g_diag_scratch;

// Partial sums of canonical one-component moments (rho, j, P), dense layout:
// block b reduces nodes [b * kStaticNodesPerRow, (b + 1) * kStaticNodesPerRow).
template <class T>
__global__ void __launch_bounds__(kDiagThreads) k_diag_partial_canonical(const T* __restrict__ m, size_t N,
                                                                         double* __restrict__ rows) {
    Part p;
    part_init(p);
    const size_t lo = (size_t)blockIdx.x * kStaticNodesPerRow;
    const size_t hi = lo + kStaticNodesPerRow < N ? lo + kStaticNodesPerRow : N;
    for (size_t i = lo + threadIdx.x; i < hi; i += kDiagThreads) {
        const double rho = (double)m[i];
        const double d = rho - 1.0;
        const double jx = (double)m[N + i], jy = (double)m[2 * N + i], jz = (double)m[3 * N + i];
        p.v[0] += d;
        p.v[1] += jx;
        p.v[2] += jy;
        p.v[3] += jz;
        if (rho > 0.5) {
            p.v[4] += rho;
            p.v[5] += 1.0;
        }
        p.v[6] = fmin(p.v[6], rho);
        bool finite = isfinite(rho) && isfinite(jx) && isfinite(jy) && isfinite(jz);
#pragma unroll
        for (int f = 4; f < 10; ++f) finite = finite && isfinite((double)m[f * N + i]);
        if (!finite) p.v[7] = 1.0;
    }
    p = block_reduce(p);
    if (threadIdx.x == 0)
        for (int k = 0; k < kRow; ++k) rows[(size_t)blockIdx.x * kRow + k] = p.v[k];
}

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
StaticScratch* g_static_ptr[kMaxDevices] = {};

}  // namespace
}  // namespace llb

extern "C" int llb_diagnostics_noalloc(const void* dev_m, int dtype, int nx, int ny, int nz, void* stream,
                                       llb_diag* host_out) {
    using namespace llb;
    if (!dev_m || !host_out || (dtype != LLB_F64 && dtype != LLB_F32) || nx < 1 || ny < 1 || nz < 1)
        return LLB_EINVAL;
    const size_t N = (size_t)nx * ny * nz;
    if (N > kStaticMaxNodes) return LLB_EINVAL;  // more nodes than the fixed scratch can reduce
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return LLB_ECUDA;
    }
    StaticScratch* scratch = nullptr;
    {
        // once per device, with that device current: the device address of the
        // array (its name in host code is only a host-side handle)
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (!g_static_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_diag_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return LLB_ECUDA;
            }
            g_static_ptr[dev] = static_cast<StaticScratch*>(p);
        }
        scratch = g_static_ptr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nb = (int)((N + kStaticNodesPerRow - 1) / kStaticNodesPerRow);
    if (dtype == LLB_F64)
        k_diag_partial_canonical<double><<<nb, kDiagThreads, 0, s>>>(static_cast<const double*>(dev_m), N,
                                                                      scratch->rows);
    else
        k_diag_partial_canonical<float><<<nb, kDiagThreads, 0, s>>>(static_cast<const float*>(dev_m), N,
                                                                     scratch->rows);
    if (cudaGetLastError() != cudaSuccess) return LLB_ECUDA;
    k_diag_final<<<1, kDiagThreads, 0, s>>>(scratch->rows, nb, N, 1, &scratch->out);
    if (cudaGetLastError() != cudaSuccess) return LLB_ECUDA;
    if (cudaMemcpyAsync(host_out, &scratch->out, sizeof(llb_diag), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return LLB_ECUDA;
    }
    return LLB_OK;
}
