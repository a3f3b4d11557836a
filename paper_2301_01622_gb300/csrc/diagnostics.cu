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

#include "internal.h"
#include "lattice.cuh"
#include "layout.cuh"

namespace llb {
namespace {

constexpr int kDiagThreads = 256;
constexpr int kRow = 8;  // sum d, sum jx, sum jy, sum jz, sum rho_in, n_in, min rho, nonfinite

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

template <class T>
__global__ void __launch_bounds__(kDiagThreads) k_diag_partial(const T* __restrict__ m, Layout L,
                                                               double* __restrict__ rows) {
    Part p;
    part_init(p);
    const size_t N = (size_t)L.nx * L.ny * L.nz, F = L.fs;
    for (size_t n = blockIdx.x * (size_t)kDiagThreads + threadIdx.x; n < N; n += (size_t)gridDim.x * kDiagThreads) {
        const int x = (int)(n % L.nx);
        const size_t r = n / L.nx;
        const size_t i = L.at(x, (int)(r % L.ny), (int)(r / L.ny));
        const double d = (double)m[i];
        const double jx = (double)m[F + i], jy = (double)m[2 * F + i], jz = (double)m[3 * F + i];
        const double rho = 1.0 + d;
        p.v[0] += d;
        p.v[1] += jx;
        p.v[2] += jy;
        p.v[3] += jz;
        if (rho > 0.5) {
            p.v[4] += rho;
            p.v[5] += 1.0;
        }
        p.v[6] = fmin(p.v[6], rho);
        bool finite = isfinite(d) && isfinite(jx) && isfinite(jy) && isfinite(jz);
#pragma unroll
        for (int f = 4; f < 10; ++f) finite = finite && isfinite((double)m[f * F + i]);
        if (!finite) p.v[7] = 1.0;
    }
    p = block_reduce(p);
    if (threadIdx.x == 0)
        for (int k = 0; k < kRow; ++k) rows[(size_t)blockIdx.x * kRow + k] = p.v[k];
}

__global__ void __launch_bounds__(kDiagThreads) k_diag_final(const double* __restrict__ rows, int nrows, size_t N,
                                                             llb_diag* __restrict__ out) {
    Part p;
    part_init(p);
    for (int r = threadIdx.x; r < nrows; r += kDiagThreads) {
        Part q;
        for (int k = 0; k < kRow; ++k) q.v[k] = rows[(size_t)r * kRow + k];
        part_merge(p, q);
    }
    p = block_reduce(p);
    if (threadIdx.x == 0) {
        out->mass[0] = (double)N + p.v[0];
        out->mass[1] = 0.0;
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
    if (c.storage == LLB_F64)
        k_diag_partial<double><<<nb, kDiagThreads, 0, c.stream>>>(static_cast<const double*>(mom), c.lay, rows);
    else
        k_diag_partial<float><<<nb, kDiagThreads, 0, c.stream>>>(static_cast<const float*>(mom), c.lay, rows);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_diag_final<<<1, kDiagThreads, 0, c.stream>>>(rows, nb, c.N, dev_out);
    return cudaGetLastError();
}

}  // namespace llb
