// Conversions between the canonical moments of the ABI and the shifted
// device storage, and initialisation at local equilibrium.
//
// canonical (one component): rho, j_x, j_y, j_z, P_xx, P_yy, P_zz, P_xy, P_xz, P_yz
// shifted storage:           d = rho - 1, j, A = P - cs^2 rho I
// Equilibrium (second moment of Eq. eq-part): P^eq = cs^2 rho I + rho u u, so
// A^eq = rho u u.  All conversions compute in FP64 and round once.
#include <cuda_runtime.h>

#include "internal.h"
#include "lattice.cuh"

namespace llb {
namespace {

template <class S>
__device__ __forceinline__ double rd(const void* p, size_t i) {
    return (double)static_cast<const S*>(p)[i];
}

__device__ __forceinline__ double rdt(const void* p, size_t i, int dt) {
    return dt == LLB_F64 ? rd<double>(p, i) : rd<float>(p, i);
}

__device__ __forceinline__ void wrt(void* p, size_t i, int dt, double v) {
    if (dt == LLB_F64) static_cast<double*>(p)[i] = v;
    else static_cast<float*>(p)[i] = (float)v;
}

__device__ __forceinline__ bool bad_rho(double r) { return !(r > 0.0) || !isfinite(r); }

template <class T>
__global__ void k_canon_to_shifted(const void* __restrict__ canon, int cdt, T* __restrict__ st, size_t N,
                                   int* bad) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        double v[10];
#pragma unroll
        for (int f = 0; f < 10; ++f) v[f] = rdt(canon, f * N + i, cdt);
        bool b = bad_rho(v[0]);
#pragma unroll
        for (int f = 1; f < 10; ++f) b = b || !isfinite(v[f]);
        if (b && bad) atomicOr(bad, 1);
        const double rho = v[0];
        st[i] = (T)(rho - 1.0);
        st[N + i] = (T)v[1];
        st[2 * N + i] = (T)v[2];
        st[3 * N + i] = (T)v[3];
        st[4 * N + i] = (T)(v[4] - kCs2 * rho);
        st[5 * N + i] = (T)(v[5] - kCs2 * rho);
        st[6 * N + i] = (T)(v[6] - kCs2 * rho);
        st[7 * N + i] = (T)v[7];
        st[8 * N + i] = (T)v[8];
        st[9 * N + i] = (T)v[9];
    }
}

template <class T>
__global__ void k_shifted_to_canon(const T* __restrict__ st, void* __restrict__ canon, int cdt, size_t N) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const double rho = 1.0 + (double)st[i];
        wrt(canon, i, cdt, rho);
        for (int f = 1; f < 4; ++f) wrt(canon, f * N + i, cdt, (double)st[f * N + i]);
        for (int f = 4; f < 7; ++f) wrt(canon, f * N + i, cdt, (double)st[f * N + i] + kCs2 * rho);
        for (int f = 7; f < 10; ++f) wrt(canon, f * N + i, cdt, (double)st[f * N + i]);
    }
}

template <class T>
__global__ void k_equilibrium(const void* __restrict__ rho_p, const void* __restrict__ u_p, int dt,
                              T* __restrict__ st, size_t N, int* bad) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const double rho = rdt(rho_p, i, dt);
        const double ux = rdt(u_p, i, dt), uy = rdt(u_p, N + i, dt), uz = rdt(u_p, 2 * N + i, dt);
        if ((bad_rho(rho) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz)) && bad) atomicOr(bad, 1);
        st[i] = (T)(rho - 1.0);
        st[N + i] = (T)(rho * ux);
        st[2 * N + i] = (T)(rho * uy);
        st[3 * N + i] = (T)(rho * uz);
        st[4 * N + i] = (T)(rho * ux * ux);
        st[5 * N + i] = (T)(rho * uy * uy);
        st[6 * N + i] = (T)(rho * uz * uz);
        st[7 * N + i] = (T)(rho * ux * uy);
        st[8 * N + i] = (T)(rho * ux * uz);
        st[9 * N + i] = (T)(rho * uy * uz);
    }
}

int grid_for(const llb_ctx& c) {
    const size_t want = (c.N + 255) / 256;
    const size_t cap = (size_t)(c.num_sms > 0 ? c.num_sms : 148) * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_canonical_to_shifted(const llb_ctx& c, const void* canon, int cdt, void* st, int* bad) {
    if (c.storage == LLB_F64)
        k_canon_to_shifted<double><<<grid_for(c), 256, 0, c.stream>>>(canon, cdt, static_cast<double*>(st), c.N, bad);
    else
        k_canon_to_shifted<float><<<grid_for(c), 256, 0, c.stream>>>(canon, cdt, static_cast<float*>(st), c.N, bad);
    return cudaGetLastError();
}

cudaError_t launch_shifted_to_canonical(const llb_ctx& c, const void* st, void* canon, int cdt) {
    if (c.storage == LLB_F64)
        k_shifted_to_canon<double><<<grid_for(c), 256, 0, c.stream>>>(static_cast<const double*>(st), canon, cdt, c.N);
    else
        k_shifted_to_canon<float><<<grid_for(c), 256, 0, c.stream>>>(static_cast<const float*>(st), canon, cdt, c.N);
    return cudaGetLastError();
}

cudaError_t launch_equilibrium(const llb_ctx& c, const void* rho, const void* u, int dt, void* st, int* bad) {
    if (c.storage == LLB_F64)
        k_equilibrium<double><<<grid_for(c), 256, 0, c.stream>>>(rho, u, dt, static_cast<double*>(st), c.N, bad);
    else
        k_equilibrium<float><<<grid_for(c), 256, 0, c.stream>>>(rho, u, dt, static_cast<float*>(st), c.N, bad);
    return cudaGetLastError();
}

}  // namespace llb
