// Conversions between the canonical moments of the ABI and the shifted
// device storage, and initialisation at local equilibrium.
//
// canonical (one component): rho, j_x, j_y, j_z, P_xx, P_yy, P_zz, P_xy, P_xz, P_yz
// shifted storage:           d = rho - 1, j, A = P - cs^2 rho I
// Equilibrium (second moment of Eq. (5)): P^eq = cs^2 rho I + rho u u, so
// A^eq = rho u u.  All conversions compute in FP64 and round once.
// Two components: canonical rho1, rho2, j, P; state rho1, d = rho1 + rho2 - 1,
// j, A (rho1 needs no shift: it lies in [0, rho]).
// Canonical buffers are dense; the shifted state follows the context's
// Layout (padded with periodic ghosts for the moment scheme), and every
// write to it also writes the node's ghost copies.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "lattice.cuh"
#include "layout.cuh"
#include "storage.cuh"

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

__device__ __forceinline__ void decode(const Layout& L, size_t i, int& x, int& y, int& z) {
    x = (int)(i % L.nx);
    const size_t r = i / L.nx;
    y = (int)(r % L.ny);
    z = (int)(r / L.ny);
}

template <class T>
__device__ __forceinline__ void put(T* __restrict__ st, const Layout& L, int x, int y, int z, const double* v) {
    for_node_and_ghosts(L, x, y, [&](int gx, int gy) {
        const size_t j = L.at(gx, gy, z);
#pragma unroll
        for (int f = 0; f < 10; ++f) st[FieldMap<T, 10>::at(j, f, L.fs)] = to_store<T>(v[f], f);
    });
}

// Nodes i0 .. i1-1 of the dense canonical order (whole planes for a z-range).
template <class T>
__global__ void k_canon_to_shifted(const void* __restrict__ canon, int cdt, T* __restrict__ st, Layout L,
                                   int* bad, size_t i0, size_t i1) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    for (size_t i = i0 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < i1; i += (size_t)gridDim.x * blockDim.x) {
        double v[10];
#pragma unroll
        for (int f = 0; f < 10; ++f) v[f] = rdt(canon, f * N + i, cdt);
        bool b = bad_rho(v[0]);
#pragma unroll
        for (int f = 1; f < 10; ++f) b = b || !isfinite(v[f]);
        if (b && bad) atomicOr(bad, 1);
        const double rho = v[0];
        const double o[10] = {rho - 1.0, v[1], v[2], v[3], v[4] - kCs2 * rho, v[5] - kCs2 * rho,
                              v[6] - kCs2 * rho, v[7], v[8], v[9]};
        int x, y, z;
        decode(L, i, x, y, z);
        put(st, L, x, y, z, o);
    }
}

template <class T>
__global__ void k_shifted_to_canon(const T* __restrict__ st, void* __restrict__ canon, int cdt, Layout L, size_t i0,
                                   size_t i1) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    for (size_t i = i0 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < i1; i += (size_t)gridDim.x * blockDim.x) {
        int x, y, z;
        decode(L, i, x, y, z);
        const size_t j = L.at(x, y, z);
        using FM = FieldMap<T, 10>;
        const double rho = 1.0 + rd_field(st[FM::at(j, 0, L.fs)], 0);
        wrt(canon, i, cdt, rho);
        for (int f = 1; f < 4; ++f) wrt(canon, f * N + i, cdt, rd_field(st[FM::at(j, f, L.fs)], f));
        for (int f = 4; f < 7; ++f) wrt(canon, f * N + i, cdt, rd_field(st[FM::at(j, f, L.fs)], f) + kCs2 * rho);
        for (int f = 7; f < 10; ++f) wrt(canon, f * N + i, cdt, rd_field(st[FM::at(j, f, L.fs)], f));
    }
}

template <class T>
__global__ void k_equilibrium(const void* __restrict__ rho_p, const void* __restrict__ u_p, int dt,
                              T* __restrict__ st, Layout L, int* bad) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const double rho = rdt(rho_p, i, dt);
        const double ux = rdt(u_p, i, dt), uy = rdt(u_p, N + i, dt), uz = rdt(u_p, 2 * N + i, dt);
        if ((bad_rho(rho) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz)) && bad) atomicOr(bad, 1);
        const double o[10] = {rho - 1.0, rho * ux, rho * uy, rho * uz, rho * ux * ux, rho * uy * uy,
                              rho * uz * uz, rho * ux * uy, rho * ux * uz, rho * uy * uz};
        int x, y, z;
        decode(L, i, x, y, z);
        put(st, L, x, y, z, o);
    }
}

// Two components.  canonical: rho1, rho2, j (3), P (6); state: rho1, d = rho1 + rho2 - 1,
// j (3), A = P - cs^2 rho I (6).
template <class T>
__device__ __forceinline__ void put11(T* __restrict__ st, const Layout& L, int x, int y, int z, const double* v) {
    for_node_and_ghosts(L, x, y, [&](int gx, int gy) {
        const size_t j = L.at(gx, gy, z);
#pragma unroll
        for (int f = 0; f < 11; ++f) st[f * L.fs + j] = (T)v[f];
    });
}

template <class T>
__global__ void k_canon_to_shifted2(const void* __restrict__ canon, int cdt, T* __restrict__ st, Layout L,
                                    int* bad, size_t i0, size_t i1) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    for (size_t i = i0 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < i1; i += (size_t)gridDim.x * blockDim.x) {
        double v[11];
#pragma unroll
        for (int f = 0; f < 11; ++f) v[f] = rdt(canon, f * N + i, cdt);
        const double rho = v[0] + v[1];
        // the total density must be positive; a colour density may dip slightly
        // below zero (the stepped colour-gradient field does so near interfaces)
        bool b = bad_rho(rho) || !isfinite(v[0]) || !isfinite(v[1]);
#pragma unroll
        for (int f = 2; f < 11; ++f) b = b || !isfinite(v[f]);
        if (b && bad) atomicOr(bad, 1);
        const double o[11] = {v[0], rho - 1.0, v[2], v[3], v[4], v[5] - kCs2 * rho, v[6] - kCs2 * rho,
                              v[7] - kCs2 * rho, v[8], v[9], v[10]};
        int x, y, z;
        decode(L, i, x, y, z);
        put11(st, L, x, y, z, o);
    }
}

template <class T>
__global__ void k_shifted_to_canon2(const T* __restrict__ st, void* __restrict__ canon, int cdt, Layout L, size_t i0,
                                    size_t i1) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    for (size_t i = i0 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < i1; i += (size_t)gridDim.x * blockDim.x) {
        int x, y, z;
        decode(L, i, x, y, z);
        const size_t j = L.at(x, y, z);
        const double r1 = (double)st[j];
        const double rho = 1.0 + (double)st[L.fs + j];
        wrt(canon, i, cdt, r1);
        wrt(canon, N + i, cdt, rho - r1);
        for (int f = 2; f < 5; ++f) wrt(canon, f * N + i, cdt, (double)st[f * L.fs + j]);
        for (int f = 5; f < 8; ++f) wrt(canon, f * N + i, cdt, (double)st[f * L.fs + j] + kCs2 * rho);
        for (int f = 8; f < 11; ++f) wrt(canon, f * N + i, cdt, (double)st[f * L.fs + j]);
    }
}

template <class T>
__global__ void k_equilibrium2(const void* __restrict__ rho_p, const void* __restrict__ u_p, int dt,
                               T* __restrict__ st, Layout L, int* bad) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const double r1 = rdt(rho_p, i, dt), r2 = rdt(rho_p, N + i, dt);
        const double rho = r1 + r2;
        const double ux = rdt(u_p, i, dt), uy = rdt(u_p, N + i, dt), uz = rdt(u_p, 2 * N + i, dt);
        if ((bad_rho(rho) || !isfinite(r1) || !isfinite(r2) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz)) && bad)
            atomicOr(bad, 1);
        const double o[11] = {r1, rho - 1.0, rho * ux, rho * uy, rho * uz, rho * ux * ux, rho * uy * uy,
                              rho * uz * uz, rho * ux * uy, rho * ux * uz, rho * uy * uz};
        int x, y, z;
        decode(L, i, x, y, z);
        put11(st, L, x, y, z, o);
    }
}

int grid_for(const llb_ctx& c) {
    const size_t want = (c.N + 255) / 256;
    const size_t cap = (size_t)(c.num_sms > 0 ? c.num_sms : 148) * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace

cudaError_t launch_canonical_to_shifted(const llb_ctx& c, const void* canon, int cdt, void* st, int* bad) {
    if (c.storage == LLB_F16S) {
        k_canon_to_shifted<__half><<<grid_for(c), 256, 0, c.stream>>>(canon, cdt, static_cast<__half*>(st), c.lay, bad, 0, c.N);
        return cudaGetLastError();
    }
    if (c.storage == LLB_BF16S) {
        k_canon_to_shifted<__nv_bfloat16><<<grid_for(c), 256, 0, c.stream>>>(canon, cdt, static_cast<__nv_bfloat16*>(st),
                                                                             c.lay, bad, 0, c.N);
        return cudaGetLastError();
    }
    if (c.ncomp == 2) {
        if (c.storage == LLB_F64)
            k_canon_to_shifted2<double><<<grid_for(c), 256, 0, c.stream>>>(canon, cdt, static_cast<double*>(st), c.lay, bad,
                                                                            0, c.N);
        else
            k_canon_to_shifted2<float><<<grid_for(c), 256, 0, c.stream>>>(canon, cdt, static_cast<float*>(st), c.lay, bad,
                                                                           0, c.N);
        return cudaGetLastError();
    }
    if (c.storage == LLB_F64)
        k_canon_to_shifted<double><<<grid_for(c), 256, 0, c.stream>>>(canon, cdt, static_cast<double*>(st), c.lay, bad,
                                                                       0, c.N);
    else
        k_canon_to_shifted<float><<<grid_for(c), 256, 0, c.stream>>>(canon, cdt, static_cast<float*>(st), c.lay, bad,
                                                                      0, c.N);
    return cudaGetLastError();
}

cudaError_t launch_shifted_to_canonical(const llb_ctx& c, const void* st, void* canon, int cdt) {
    if (c.storage == LLB_F16S) {
        k_shifted_to_canon<__half><<<grid_for(c), 256, 0, c.stream>>>(static_cast<const __half*>(st), canon, cdt, c.lay, 0, c.N);
        return cudaGetLastError();
    }
    if (c.storage == LLB_BF16S) {
        k_shifted_to_canon<__nv_bfloat16><<<grid_for(c), 256, 0, c.stream>>>(static_cast<const __nv_bfloat16*>(st), canon,
                                                                             cdt, c.lay, 0, c.N);
        return cudaGetLastError();
    }
    if (c.ncomp == 2) {
        if (c.storage == LLB_F64)
            k_shifted_to_canon2<double><<<grid_for(c), 256, 0, c.stream>>>(static_cast<const double*>(st), canon, cdt, c.lay,
                                                                            0, c.N);
        else
            k_shifted_to_canon2<float><<<grid_for(c), 256, 0, c.stream>>>(static_cast<const float*>(st), canon, cdt, c.lay,
                                                                           0, c.N);
        return cudaGetLastError();
    }
    if (c.storage == LLB_F64)
        k_shifted_to_canon<double><<<grid_for(c), 256, 0, c.stream>>>(static_cast<const double*>(st), canon, cdt, c.lay,
                                                                       0, c.N);
    else
        k_shifted_to_canon<float><<<grid_for(c), 256, 0, c.stream>>>(static_cast<const float*>(st), canon, cdt, c.lay,
                                                                      0, c.N);
    return cudaGetLastError();
}

cudaError_t launch_canonical_to_shifted_range(const llb_ctx& c, const void* canon, int cdt, void* st, int* bad, int zlo,
                                              int zhi, cudaStream_t s) {
    const size_t per = (size_t)c.nx * c.ny, i0 = per * zlo, i1 = per * zhi;
    const int grid = (int)std::min<size_t>((i1 - i0 + 255) / 256, (size_t)c.num_sms * 8);
    if (c.ncomp == 2) {
        if (c.storage == LLB_F64)
            k_canon_to_shifted2<double><<<grid, 256, 0, s>>>(canon, cdt, static_cast<double*>(st), c.lay, bad, i0, i1);
        else
            k_canon_to_shifted2<float><<<grid, 256, 0, s>>>(canon, cdt, static_cast<float*>(st), c.lay, bad, i0, i1);
        return cudaGetLastError();
    }
    switch (c.storage) {
        case LLB_F64:
            k_canon_to_shifted<double><<<grid, 256, 0, s>>>(canon, cdt, static_cast<double*>(st), c.lay, bad, i0, i1);
            break;
        case LLB_F16S:
            k_canon_to_shifted<__half><<<grid, 256, 0, s>>>(canon, cdt, static_cast<__half*>(st), c.lay, bad, i0, i1);
            break;
        case LLB_BF16S:
            k_canon_to_shifted<__nv_bfloat16><<<grid, 256, 0, s>>>(canon, cdt, static_cast<__nv_bfloat16*>(st), c.lay,
                                                                  bad, i0, i1);
            break;
        default:
            k_canon_to_shifted<float><<<grid, 256, 0, s>>>(canon, cdt, static_cast<float*>(st), c.lay, bad, i0, i1);
    }
    return cudaGetLastError();
}

cudaError_t launch_shifted_to_canonical_range(const llb_ctx& c, const void* st, void* canon, int cdt, int zlo, int zhi,
                                              cudaStream_t s) {
    const size_t per = (size_t)c.nx * c.ny, i0 = per * zlo, i1 = per * zhi;
    const int grid = (int)std::min<size_t>((i1 - i0 + 255) / 256, (size_t)c.num_sms * 8);
    if (c.ncomp == 2) {
        if (c.storage == LLB_F64)
            k_shifted_to_canon2<double><<<grid, 256, 0, s>>>(static_cast<const double*>(st), canon, cdt, c.lay, i0, i1);
        else
            k_shifted_to_canon2<float><<<grid, 256, 0, s>>>(static_cast<const float*>(st), canon, cdt, c.lay, i0, i1);
        return cudaGetLastError();
    }
    switch (c.storage) {
        case LLB_F64:
            k_shifted_to_canon<double><<<grid, 256, 0, s>>>(static_cast<const double*>(st), canon, cdt, c.lay, i0, i1);
            break;
        case LLB_F16S:
            k_shifted_to_canon<__half><<<grid, 256, 0, s>>>(static_cast<const __half*>(st), canon, cdt, c.lay, i0, i1);
            break;
        case LLB_BF16S:
            k_shifted_to_canon<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(st), canon, cdt,
                                                                  c.lay, i0, i1);
            break;
        default:
            k_shifted_to_canon<float><<<grid, 256, 0, s>>>(static_cast<const float*>(st), canon, cdt, c.lay, i0, i1);
    }
    return cudaGetLastError();
}

cudaError_t launch_equilibrium(const llb_ctx& c, const void* rho, const void* u, int dt, void* st, int* bad) {
    if (c.storage == LLB_F16S) {
        k_equilibrium<__half><<<grid_for(c), 256, 0, c.stream>>>(rho, u, dt, static_cast<__half*>(st), c.lay, bad);
        return cudaGetLastError();
    }
    if (c.storage == LLB_BF16S) {
        k_equilibrium<__nv_bfloat16><<<grid_for(c), 256, 0, c.stream>>>(rho, u, dt, static_cast<__nv_bfloat16*>(st),
                                                                        c.lay, bad);
        return cudaGetLastError();
    }
    if (c.ncomp == 2) {
        if (c.storage == LLB_F64)
            k_equilibrium2<double><<<grid_for(c), 256, 0, c.stream>>>(rho, u, dt, static_cast<double*>(st), c.lay, bad);
        else
            k_equilibrium2<float><<<grid_for(c), 256, 0, c.stream>>>(rho, u, dt, static_cast<float*>(st), c.lay, bad);
        return cudaGetLastError();
    }
    if (c.storage == LLB_F64)
        k_equilibrium<double><<<grid_for(c), 256, 0, c.stream>>>(rho, u, dt, static_cast<double*>(st), c.lay, bad);
    else
        k_equilibrium<float><<<grid_for(c), 256, 0, c.stream>>>(rho, u, dt, static_cast<float*>(st), c.lay, bad);
    return cudaGetLastError();
}

}  // namespace llb
