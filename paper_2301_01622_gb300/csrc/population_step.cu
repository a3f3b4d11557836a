// Population-storing lattice Boltzmann baselines (one component).
//
// These keep all Q populations per node in global memory, the layout the
// paper compares the moment-only method against (Sec. III A: 38 arrays for
// D3Q19 in the flip-flop scheme; Sec. IV A: the "standard" LB with
// populations).  Each kernel is the usual one-thread-per-node pull step:
// read f_i(x - c_i) (post-collision values of the previous step), project
// to moments (Eqs. (1)-(3)), collide, write the Q post-collision values at x.
//   regularized: f'_i = h^eq_i + (1 - omega) h^neq_i from the moments (Eq. (8)),
//                the same map as the moment-only step;
//   BGK:         f'_i = (1 - omega) f_i + omega h^eq_i (Eq. (7) on the stored f_i),
//                which keeps the ghost components.
// The state holds shifted values g_i = f_i - w_i in a dense [Q][N] layout;
// direction k runs over (cz, cy, cx) in {-1,0,1}^3 in that loop order,
// skipping absent vectors.  Moment temporaries follow the context's Layout.
//
// Two components (the colour-gradient LB with populations of Sec. IV, the
// paper's "standard CGLB" of Sec. IV A): the state holds the shifted total
// populations g_i and the colour-1 populations f1_i, [2Q][N]; the colour-2
// populations are w_i + g_i - f1_i.  One step is two kernels, the split
// approach of Sec. III A: k_pop2_phase pulls both sets and writes the phase
// field phi = (rho1 - rho2)/rho of every node; k_pop2_step pulls them again,
// takes the gradient of phi from the 26 neighbours, collides (regularized:
// the Hermite-2 reconstruction of the collided moments, the same map as the
// moment-only step; BGK: Eq. (7) on the stored populations, ghosts kept) with
// the same forcing, perturbation and recolouring as the moment-only
// two-component kernel, and writes both sets.
#include <cuda_runtime.h>

#include "cg_kernel.cuh"
#include "internal.h"
#include "lattice.cuh"

namespace llb {
namespace {

// Ten shifted moments of node idx in a moment buffer of NF fields (10: the
// one-component state, whose field order follows FieldMap; 11: the
// two-component state, field-major, read from its field 1 on).
template <int NF, class T>
__device__ __forceinline__ Mom<T> load_mom(const T* __restrict__ p, size_t idx, size_t N) {
    using FM = FieldMap<T, NF>;
    Mom<T> m;
    m.d = p[FM::at(idx, 0, N)]; m.jx = p[FM::at(idx, 1, N)]; m.jy = p[FM::at(idx, 2, N)];
    m.jz = p[FM::at(idx, 3, N)]; m.axx = p[FM::at(idx, 4, N)]; m.ayy = p[FM::at(idx, 5, N)];
    m.azz = p[FM::at(idx, 6, N)]; m.axy = p[FM::at(idx, 7, N)]; m.axz = p[FM::at(idx, 8, N)];
    m.ayz = p[FM::at(idx, 9, N)];
    return m;
}

template <int NF, class T>
__device__ __forceinline__ void store_mom(T* __restrict__ p, size_t idx, size_t N, const Mom<T>& m) {
    using FM = FieldMap<T, NF>;
    p[FM::at(idx, 0, N)] = m.d; p[FM::at(idx, 1, N)] = m.jx; p[FM::at(idx, 2, N)] = m.jy;
    p[FM::at(idx, 3, N)] = m.jz; p[FM::at(idx, 4, N)] = m.axx; p[FM::at(idx, 5, N)] = m.ayy;
    p[FM::at(idx, 6, N)] = m.azz; p[FM::at(idx, 7, N)] = m.axy; p[FM::at(idx, 8, N)] = m.axz;
    p[FM::at(idx, 9, N)] = m.ayz;
}

template <class L, class T, bool BGK>
__global__ void __launch_bounds__(128) k_pop_step(const T* __restrict__ in, T* __restrict__ out, int nx, int ny,
                                                  int nz, size_t N, T omega) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const size_t idx = LLB_CLAMP(((size_t)z * ny + y) * nx + x, N, kChkPop);
    T g[L::Q];
    Acc<T> acc;
    acc.zero();
    int k = 0;
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz)) continue;
                const size_t s = LLB_CLAMP(((size_t)wrap_idx(z - cz, nz) * ny + wrap_idx(y - cy, ny)) * nx + wrap_idx(x - cx, nx), N, kChkPop);
                g[k] = in[(size_t)k * N + s];
                acc.add(g[k], cx, cy, cz);
                ++k;
            }
    const Mom<T> m = acc.finish();
    // regularized: collided moments; BGK: the equilibrium (omega = 1 collision)
    const Mom<T> c = BGK ? collide(m, T(1)) : collide(m, omega);
    const T s0 = g_shared(c);
    k = 0;
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz)) continue;
                const T ge = g_dir<L, T>(c, s0, cx, cy, cz);
                out[(size_t)k * N + idx] = BGK ? (T(1) - omega) * g[k] + omega * ge : ge;
                ++k;
            }
}

// state_k(x) = g^R_k(m(x + c_k)): the population that a pull at x + c_k will read.
template <class L, class T>
__global__ void k_pop_from_moments(const T* __restrict__ mom, T* __restrict__ st, int nx, int ny, int nz,
                                   size_t N, Layout lay) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const size_t idx = LLB_CLAMP(((size_t)z * ny + y) * nx + x, N, kChkPop);
    int k = 0;
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz)) continue;
                const size_t s = LLB_CLAMP(lay.at(wrap_idx(x + cx, nx), wrap_idx(y + cy, ny), wrap_idx(z + cz, nz)), lay.fs, kChkLoad);
                const Mom<T> m = load_mom<10>(mom, s, lay.fs);
                st[(size_t)k * N + idx] = g_dir<L, T>(m, g_shared(m), cx, cy, cz);
                ++k;
            }
}

template <class L, class T>
__global__ void k_moments_from_pop(const T* __restrict__ st, T* __restrict__ mom, int nx, int ny, int nz,
                                   size_t N, Layout lay) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    Acc<T> acc;
    acc.zero();
    int k = 0;
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz)) continue;
                const size_t s = LLB_CLAMP(((size_t)wrap_idx(z - cz, nz) * ny + wrap_idx(y - cy, ny)) * nx + wrap_idx(x - cx, nx), N, kChkPop);
                acc.add(st[(size_t)k * N + s], cx, cy, cz);
                ++k;
            }
    store_mom<10>(mom, LLB_CLAMP(lay.at(x, y, z), lay.fs, kChkStore), lay.fs, acc.finish());
}

// ---------------------------------------------------------------------------
// Two components.

// phi(x) = 2 rho1 / rho - 1 from the pulled populations of both sets.
template <class L, class T>
__global__ void __launch_bounds__(128) k_pop2_phase(const T* __restrict__ in, T* __restrict__ phi, int nx, int ny,
                                                    int nz, size_t N) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    T d = T(0), r1 = T(0);
    int k = 0;
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz)) continue;
                const size_t s = LLB_CLAMP(((size_t)wrap_idx(z - cz, nz) * ny + wrap_idx(y - cy, ny)) * nx + wrap_idx(x - cx, nx), N, kChkPop);
                d += in[(size_t)k * N + s];
                r1 += in[(size_t)(L::Q + k) * N + s];
                ++k;
            }
    phi[LLB_CLAMP(((size_t)z * ny + y) * nx + x, N, kChkPhi)] = T(2) * r1 / (T(1) + d) - T(1);
}

template <class L, class T, bool BGK>
__global__ void __launch_bounds__(128) k_pop2_step(const T* __restrict__ in, T* __restrict__ out,
                                                   const T* __restrict__ phi, int nx, int ny, int nz, size_t N,
                                                   cg::CGPar<T> prm) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const size_t idx = LLB_CLAMP(((size_t)z * ny + y) * nx + x, N, kChkPop);
    T g[L::Q];
    Acc<T> acc;
    acc.zero();
    T r1 = T(0);
    int k = 0;
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz)) continue;
                const size_t s = LLB_CLAMP(((size_t)wrap_idx(z - cz, nz) * ny + wrap_idx(y - cy, ny)) * nx + wrap_idx(x - cx, nx), N, kChkPop);
                g[k] = in[(size_t)k * N + s];
                r1 += in[(size_t)(L::Q + k) * N + s];
                acc.add(g[k], cx, cy, cz);
                ++k;
            }
    cg::Node2<T> a;
    a.r1 = r1;
    a.m = acc.finish();
    // isotropic gradient of phi from the neighbours: (1/cs^2) sum_k w_k c_k phi(x + c_k)
    T Gx = T(0), Gy = T(0), Gz = T(0);
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz) || (cx == 0 && cy == 0 && cz == 0)) continue;
                const T v = phi[LLB_CLAMP(((size_t)wrap_idx(z + cz, nz) * ny + wrap_idx(y + cy, ny)) * nx + wrap_idx(x + cx, nx), N, kChkPhi)];
                const T wv = T(3.0 * L::w(cx, cy, cz)) * v;
                if (cx) Gx += T(cx) * wv;
                if (cy) Gy += T(cy) * wv;
                if (cz) Gz += T(cz) * wv;
            }
    const cg::Src2<T> s = cg::cg_collide<T, false>(a, Gx, Gy, Gz, phi[idx], prm, [&](int ox, int oy, int oz) {
        const int px = cg::pmod2(x + ox, nx), py = cg::pmod2(y + oy, ny), pz = cg::pmod2(z + oz, nz);
        return phi[LLB_CLAMP(((size_t)pz * ny + py) * nx + px, N, kChkProbe)];
    });
    const T s0c = g_shared(s.c), s0m = g_shared(a.m);
    const T one_m = T(1) - prm.omega;
    k = 0;
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz)) continue;
                T gp = g_dir<L, T>(s.c, s0c, cx, cy, cz);
                // BGK keeps the stored non-hydrodynamic part: + (1 - omega)(f_i - R_i(m))
                if (BGK) gp += one_m * (g[k] - g_dir<L, T>(a.m, s0m, cx, cy, cz));
                const T w = T(L::w(cx, cy, cz));
                T h1 = s.r1 * (w + gp);
                if (cx || cy || cz)
                    h1 += s.e * T(L::w(cx, cy, cz) * cg::inv_len(cx, cy, cz)) *
                          (T(cx) * s.nx + T(cy) * s.ny + T(cz) * s.nz);
                out[(size_t)k * N + idx] = gp;
                out[(size_t)(L::Q + k) * N + idx] = h1;
                ++k;
            }
}

// state_k(x) = g^R_k(m(x + c_k)), state_{Q+k}(x) = (rho1/rho)(w_k + g^R_k)(x + c_k):
// the colour populations f = R(m) split by the colour fractions.
template <class L, class T>
__global__ void k_pop2_from_moments(const T* __restrict__ mom, T* __restrict__ st, int nx, int ny, int nz,
                                    size_t N, Layout lay) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const size_t idx = LLB_CLAMP(((size_t)z * ny + y) * nx + x, N, kChkPop);
    int k = 0;
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz)) continue;
                const size_t s = LLB_CLAMP(lay.at(wrap_idx(x + cx, nx), wrap_idx(y + cy, ny), wrap_idx(z + cz, nz)), lay.fs, kChkLoad);
                const T r1 = mom[s];
                const Mom<T> m = load_mom<11>(mom + lay.fs, s, lay.fs);
                const T gr = g_dir<L, T>(m, g_shared(m), cx, cy, cz);
                st[(size_t)k * N + idx] = gr;
                st[(size_t)(L::Q + k) * N + idx] = r1 / (T(1) + m.d) * (T(L::w(cx, cy, cz)) + gr);
                ++k;
            }
}

template <class L, class T>
__global__ void k_moments2_from_pop(const T* __restrict__ st, T* __restrict__ mom, int nx, int ny, int nz,
                                    size_t N, Layout lay) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    Acc<T> acc;
    acc.zero();
    T r1 = T(0);
    int k = 0;
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz)) continue;
                const size_t s = LLB_CLAMP(((size_t)wrap_idx(z - cz, nz) * ny + wrap_idx(y - cy, ny)) * nx + wrap_idx(x - cx, nx), N, kChkPop);
                acc.add(st[(size_t)k * N + s], cx, cy, cz);
                r1 += st[(size_t)(L::Q + k) * N + s];
                ++k;
            }
    const size_t i = LLB_CLAMP(lay.at(x, y, z), lay.fs, kChkStore);
    mom[i] = r1;
    store_mom<11>(mom + lay.fs, i, lay.fs, acc.finish());
}

dim3 node_grid(const llb_ctx& c) { return dim3((c.nx + 127) / 128, c.ny, c.nz); }

template <class T>
cg::CGPar<T> pop2_params(const llb_ctx& c) {
    cg::CGPar<T> p;
    p.omega = (T)c.omega;
    p.beta = (T)c.params.beta;
    p.A_s = (T)c.params.A_s;
    p.A_h = (T)c.params.A_h;
    p.g_min = (T)c.params.g_min;
    p.g_nci = (T)cg::kGNci;
    p.eps2 = (T)(c.params.grad_eps * c.params.grad_eps);
    p.h_c = c.params.h_c;
    return p;
}

template <class L, class T>
cudaError_t step_t(const llb_ctx& c, const void* in, void* out, bool bgk) {
    if (c.ncomp == 2) {
        T* phi = static_cast<T*>(c.phi_scratch);
        k_pop2_phase<L, T><<<node_grid(c), 128, 0, c.stream>>>(static_cast<const T*>(in), phi, c.nx, c.ny, c.nz,
                                                               c.N);
        if (bgk)
            k_pop2_step<L, T, true><<<node_grid(c), 128, 0, c.stream>>>(
                static_cast<const T*>(in), static_cast<T*>(out), phi, c.nx, c.ny, c.nz, c.N, pop2_params<T>(c));
        else
            k_pop2_step<L, T, false><<<node_grid(c), 128, 0, c.stream>>>(
                static_cast<const T*>(in), static_cast<T*>(out), phi, c.nx, c.ny, c.nz, c.N, pop2_params<T>(c));
        return cudaGetLastError();
    }
    if (bgk)
        k_pop_step<L, T, true><<<node_grid(c), 128, 0, c.stream>>>(static_cast<const T*>(in), static_cast<T*>(out),
                                                                   c.nx, c.ny, c.nz, c.N, (T)c.omega);
    else
        k_pop_step<L, T, false><<<node_grid(c), 128, 0, c.stream>>>(static_cast<const T*>(in), static_cast<T*>(out),
                                                                    c.nx, c.ny, c.nz, c.N, (T)c.omega);
    return cudaGetLastError();
}

template <class L, class T>
cudaError_t from_mom_t(const llb_ctx& c, const void* mom, void* st) {
    if (c.ncomp == 2) {
        k_pop2_from_moments<L, T><<<node_grid(c), 128, 0, c.stream>>>(static_cast<const T*>(mom),
                                                                       static_cast<T*>(st), c.nx, c.ny, c.nz, c.N,
                                                                       c.lay);
        return cudaGetLastError();
    }
    k_pop_from_moments<L, T><<<node_grid(c), 128, 0, c.stream>>>(static_cast<const T*>(mom), static_cast<T*>(st),
                                                                  c.nx, c.ny, c.nz, c.N, c.lay);
    return cudaGetLastError();
}

template <class L, class T>
cudaError_t to_mom_t(const llb_ctx& c, const void* st, void* mom) {
    if (c.ncomp == 2) {
        k_moments2_from_pop<L, T><<<node_grid(c), 128, 0, c.stream>>>(static_cast<const T*>(st),
                                                                       static_cast<T*>(mom), c.nx, c.ny, c.nz, c.N,
                                                                       c.lay);
        return cudaGetLastError();
    }
    k_moments_from_pop<L, T><<<node_grid(c), 128, 0, c.stream>>>(static_cast<const T*>(st), static_cast<T*>(mom),
                                                                  c.nx, c.ny, c.nz, c.N, c.lay);
    return cudaGetLastError();
}

}  // namespace

#define LLB_DISPATCH(fn, ...)                                                                   \
    (c.Q == 19 ? (c.storage == LLB_F64 ? fn<D3Q19, double>(__VA_ARGS__) : fn<D3Q19, float>(__VA_ARGS__)) \
               : (c.storage == LLB_F64 ? fn<D3Q27, double>(__VA_ARGS__) : fn<D3Q27, float>(__VA_ARGS__)))

cudaError_t launch_population_step(const llb_ctx& c, const void* in, void* out, bool bgk) {
    return LLB_DISPATCH(step_t, c, in, out, bgk);
}

cudaError_t launch_population_from_moments(const llb_ctx& c, const void* mom, void* state) {
    return LLB_DISPATCH(from_mom_t, c, mom, state);
}

cudaError_t launch_moments_from_population(const llb_ctx& c, const void* state, void* mom) {
    return LLB_DISPATCH(to_mom_t, c, state, mom);
}

LLB_CHK_TU(pop)

}  // namespace llb
