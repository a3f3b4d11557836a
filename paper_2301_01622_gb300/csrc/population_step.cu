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
#include <cuda_runtime.h>

#include "internal.h"
#include "lattice.cuh"

namespace llb {
namespace {

template <class T>
__device__ __forceinline__ Mom<T> load_mom(const T* __restrict__ p, size_t idx, size_t N) {
    Mom<T> m;
    m.d = p[idx]; m.jx = p[N + idx]; m.jy = p[2 * N + idx]; m.jz = p[3 * N + idx];
    m.axx = p[4 * N + idx]; m.ayy = p[5 * N + idx]; m.azz = p[6 * N + idx];
    m.axy = p[7 * N + idx]; m.axz = p[8 * N + idx]; m.ayz = p[9 * N + idx];
    return m;
}

template <class T>
__device__ __forceinline__ void store_mom(T* __restrict__ p, size_t idx, size_t N, const Mom<T>& m) {
    p[idx] = m.d; p[N + idx] = m.jx; p[2 * N + idx] = m.jy; p[3 * N + idx] = m.jz;
    p[4 * N + idx] = m.axx; p[5 * N + idx] = m.ayy; p[6 * N + idx] = m.azz;
    p[7 * N + idx] = m.axy; p[8 * N + idx] = m.axz; p[9 * N + idx] = m.ayz;
}

template <class L, class T, bool BGK>
__global__ void __launch_bounds__(128) k_pop_step(const T* __restrict__ in, T* __restrict__ out, int nx, int ny,
                                                  int nz, size_t N, T omega) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= nx) return;
    const size_t idx = ((size_t)z * ny + y) * nx + x;
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
                const size_t s = ((size_t)wrap_idx(z - cz, nz) * ny + wrap_idx(y - cy, ny)) * nx + wrap_idx(x - cx, nx);
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
    const size_t idx = ((size_t)z * ny + y) * nx + x;
    int k = 0;
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz)) continue;
                const size_t s = lay.at(wrap_idx(x + cx, nx), wrap_idx(y + cy, ny), wrap_idx(z + cz, nz));
                const Mom<T> m = load_mom(mom, s, lay.fs);
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
                const size_t s = ((size_t)wrap_idx(z - cz, nz) * ny + wrap_idx(y - cy, ny)) * nx + wrap_idx(x - cx, nx);
                acc.add(st[(size_t)k * N + s], cx, cy, cz);
                ++k;
            }
    store_mom(mom, lay.at(x, y, z), lay.fs, acc.finish());
}

dim3 node_grid(const llb_ctx& c) { return dim3((c.nx + 127) / 128, c.ny, c.nz); }

template <class L, class T>
cudaError_t step_t(const llb_ctx& c, const void* in, void* out, bool bgk) {
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
    k_pop_from_moments<L, T><<<node_grid(c), 128, 0, c.stream>>>(static_cast<const T*>(mom), static_cast<T*>(st),
                                                                  c.nx, c.ny, c.nz, c.N, c.lay);
    return cudaGetLastError();
}

template <class L, class T>
cudaError_t to_mom_t(const llb_ctx& c, const void* st, void* mom) {
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

}  // namespace llb
