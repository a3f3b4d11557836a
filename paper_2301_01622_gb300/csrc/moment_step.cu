// Moment-only lattice Boltzmann step, one component (Sec. II-III A).
//
// One step maps the shifted moments m(t) to m(t+1):
//   1. collision at every source node y (local):  A'(y) = (1-omega) A + omega j j / rho
//   2. reconstruction of the post-collision population travelling from y
//      along c_i (Eq. coll2):  g'_i(y) = w_i [d + 3 c_i.j + 4.5 c_i c_i:A' - 1.5 tr A']
//   3. pull streaming (Eq. stream):  g_i(x, t+1) = g'_i(x - c_i)
//   4. projection (Eq. HYD):  d = sum g_i, j = sum g_i c_i, A = sum g_i c_i c_i - cs^2 d I
// No population is ever stored in global memory (Sec. III A, "without arrays").
//
// Two kernels:
//   * k_moment_direct: one thread per output node, gathers the ten moments of
//     each of its Q neighbours and repeats the collision per neighbour.
//     Simple and shape-agnostic; the reference GPU path.
//   * k_moment_tiled: persistent z-marching kernel.  A CTA owns a BX x BY
//     column of output nodes and walks it plane by plane.  For every source
//     plane it collides each node of the tile plus a one-node halo ONCE,
//     evaluates the Q-3 populations that cross to another column and
//     publishes them in shared memory; each output thread then pulls one
//     scalar per direction (instead of ten moments) and adds it into one of
//     three rolling per-plane accumulators (planes s-1, s, s+1), so that each
//     moment is read from and written to HBM once per step.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "lattice.cuh"

namespace llb {
namespace {

template <class T>
__device__ __forceinline__ Mom<T> load_mom(const T* __restrict__ p, size_t idx, size_t N) {
    Mom<T> m;
    m.d = __ldg(p + idx);
    m.jx = __ldg(p + N + idx);
    m.jy = __ldg(p + 2 * N + idx);
    m.jz = __ldg(p + 3 * N + idx);
    m.axx = __ldg(p + 4 * N + idx);
    m.ayy = __ldg(p + 5 * N + idx);
    m.azz = __ldg(p + 6 * N + idx);
    m.axy = __ldg(p + 7 * N + idx);
    m.axz = __ldg(p + 8 * N + idx);
    m.ayz = __ldg(p + 9 * N + idx);
    return m;
}

template <class T>
__device__ __forceinline__ void store_mom(T* __restrict__ p, size_t idx, size_t N, const Mom<T>& m) {
    p[idx] = m.d;
    p[N + idx] = m.jx;
    p[2 * N + idx] = m.jy;
    p[3 * N + idx] = m.jz;
    p[4 * N + idx] = m.axx;
    p[5 * N + idx] = m.ayy;
    p[6 * N + idx] = m.azz;
    p[7 * N + idx] = m.axy;
    p[8 * N + idx] = m.axz;
    p[9 * N + idx] = m.ayz;
}

__device__ __forceinline__ int pmod(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------
// Direct kernel: grid (ceil(nx/128), ny, nz), one thread per output node.
template <class L, class T>
__global__ void __launch_bounds__(128) k_moment_direct(const T* __restrict__ in, T* __restrict__ out, int nx,
                                                       int ny, int nz, size_t N, T omega) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int z = blockIdx.z;
    if (x >= nx) return;
    Acc<T> acc;
    acc.zero();
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz)) continue;
                const int sx = wrap_idx(x - cx, nx), sy = wrap_idx(y - cy, ny), sz = wrap_idx(z - cz, nz);
                const size_t s = ((size_t)sz * ny + sy) * nx + sx;
                const Mom<T> c = collide(load_mom(in, s, N), omega);
                acc.add(g_dir<L, T>(c, g_shared(c), cx, cy, cz), cx, cy, cz);
            }
    store_mom(out, ((size_t)z * ny + y) * nx + x, N, acc.finish());
}

// ---------------------------------------------------------------------------
// Tiled z-marching kernel.
template <class L, class T, int BX, int BY>
struct Tiled {
    static constexpr int NT = BX * BY;             // threads = output columns of a tile
    static constexpr int HX = BX + 2, HY = BY + 2; // tile plus one-node halo
    static constexpr int HN = HX * HY;
    static constexpr int NH = HN - NT;             // halo nodes, one per thread t < NH
    static constexpr int NS = n_xy_shifted<L>();   // directions crossing columns
    static constexpr size_t smem_bytes = sizeof(T) * 2 * NS * HN;
    static_assert(NH <= NT, "halo must fit one node per thread");
};

// Publish the column-crossing populations of one collided node into G[k][n].
template <class L, class T, int HN>
__device__ __forceinline__ void publish(T* __restrict__ G, int n, const Mom<T>& c) {
    const T s0 = g_shared(c);
    int k = 0;
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz) || (cx == 0 && cy == 0)) continue;
                G[k * HN + n] = g_dir<L, T>(c, s0, cx, cy, cz);
                ++k;
            }
}

template <class L, class T, int BX, int BY>
__global__ void __launch_bounds__(BX * BY, 2)
    k_moment_tiled(const T* __restrict__ in, T* __restrict__ out, int nx, int ny, int nz, size_t N, T omega,
                   int ncx, long long W) {
    using K = Tiled<L, T, BX, BY>;
    constexpr int HX = K::HX, HN = K::HN, NS = K::NS, NH = K::NH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* const Gbase = reinterpret_cast<T*>(smem_raw);

    const int t = threadIdx.x;
    const int tx = t % BX, ty = t / BX;
    const int n1 = (ty + 1) * HX + (tx + 1);  // own node, halo coordinates
    // halo node handled by this thread (if t < NH): top row, bottom row, then side columns
    const bool has2 = t < NH;
    int hx2 = 0, hy2 = 0;
    if (t < HX) {
        hx2 = t; hy2 = 0;
    } else if (t < 2 * HX) {
        hx2 = t - HX; hy2 = BY + 1;
    } else {
        const int k = t - 2 * HX;
        hy2 = 1 + (k >> 1);
        hx2 = (k & 1) ? (BX + 1) : 0;
    }
    const int n2 = hy2 * HX + hx2;
    const size_t plane = (size_t)nx * ny;

    const long long w0 = (long long)blockIdx.x * W / gridDim.x;
    const long long w1 = (long long)(blockIdx.x + 1) * W / gridDim.x;
    int buf = 0;

    for (long long w = w0; w < w1;) {
        const int col = (int)(w / nz);
        const int za = (int)(w - (long long)col * nz);
        const long long wend = min(w1, (long long)(col + 1) * nz);
        const int zb = za + (int)(wend - w);  // outputs za .. zb-1
        w = wend;
        const int x0 = (col % ncx) * BX, y0 = (col / ncx) * BY;
        const size_t off1 = (size_t)pmod(y0 + ty, ny) * nx + pmod(x0 + tx, nx);
        const size_t off2 = (size_t)pmod(y0 - 1 + hy2, ny) * nx + pmod(x0 - 1 + hx2, nx);
        const bool store_ok = (x0 + tx < nx) && (y0 + ty < ny);

        int zs = pmod(za - 1, nz);
        Mom<T> m1 = load_mom(in, zs * plane + off1, N);
        Mom<T> m2;
        if (has2) m2 = load_mom(in, zs * plane + off2, N);

        Acc<T> a0, a1, a2;
        a0.zero(); a1.zero(); a2.zero();

        // One source plane s: X collects plane s-1 (complete afterwards),
        // Y plane s, Z plane s+1 (started here).
        auto plane_step = [&](int s, Acc<T>& X, Acc<T>& Y, Acc<T>& Z) {
            T* const G = Gbase + buf * (NS * HN);
            // prefetch source plane s+1
            Mom<T> p1, p2;
            const bool more = s + 1 <= zb;
            if (more) {
                const size_t zo = (size_t)pmod(s + 1, nz) * plane;
                p1 = load_mom(in, zo + off1, N);
                if (has2) p2 = load_mom(in, zo + off2, N);
            }
            const Mom<T> c1 = collide(m1, omega);
            publish<L, T, HN>(G, n1, c1);
            const T s01 = g_shared(c1);
            const T g_m = g_dir<L, T>(c1, s01, 0, 0, -1);
            const T g_0 = g_dir<L, T>(c1, s01, 0, 0, 0);
            const T g_p = g_dir<L, T>(c1, s01, 0, 0, 1);
            if (has2) publish<L, T, HN>(G, n2, collide(m2, omega));
            __syncthreads();
            Z.zero();
            int k = 0;
#pragma unroll
            for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
                for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
                    for (int cx = -1; cx <= 1; ++cx) {
                        if (!L::has(cx, cy, cz) || (cx == 0 && cy == 0)) continue;
                        const T g = G[k * HN + n1 - cy * HX - cx];
                        if (cz < 0) X.add(g, cx, cy, cz);
                        else if (cz == 0) Y.add(g, cx, cy, cz);
                        else Z.add(g, cx, cy, cz);
                        ++k;
                    }
            X.add(g_m, 0, 0, -1);
            Y.add(g_0, 0, 0, 0);
            Z.add(g_p, 0, 0, 1);
            if (s - 1 >= za && store_ok) store_mom(out, (size_t)(s - 1) * plane + off1, N, X.finish());
            buf ^= 1;
            if (more) {
                m1 = p1;
                if (has2) m2 = p2;
            }
        };

        int s = za - 1;
        for (;;) {
            if (s > zb) break;
            plane_step(s, a0, a1, a2);
            ++s;
            if (s > zb) break;
            plane_step(s, a1, a2, a0);
            ++s;
            if (s > zb) break;
            plane_step(s, a2, a0, a1);
            ++s;
        }
    }
}

constexpr int kBX = 32, kBY = 8;

template <class L, class T>
cudaError_t run_direct(const llb_ctx& c, const void* in, void* out) {
    dim3 block(128), grid((c.nx + 127) / 128, c.ny, c.nz);
    k_moment_direct<L, T><<<grid, block, 0, c.stream>>>(static_cast<const T*>(in), static_cast<T*>(out), c.nx,
                                                         c.ny, c.nz, c.N, (T)c.omega);
    return cudaGetLastError();
}

template <class L, class T>
int tiled_ctas(const llb_ctx& c) {
    using K = Tiled<L, T, kBX, kBY>;
    auto kern = k_moment_tiled<L, T, kBX, kBY>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem_bytes) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, K::NT, K::smem_bytes) != cudaSuccess ||
        per_sm < 1)
        return 0;
    const long long ncol = (long long)((c.nx + kBX - 1) / kBX) * ((c.ny + kBY - 1) / kBY);
    const long long W = ncol * c.nz;
    return (int)std::min<long long>(W, (long long)per_sm * c.num_sms);
}

template <class L, class T>
cudaError_t run_tiled(const llb_ctx& c, const void* in, void* out) {
    using K = Tiled<L, T, kBX, kBY>;
    const int ncx = (c.nx + kBX - 1) / kBX;
    const long long ncol = (long long)ncx * ((c.ny + kBY - 1) / kBY);
    const long long W = ncol * c.nz;
    const int grid = c.tile_ctas > 0 ? c.tile_ctas : 1;
    k_moment_tiled<L, T, kBX, kBY><<<grid, K::NT, K::smem_bytes, c.stream>>>(
        static_cast<const T*>(in), static_cast<T*>(out), c.nx, c.ny, c.nz, c.N, (T)c.omega, ncx, W);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_moment_direct(const llb_ctx& c, const void* in, void* out) {
    if (c.Q == 19) return c.storage == LLB_F64 ? run_direct<D3Q19, double>(c, in, out) : run_direct<D3Q19, float>(c, in, out);
    return c.storage == LLB_F64 ? run_direct<D3Q27, double>(c, in, out) : run_direct<D3Q27, float>(c, in, out);
}

int moment_tiled_ctas(const llb_ctx& c) {
    if (c.Q == 19) return c.storage == LLB_F64 ? tiled_ctas<D3Q19, double>(c) : tiled_ctas<D3Q19, float>(c);
    return c.storage == LLB_F64 ? tiled_ctas<D3Q27, double>(c) : tiled_ctas<D3Q27, float>(c);
}

cudaError_t launch_moment_tiled(const llb_ctx& c, const void* in, void* out) {
    if (c.Q == 19) return c.storage == LLB_F64 ? run_tiled<D3Q19, double>(c, in, out) : run_tiled<D3Q19, float>(c, in, out);
    return c.storage == LLB_F64 ? run_tiled<D3Q27, double>(c, in, out) : run_tiled<D3Q27, float>(c, in, out);
}

}  // namespace llb
