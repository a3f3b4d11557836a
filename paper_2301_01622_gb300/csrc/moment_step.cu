// Moment-only lattice Boltzmann step, one component (Sec. II-III A).
//
// One step maps the shifted moments m(t) to m(t+1):
//   1. collision at every source node y (local):  A'(y) = (1-omega) A + omega j j / rho
//   2. reconstruction of the post-collision population travelling from y
//      along c_i (Eq. (8)):  g'_i(y) = w_i [d + 3 c_i.j + 4.5 c_i c_i:A' - 1.5 tr A']
//   3. pull streaming (Eq. (9)):  g_i(x, t+1) = g'_i(x - c_i)
//   4. projection (Eqs. (1)-(3)):  d = sum g_i, j = sum g_i c_i, A = sum g_i c_i c_i - cs^2 d I
// No population is ever stored in global memory (Sec. III A, "without arrays").
//
// Three kernels:
//   * k_moment_direct: one thread per output node, gathers the ten moments of
//     each of its Q neighbours and repeats the collision per neighbour.
//     Shape-agnostic; the reference GPU path.
//   * k_moment_tiled: persistent z-marching kernel with plain loads.  A CTA
//     owns a BX x BY column of output nodes and walks it plane by plane.  For
//     every source plane it collides each node of the tile plus a one-node
//     halo ONCE, evaluates the Q-3 populations that cross to another column
//     and publishes them in shared memory; each output thread then pulls one
//     scalar per direction (instead of ten moments) and adds it into one of
//     three rolling per-plane accumulators (planes s-1, s, s+1).  Each moment
//     is read from and written to HBM once per step.
//   * k_moment_tma: the same computation, with the tile-plus-halo moments of
//     each source plane fetched by one TMA box load into an NST-deep ring of
//     shared-memory stages (mbarrier completion), so that several planes of
//     loads are in flight per CTA without holding registers.  Needs the
//     padded layout (periodic ghosts, 16-byte aligned tile start).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "internal.h"
#include "lattice.cuh"
#include "layout.cuh"
#include "storage.cuh"
#include "tma.cuh"

namespace llb {
namespace {

// cycles (~50 ms) to let this CTA's copies in flight land after an abort: a
// 16 KB box arrives within microseconds even under heavy load
constexpr long long kDrainBudget = 100000000LL;

// Ten shifted moments of node idx from a state of element type S (converted to T).
template <class T, class S>
__device__ __forceinline__ Mom<T> load_mom(const S* __restrict__ p, size_t idx, size_t fs) {
    Mom<T> m;
    m.d = ld_field<T>(p + idx, 0);
    m.jx = ld_field<T>(p + fs + idx, 1);
    m.jy = ld_field<T>(p + 2 * fs + idx, 2);
    m.jz = ld_field<T>(p + 3 * fs + idx, 3);
    m.axx = ld_field<T>(p + 4 * fs + idx, 4);
    m.ayy = ld_field<T>(p + 5 * fs + idx, 5);
    m.azz = ld_field<T>(p + 6 * fs + idx, 6);
    m.axy = ld_field<T>(p + 7 * fs + idx, 7);
    m.axz = ld_field<T>(p + 8 * fs + idx, 8);
    m.ayz = ld_field<T>(p + 9 * fs + idx, 9);
    return m;
}

template <class T, class S>
__device__ __forceinline__ void store_mom(S* __restrict__ p, size_t idx, size_t fs, const Mom<T>& m) {
    p[idx] = to_store<S>(m.d, 0);
    p[fs + idx] = to_store<S>(m.jx, 1);
    p[2 * fs + idx] = to_store<S>(m.jy, 2);
    p[3 * fs + idx] = to_store<S>(m.jz, 3);
    p[4 * fs + idx] = to_store<S>(m.axx, 4);
    p[5 * fs + idx] = to_store<S>(m.ayy, 5);
    p[6 * fs + idx] = to_store<S>(m.azz, 6);
    p[7 * fs + idx] = to_store<S>(m.axy, 7);
    p[8 * fs + idx] = to_store<S>(m.axz, 8);
    p[9 * fs + idx] = to_store<S>(m.ayz, 9);
}

// Store node (x, y, z) and its periodic ghost copies.
template <class T, class S>
__device__ __forceinline__ void store_node(S* __restrict__ p, const Layout& L, int x, int y, int z, const Mom<T>& m) {
    for_node_and_ghosts(L, x, y, [&](int gx, int gy) { store_mom(p, L.at(gx, gy, z), L.fs, m); });
}

__device__ __forceinline__ int pmod(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// Work of the z-marching kernels: items (z-chunk, xy-tile) in chunk-major
// order, handed out round-robin to the persistent CTAs, so that the CTAs
// resident at any moment hold neighbouring tiles of the same z-chunk and
// march through z together -- the halo planes a CTA reads from its
// neighbours' tiles were just fetched by them and are still in L2.
struct Sched {
    int ncx;      // tiles along x
    int ntiles;   // tiles per z-chunk
    int zc;       // planes per chunk (the last chunk may be shorter)
    int nitems;   // ntiles * chunks

    __device__ __forceinline__ void item(int it, int BX, int BY, int nz, int& x0, int& y0, int& za,
                                         int& zb) const {
        const int chunk = it / ntiles, tile = it - chunk * ntiles;
        x0 = (tile % ncx) * BX;
        y0 = (tile / ncx) * BY;
        za = chunk * zc;
        zb = min(nz, za + zc);
    }
};

// Pick the chunk length that minimises rounds * (planes per item + 2 warm-up
// planes) for `grid` persistent CTAs.
Sched plan(int nx, int ny, int nz, int BX, int BY, int grid) {
    Sched s;
    s.ncx = (nx + BX - 1) / BX;
    s.ntiles = s.ncx * ((ny + BY - 1) / BY);
    long long best = -1;
    for (int nch = 1; nch <= nz; ++nch) {
        const int zc = (nz + nch - 1) / nch;
        const int chunks = (nz + zc - 1) / zc;
        const long long items = (long long)s.ntiles * chunks;
        if (items > (1LL << 30)) break;
        const long long rounds = (items + grid - 1) / grid;
        const long long cost = rounds * (zc + 2);
        if (best < 0 || cost < best) {
            best = cost;
            s.zc = zc;
            s.nitems = (int)items;
        }
    }
    return s;
}

// ---------------------------------------------------------------------------
// Direct kernel: grid (ceil(nx/128), ny, nz), one thread per output node.
template <class L, class T, class S>
__global__ void __launch_bounds__(128) k_moment_direct(const S* __restrict__ in, S* __restrict__ out, Layout lay,
                                                       T omega) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    const int z = blockIdx.z;
    if (x >= lay.nx) return;
    Acc<T> acc;
    acc.zero();
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz)) continue;
                const size_t s = lay.at(wrap_idx(x - cx, lay.nx), wrap_idx(y - cy, lay.ny), wrap_idx(z - cz, lay.nz));
                const Mom<T> c = collide(load_mom<T>(in, s, lay.fs), omega);
                acc.add(g_dir<L, T>(c, g_shared(c), cx, cy, cz), cx, cy, cz);
            }
    store_node(out, lay, x, y, z, acc.finish());
}

// ---------------------------------------------------------------------------
// Shared pieces of the two z-marching kernels.

// Slot of direction (cx, cy, cz) among the column-crossing directions
// ((cx, cy) != (0, 0)), enumerated over cz, cy, cx in {-1, 0, 1}.
template <class L>
__host__ __device__ constexpr int kslot(int cx, int cy, int cz) {
    int k = 0;
    for (int z = -1; z <= 1; ++z)
        for (int y = -1; y <= 1; ++y)
            for (int x = -1; x <= 1; ++x) {
                if (!L::has(x, y, z) || (x == 0 && y == 0)) continue;
                if (x == cx && y == cy && z == cz) return k;
                ++k;
            }
    return -1;
}

// Which crossing directions a node of the staged tile publishes: all of them
// for a tile node, only those pointing into the tile for a halo node (a halo
// node above the tile feeds its outputs only along c_y = +1, and so on).
constexpr int kAny = 2;

template <int RX, int RY>
__host__ __device__ constexpr bool wanted(int cx, int cy) {
    return (RX == kAny || cx == RX) && (RY == kAny || cy == RY);
}

// Publish the crossing populations of one collided node into G[k][n].
// Directions come in opposite pairs (c, -c) sharing the even part of Eq.
// (8): g'_{+-c} = w (q +- l) with q = d - 1.5 tr A' + 4.5 c c : A',
// l = 3 c.j.
template <class L, class T, int HN, int RX = kAny, int RY = kAny>
__device__ __forceinline__ void publish(T* __restrict__ G, int n, const Mom<T>& c) {
    const T s0 = g_shared(c);
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                // visit each pair once, from its member with the first non-zero component > 0
                const bool lead = cx > 0 || (cx == 0 && (cy > 0 || (cy == 0 && cz > 0)));
                if (!lead || !L::has(cx, cy, cz) || (cx == 0 && cy == 0)) continue;
                const bool wp = wanted<RX, RY>(cx, cy), wm = wanted<RX, RY>(-cx, -cy);
                if (!wp && !wm) continue;
                T q = s0;
                if (cx) q += T(4.5) * c.axx;
                if (cy) q += T(4.5) * c.ayy;
                if (cz) q += T(4.5) * c.azz;
                if (cx * cy) q += T(9 * cx * cy) * c.axy;
                if (cx * cz) q += T(9 * cx * cz) * c.axz;
                if (cy * cz) q += T(9 * cy * cz) * c.ayz;
                T l = T(0);
                if (cx) l += T(3 * cx) * c.jx;
                if (cy) l += T(3 * cy) * c.jy;
                if (cz) l += T(3 * cz) * c.jz;
                const T w = T(L::w(cx, cy, cz));
                const T wq = w * q, wl = w * l;
                if (wp) G[kslot<L>(cx, cy, cz) * HN + n] = wq + wl;
                if (wm) G[kslot<L>(-cx, -cy, -cz) * HN + n] = wq - wl;
            }
}

// Populations g'_i of the own column (c_x = c_y = 0): directions -z, 0, +z.
template <class L, class T>
__device__ __forceinline__ void own_column(const Mom<T>& c, T& g_m, T& g_0, T& g_p) {
    const T s0 = g_shared(c);
    const T wz = T(L::w(0, 0, 1));
    const T wq = wz * (s0 + T(4.5) * c.azz), wl = wz * (T(3) * c.jz);
    g_p = wq + wl;
    g_m = wq - wl;
    g_0 = T(L::w(0, 0, 0)) * s0;
}

// Add the populations that node n1 pulls from source plane s with c_z = CZ
// into the accumulator of plane s + CZ (INIT: the accumulator starts here
// and is assigned instead).  Opposite directions in x (and y) are combined
// first (sum and difference), so each moment gets one add per pair instead
// of one per direction; no partial sum starts from an explicit zero.
template <class T, bool INIT>
__device__ __forceinline__ void acc_to(T& a, T v) {
    if constexpr (INIT) a = v; else a += v;
}

template <class L, class T, int CZ, bool INIT = false>
__device__ __forceinline__ void add_plane(const T* __restrict__ g, T g_own, Acc<T>& A) {
    static_assert(L::has(1, 0, CZ) && L::has(0, 1, CZ), "lattice without the axis-plane directions");
    const T ax = g[kslot<L>(1, 0, CZ)], bx = g[kslot<L>(-1, 0, CZ)];
    const T ay = g[kslot<L>(0, 1, CZ)], by = g[kslot<L>(0, -1, CZ)];
    const T sx = ax + bx, sy = ay + by;
    T jx = ax - bx, jy = ay - by;
    T sxx = sx, syy = sy;
    T sum = (g_own + sx) + sy;
    if constexpr (L::has(1, 1, CZ)) {
        const T pp = g[kslot<L>(1, 1, CZ)], mm = g[kslot<L>(-1, -1, CZ)];
        const T pm = g[kslot<L>(1, -1, CZ)], mp = g[kslot<L>(-1, 1, CZ)];
        const T a = pp + mm, b = pm + mp, c = pp - mm, e = pm - mp;
        const T sd = a + b;
        sum += sd;
        sxx += sd;
        syy += sd;
        jx += c + e;
        jy += c - e;
        acc_to<T, INIT>(A.sxy, a - b);
    } else if constexpr (INIT) {
        A.sxy = T(0);
    }
    acc_to<T, INIT>(A.d, sum);
    acc_to<T, INIT>(A.jx, jx);
    acc_to<T, INIT>(A.jy, jy);
    acc_to<T, INIT>(A.sxx, sxx);
    acc_to<T, INIT>(A.syy, syy);
    if constexpr (CZ != 0) {
        acc_to<T, INIT>(A.szz, sum);
        if constexpr (CZ > 0) {
            acc_to<T, INIT>(A.jz, sum);
            acc_to<T, INIT>(A.sxz, jx);
            acc_to<T, INIT>(A.syz, jy);
        } else {
            static_assert(!INIT, "only the plane ahead starts here");
            A.jz -= sum;
            A.sxz -= jx;
            A.syz -= jy;
        }
    } else {
        static_assert(!INIT, "only the plane ahead starts here");
    }
}

// Pull the crossing populations of output node n1 from G and add them to the
// accumulators of planes s-1 (X), s (Y), s+1 (Z, started here); the
// own-column populations come from registers.
template <class L, class T, int HN, int HX>
__device__ __forceinline__ void gather(const T* __restrict__ G, int n1, T g_m, T g_0, T g_p, Acc<T>& X, Acc<T>& Y,
                                       Acc<T>& Z) {
    constexpr int NS = n_xy_shifted<L>();
    T g[NS];
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz) || (cx == 0 && cy == 0)) continue;
                const int k = kslot<L>(cx, cy, cz);
                g[k] = G[k * HN + n1 - cy * HX - cx];
            }
    add_plane<L, T, -1>(g, g_m, X);
    add_plane<L, T, 0>(g, g_0, Y);
    add_plane<L, T, 1, true>(g, g_p, Z);
}

// Halo node handled by thread t < NH and its role.  Threads [0, BX) take the
// row above the tile and publish only c_y = +1, threads [BX, 2 BX) the row
// below (c_y = -1); both roles are warp-uniform when BX is a multiple of 32.
// The remaining threads take the left and right columns and the corners
// and publish every crossing direction: one code path for the whole warp
// (the directions nobody pulls are simply never read).
enum HaloRole { kNone, kTop, kBottom, kSide };

template <int BX, int BY>
__device__ __forceinline__ int halo_node(int t, int& hx, int& hy) {
    if (t < BX) { hx = t + 1; hy = 0; return kTop; }
    if (t < 2 * BX) { hx = t - BX + 1; hy = BY + 1; return kBottom; }
    const int s = t - 2 * BX;
    if (s < BY) { hx = 0; hy = s + 1; return kSide; }
    if (s < 2 * BY) { hx = BX + 1; hy = s - BY + 1; return kSide; }
    switch (s - 2 * BY) {
        case 0: hx = 0; hy = 0; return kSide;
        case 1: hx = BX + 1; hy = 0; return kSide;
        case 2: hx = 0; hy = BY + 1; return kSide;
        case 3: hx = BX + 1; hy = BY + 1; return kSide;
        default: hx = 0; hy = 0; return kNone;
    }
}

// Publish a collided halo node: only the directions its role feeds.
template <class L, class T, int HN>
__device__ __forceinline__ void publish_halo(T* __restrict__ G, int n, int role, const Mom<T>& c) {
    if (role == kTop) publish<L, T, HN, kAny, 1>(G, n, c);
    else if (role == kBottom) publish<L, T, HN, kAny, -1>(G, n, c);
    else if (role == kSide) publish<L, T, HN>(G, n, c);
}

// ---------------------------------------------------------------------------
// Tiled z-marching kernel, plain loads.
// Options of the tiled kernel (bit flags):
//   kSplit   -- split-phase plane barrier: each thread arrives on an mbarrier
//               as soon as its populations are published, stores the plane
//               finished one step earlier while the others catch up, and only
//               then waits (bounded) before pulling; replaces __syncthreads.
//   kFastRcp -- FP32 collision with the approximate division for 1/rho.
//   kHaloWarps -- two extra warps collide and publish the halo ring of the
//               tile (top row, bottom row, side columns and corners) so that
//               every output warp does the same work per plane (BX = 64).
constexpr int kSplit = 1, kFastRcp = 2, kHaloWarps = 4;

template <class L, class T, int BX, int BY>
struct Tiled {
    static constexpr int NT = BX * BY;             // threads = output columns of a tile
    static constexpr int HX = BX + 2, HY = BY + 2; // tile plus one-node halo
    static constexpr int HN = HX * HY;
    static constexpr int NH = HN - NT;             // halo nodes, one per thread t < NH
    static constexpr int NS = n_xy_shifted<L>();   // directions crossing columns
    static constexpr size_t g_bytes = sizeof(T) * 2 * NS * HN;
    static constexpr size_t smem_bytes = g_bytes + 16;  // + two mbarriers (split-phase option)
    static_assert(NH <= NT, "halo must fit one node per thread");
    static_assert(g_bytes % 8 == 0, "mbarriers need 8-byte alignment");
};

template <class L, class T, int BX, int BY, int MINB, int OPT, class S>
__global__ void __launch_bounds__(BX * BY, MINB)
    k_moment_tiled(const S* __restrict__ in, S* __restrict__ out, Layout lay, T omega, Sched sc, int* err,
                   long long budget) {
    using K = Tiled<L, T, BX, BY>;
    constexpr int HX = K::HX, HN = K::HN, NS = K::NS;
    constexpr bool SPLIT = (OPT & kSplit) != 0, FAST = (OPT & kFastRcp) != 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* const Gbase = reinterpret_cast<T*>(smem_raw);
    const uint32_t bar0 = smem_u32(smem_raw + K::g_bytes);  // mbarrier of G buffer b at bar0 + 8 b
    const int nx = lay.nx, ny = lay.ny, nz = lay.nz;
    if constexpr (SPLIT) {
        if (threadIdx.x == 0) {
            mbar_init(bar0, K::NT);
            mbar_init(bar0 + 8, K::NT);
        }
        __syncthreads();
    }
    uint32_t phase = 0;  // bit b: parity of the next phase of buffer b's mbarrier

    const int t = threadIdx.x;
    const int tx = t % BX, ty = t / BX;
    const int n1 = (ty + 1) * HX + (tx + 1);
    int hx2, hy2;
    const int role2 = halo_node<BX, BY>(t, hx2, hy2);
    const bool has2 = role2 != kNone;
    const int n2 = hy2 * HX + hx2;
    const size_t plane = (size_t)lay.px * lay.py;
    int buf = 0;

    for (int it = blockIdx.x; it < sc.nitems; it += gridDim.x) {
        int x0, y0, za, zb;  // outputs za .. zb-1 of the tile at (x0, y0)
        sc.item(it, BX, BY, nz, x0, y0, za, zb);
        const S* const in1 = in + lay.at(pmod(x0 + tx, nx), pmod(y0 + ty, ny), 0);
        const S* const in2 = in + lay.at(pmod(x0 - 1 + hx2, nx), pmod(y0 - 1 + hy2, ny), 0);
        const int ox = x0 + tx, oy = y0 + ty;
        const bool store_ok = (ox < nx) && (oy < ny);
        // periodic ghost copies are needed only near the x and y faces of the box
        const bool ghost = store_ok && lay.ghosts &&
                           (ox < kGhostX || ox >= nx - kGhostX || oy < lay.yo || oy >= ny - lay.yo);
        S* out1 = out + (store_ok ? lay.at(ox, oy, za) : 0);   // output plane za, advanced per plane

        // source plane of the next load, wrapped incrementally (no division per plane)
        int zn = pmod(za - 1, nz);
        size_t zn_off = (size_t)zn * plane;
        Mom<T> m1 = load_mom<T>(in1 + zn_off, 0, lay.fs);
        Mom<T> m2;
        if (has2) m2 = load_mom<T>(in2 + zn_off, 0, lay.fs);

        Acc<T> a0, a1, a2;
        a0.zero(); a1.zero(); a2.zero();

        auto put = [&](const Acc<T>& A, int z) {
            const Mom<T> r = A.finish();
            store_mom(out1, 0, lay.fs, r);
            if (ghost) store_node(out, lay, ox, oy, z, r);
            out1 += plane;
        };

        // One source plane s: X, Y, Z accumulate output planes s-1, s, s+1.
        // Without kSplit, plane s-1 is finished and stored here; with kSplit
        // it is stored in the next step (from Z, before Z restarts as s+2).
        auto plane_step = [&](int s, Acc<T>& X, Acc<T>& Y, Acc<T>& Z) -> bool {
            T* const G = Gbase + buf * (NS * HN);
            // the next source plane is loaded into m1 / m2 as soon as their
            // collision is done (no second set of prefetch registers)
            const bool more = s + 1 <= zb;
            if (more) {
                if (++zn == nz) {
                    zn = 0;
                    zn_off = 0;
                } else {
                    zn_off += plane;
                }
            }
            const Mom<T> c1 = collide<T, FAST>(m1, omega);
            if (more) m1 = load_mom<T>(in1 + zn_off, 0, lay.fs);
            publish<L, T, HN>(G, n1, c1);
            T g_m, g_0, g_p;
            own_column<L, T>(c1, g_m, g_0, g_p);
            if (has2) {
                const Mom<T> c2 = collide<T, FAST>(m2, omega);
                if (more) m2 = load_mom<T>(in2 + zn_off, 0, lay.fs);
                publish_halo<L, T, HN>(G, n2, role2, c2);
            }
            if constexpr (SPLIT) {
                const uint32_t bar = bar0 + 8 * buf;
                mbar_arrive(bar);
                if (s - 2 >= za && store_ok) put(Z, s - 2);
                if (!mbar_wait_bounded(bar, (phase >> buf) & 1u, budget)) {
                    atomicExch(err, 2);
                    return false;
                }
                phase ^= 1u << buf;
            } else {
                __syncthreads();
            }
            gather<L, T, HN, HX>(G, n1, g_m, g_0, g_p, X, Y, Z);
            if (!SPLIT && s - 1 >= za && store_ok) put(X, s - 1);
            buf ^= 1;
            return true;
        };
        // the accumulator of the last output plane (zb - 1) when the march ends
        auto last = [&](const Acc<T>& X) {
            if (SPLIT && store_ok && zb - 1 >= za) put(X, zb - 1);
        };

        int s = za - 1;  // za - 1 < zb: every item has at least one output plane
        for (;;) {
            if (!plane_step(s, a0, a1, a2)) return;
            if (s == zb) { last(a0); break; }
            ++s;
            if (!plane_step(s, a1, a2, a0)) return;
            if (s == zb) { last(a1); break; }
            ++s;
            if (!plane_step(s, a2, a0, a1)) return;
            if (s == zb) { last(a2); break; }
            ++s;
        }
    }
}

// ---------------------------------------------------------------------------
// Tiled z-marching kernel with dedicated halo warps (kHaloWarps).  Threads
// [0, BX BY) own the output columns; the 64 threads after them (two warps)
// collide the halo ring of every source plane: thread h takes top-row node
// h, bottom-row node h and, for h < 2 BY + 4, one side-column or corner
// node.  Both groups pass the same barrier once per plane; since the
// exchange buffer is double-buffered, the halo warps may run one plane ahead
// of the output warps' pulls.
template <class L, class T, int BX, int BY, int MINB, int OPT, class S>
__global__ void __launch_bounds__(BX * BY + 64, MINB)
    k_moment_tiled_hw(const S* __restrict__ in, S* __restrict__ out, Layout lay, T omega, Sched sc) {
    static_assert(BX == 64, "the halo warps take one top-row and one bottom-row node per thread");
    using K = Tiled<L, T, BX, BY>;
    constexpr int HX = K::HX, HN = K::HN, NS = K::NS, NO = BX * BY;
    constexpr bool FAST = (OPT & kFastRcp) != 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* const Gbase = reinterpret_cast<T*>(smem_raw);
    const int nx = lay.nx, ny = lay.ny, nz = lay.nz;
    const size_t plane = (size_t)lay.px * lay.py;

    const int t = threadIdx.x;
    const bool outw = t < NO;  // warp-uniform: NO is a multiple of 32
    const int h = t - NO;
    // output role
    const int tx = t % BX, ty = t / BX;
    const int n1 = (ty + 1) * HX + (tx + 1);
    // halo role: top node (h + 1, 0), bottom node (h + 1, BY + 1), side / corner node
    int hxc = 0, hyc = 0;
    const bool hasc = !outw && h < 2 * BY + 4;
    if (hasc) {
        if (h < BY) { hxc = 0; hyc = h + 1; }
        else if (h < 2 * BY) { hxc = BX + 1; hyc = h - BY + 1; }
        else {
            const int k = h - 2 * BY;
            hxc = (k & 1) ? BX + 1 : 0;
            hyc = (k & 2) ? BY + 1 : 0;
        }
    }
    const int nA = h + 1, nB = (BY + 1) * HX + h + 1, nC = hyc * HX + hxc;
    int buf = 0;

    for (int it = blockIdx.x; it < sc.nitems; it += gridDim.x) {
        int x0, y0, za, zb;
        sc.item(it, BX, BY, nz, x0, y0, za, zb);
        // per-thread base pointers (plane 0) of up to three source nodes
        const S* pA;
        const S* pB = in;
        const S* pC = in;
        if (outw) {
            pA = in + lay.at(pmod(x0 + tx, nx), pmod(y0 + ty, ny), 0);
        } else {
            pA = in + lay.at(pmod(x0 + h, nx), pmod(y0 - 1, ny), 0);
            pB = in + lay.at(pmod(x0 + h, nx), pmod(y0 + BY, ny), 0);
            if (hasc) pC = in + lay.at(pmod(x0 - 1 + hxc, nx), pmod(y0 - 1 + hyc, ny), 0);
        }
        const int ox = x0 + tx, oy = y0 + ty;
        const bool store_ok = outw && (ox < nx) && (oy < ny);
        const bool ghost = store_ok && lay.ghosts &&
                           (ox < kGhostX || ox >= nx - kGhostX || oy < lay.yo || oy >= ny - lay.yo);
        S* out1 = out + (store_ok ? lay.at(ox, oy, za) : 0);

        int zn = pmod(za - 1, nz);
        size_t zn_off = (size_t)zn * plane;
        Mom<T> mA = load_mom<T>(pA + zn_off, 0, lay.fs);
        Mom<T> mB, mC;
        if (!outw) mB = load_mom<T>(pB + zn_off, 0, lay.fs);
        if (hasc) mC = load_mom<T>(pC + zn_off, 0, lay.fs);

        Acc<T> a0, a1, a2;
        a0.zero(); a1.zero(); a2.zero();

        auto plane_step = [&](int s, Acc<T>& X, Acc<T>& Y, Acc<T>& Z) {
            T* const G = Gbase + buf * (NS * HN);
            const bool more = s + 1 <= zb;
            if (more) {
                if (++zn == nz) {
                    zn = 0;
                    zn_off = 0;
                } else {
                    zn_off += plane;
                }
            }
            T g_m = T(0), g_0 = T(0), g_p = T(0);
            if (outw) {
                const Mom<T> c1 = collide<T, FAST>(mA, omega);
                if (more) mA = load_mom<T>(pA + zn_off, 0, lay.fs);
                publish<L, T, HN>(G, n1, c1);
                own_column<L, T>(c1, g_m, g_0, g_p);
            } else {
                const Mom<T> cA = collide<T, FAST>(mA, omega);
                if (more) mA = load_mom<T>(pA + zn_off, 0, lay.fs);
                publish<L, T, HN, kAny, 1>(G, nA, cA);
                const Mom<T> cB = collide<T, FAST>(mB, omega);
                if (more) mB = load_mom<T>(pB + zn_off, 0, lay.fs);
                publish<L, T, HN, kAny, -1>(G, nB, cB);
                if (hasc) {
                    const Mom<T> cC = collide<T, FAST>(mC, omega);
                    if (more) mC = load_mom<T>(pC + zn_off, 0, lay.fs);
                    publish<L, T, HN>(G, nC, cC);
                }
            }
            __syncthreads();
            if (outw) {
                gather<L, T, HN, HX>(G, n1, g_m, g_0, g_p, X, Y, Z);
                if (s - 1 >= za && store_ok) {
                    const Mom<T> r = X.finish();
                    store_mom(out1, 0, lay.fs, r);
                    if (ghost) store_node(out, lay, ox, oy, s - 1, r);
                    out1 += plane;
                }
            }
            buf ^= 1;
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

// ---------------------------------------------------------------------------
// TMA-staged z-marching kernel.
template <class L, class T, int BX_, int BY_, int NST_, int MINB_>
struct TmaCfg {
    static constexpr int BX = BX_, BY = BY_, NST = NST_;
    static constexpr int NT = BX * BY;
    static constexpr int HX = BX + 2, HY = BY + 2, HN = HX * HY, NH = HN - NT;
    static constexpr int NS = n_xy_shifted<L>();
    static constexpr int SW = BX + 8;        // staged row: x0-4 .. x0+BX+3
    static constexpr int SR = BY + 2;        // staged rows: y0-1 .. y0+BY
    static constexpr int SF = SW * SR;       // elements per staged field
    static constexpr int STAGE_BYTES = 10 * SF * (int)sizeof(T);
    static constexpr int STAGE_STRIDE = (STAGE_BYTES + 1023) / 1024 * 1024;
    static constexpr int G_OFF = NST * STAGE_STRIDE;
    static constexpr int G_BYTES = 2 * NS * HN * (int)sizeof(T);
    static constexpr int BAR_OFF = (G_OFF + G_BYTES + 7) / 8 * 8;
    static constexpr int SMEM = BAR_OFF + 8 * NST + 1024;  // + slack to align the base to 1 KB
    static constexpr int MINB = MINB_;                      // CTAs per SM the register budget targets
    static_assert(NH <= NT, "halo must fit one node per thread");
    static_assert(SW * (int)sizeof(T) % 16 == 0, "TMA box row must be a multiple of 16 bytes");
    static_assert(SW <= 256 && SR <= 256, "TMA box dimension limit");
};

template <class T, int SF, int SW>
__device__ __forceinline__ Mom<T> stage_mom(const T* __restrict__ S, int hx, int hy) {
    const T* p = S + hy * SW + hx + 3;
    Mom<T> m;
    m.d = p[0];
    m.jx = p[SF];
    m.jy = p[2 * SF];
    m.jz = p[3 * SF];
    m.axx = p[4 * SF];
    m.ayy = p[5 * SF];
    m.azz = p[6 * SF];
    m.axy = p[7 * SF];
    m.axz = p[8 * SF];
    m.ayz = p[9 * SF];
    return m;
}

template <class L, class T, class C>
__global__ void __launch_bounds__(C::NT, C::MINB)
    k_moment_tma(const __grid_constant__ CUtensorMap tmap, T* __restrict__ out, Layout lay, T omega, Sched sc,
                 int* __restrict__ err, long long wait_budget, int extra_tx) {
    constexpr int BX = C::BX, BY = C::BY, NST = C::NST, HX = C::HX, HN = C::HN, NS = C::NS;
    constexpr int SF = C::SF, SW = C::SW;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    T* const Gbase = reinterpret_cast<T*>(smem + C::G_OFF);
    const uint32_t stage0 = smem_u32(smem);
    const uint32_t bar0 = smem_u32(smem + C::BAR_OFF);
    const T* const S0 = reinterpret_cast<const T*>(smem);
    const int nx = lay.nx, ny = lay.ny, nz = lay.nz;

    const int t = threadIdx.x;
    const int tx = t % BX, ty = t / BX;
    const int n1 = (ty + 1) * HX + (tx + 1);
    int hx2, hy2;
    const int role2 = halo_node<BX, BY>(t, hx2, hy2);
    const bool has2 = role2 != kNone;
    const int n2 = hy2 * HX + hx2;

    if (t == 0) {
        prefetch_tensormap(&tmap);
        for (int k = 0; k < NST; ++k) mbar_init(bar0 + 8 * k, 1);
        fence_barrier_init();
        fence_proxy_async();
    }
    __syncthreads();

    int buf = 0;
    unsigned q = 0;         // sequence number of the next source plane (all items)
    unsigned issued = 0;    // sequence numbers < issued have a TMA in flight or done (thread 0)
    // box origin: real (x0 - 4, y0 - 1) in padded coordinates
    const int bxo = lay.xo - 4, byo = lay.yo - 1;

    for (int it = blockIdx.x; it < sc.nitems; it += gridDim.x) {
        int x0, y0, za, zb;  // outputs za .. zb-1 of the tile at (x0, y0)
        sc.item(it, BX, BY, nz, x0, y0, za, zb);
        const int P = zb - za + 2;            // source planes za-1 .. zb
        const unsigned q0 = q;
        const bool store_ok = (x0 + tx < nx) && (y0 + ty < ny);

        if (t == 0) {
            for (int i = 0; i < NST && i < P; ++i) {
                const unsigned qq = q0 + i;
                const uint32_t bar = bar0 + 8 * (qq % NST);
                mbar_arrive_expect_tx(bar, C::STAGE_BYTES + extra_tx);
                tma_load_4d(stage0 + (qq % NST) * C::STAGE_STRIDE, &tmap, x0 + bxo, y0 + byo, pmod(za - 1 + i, nz), 0,
                            bar);
            }
            issued = q0 + min(NST, P);
        }

        Acc<T> a0, a1, a2;
        a0.zero(); a1.zero(); a2.zero();
        const int ox = x0 + tx, oy = y0 + ty;
        // periodic ghost copies are needed only near the x and y faces of the box
        const bool ghost = store_ok && (ox < kGhostX || ox >= nx - kGhostX || oy < lay.yo || oy >= ny - lay.yo);
        T* out1 = out + (store_ok ? lay.at(ox, oy, za) : 0);   // output plane za, advanced per plane
        const size_t plane = (size_t)lay.px * lay.py;

        auto plane_step = [&](int s, Acc<T>& X, Acc<T>& Y, Acc<T>& Z) -> bool {
            const int k = q % NST;
            const bool ok = mbar_wait_bounded(bar0 + 8 * k, (q / NST) & 1, wait_budget);
            const T* const S = S0 + (size_t)k * (C::STAGE_STRIDE / sizeof(T));
            T* const G = Gbase + buf * (NS * HN);
            T g_m = T(0), g_0 = T(0), g_p = T(0);
            if (ok) {
                const Mom<T> c1 = collide<T, true>(stage_mom<T, SF, SW>(S, tx + 1, ty + 1), omega);
                publish<L, T, HN>(G, n1, c1);
                own_column<L, T>(c1, g_m, g_0, g_p);
                if (has2)
                    publish_halo<L, T, HN>(G, n2, role2, collide<T, true>(stage_mom<T, SF, SW>(S, hx2, hy2), omega));
            }
            if (__syncthreads_or(!ok)) return false;
            // every thread is done with stage k: refill it with plane s + NST
            if (t == 0 && (int)(q - q0) + NST < P) {
                fence_proxy_async();
                const unsigned qq = q + NST;
                const uint32_t bar = bar0 + 8 * k;
                mbar_arrive_expect_tx(bar, C::STAGE_BYTES + extra_tx);
                tma_load_4d(stage0 + k * C::STAGE_STRIDE, &tmap, x0 + bxo, y0 + byo, pmod(s + NST, nz), 0, bar);
                issued = qq + 1;
            }
            gather<L, T, HN, HX>(G, n1, g_m, g_0, g_p, X, Y, Z);
            if (s - 1 >= za && store_ok) {
                const Mom<T> r = X.finish();
                store_mom(out1, 0, lay.fs, r);
                if (ghost) store_node(out, lay, ox, oy, s - 1, r);
                out1 += plane;
            }
            buf ^= 1;
            ++q;
            return true;
        };

        bool alive = true;
        int s = za - 1;
        for (;;) {
            if (s > zb) break;
            if (!(alive = plane_step(s, a0, a1, a2))) break;
            ++s;
            if (s > zb) break;
            if (!(alive = plane_step(s, a1, a2, a0))) break;
            ++s;
            if (s > zb) break;
            if (!(alive = plane_step(s, a2, a0, a1))) break;
            ++s;
        }
        if (!alive) {
            // A wait gave up: report, let the loads still in flight land (bounded), leave.
            if (t == 0) {
                atomicExch(err, 1);
                for (unsigned qq = q; qq < issued; ++qq)
                    mbar_wait_bounded(bar0 + 8 * (qq % NST), (qq / NST) & 1, kDrainBudget);
            }
            return;
        }
    }
}

// ---------------------------------------------------------------------------
// Host side.


// TMA kernel variants (tile BX x BY, ring depth, CTAs per SM).  Variant 0 is
// the default; the others exist for tuning sweeps (llb_params.variant).
template <class L, class T, int V>
struct TmaVariant;
// Ring depths are chosen so that two CTAs of the 256-thread tiles fit in
// the shared memory of one SM (2-3 x 17 KB stages + 51 KB exchange buffers);
// the 2-deep ring measured fastest on 256^3.
template <class L> struct TmaVariant<L, float, 0> { using type = TmaCfg<L, float, 64, 4, 2, 2>; };
template <class L> struct TmaVariant<L, float, 1> { using type = TmaCfg<L, float, 64, 8, 3, 1>; };
template <class L> struct TmaVariant<L, float, 2> { using type = TmaCfg<L, float, 64, 4, 3, 2>; };
template <class L> struct TmaVariant<L, float, 3> { using type = TmaCfg<L, float, 32, 8, 3, 2>; };
template <class L> struct TmaVariant<L, float, 4> { using type = TmaCfg<L, float, 128, 4, 3, 1>; };
template <class L, int V> struct TmaVariant<L, double, V> { using type = TmaCfg<L, double, 32, 8, 2, 1>; };
constexpr int kTmaVariants = 5;

template <class L, class T, class S>
cudaError_t run_direct(const llb_ctx& c, const void* in, void* out) {
    dim3 block(128), grid((c.nx + 127) / 128, c.ny, c.nz);
    k_moment_direct<L, T, S><<<grid, block, 0, c.stream>>>(static_cast<const S*>(in), static_cast<S*>(out), c.lay,
                                                            (T)c.omega);
    return cudaGetLastError();
}

// Plain-load tiled kernel variants (tile BX x BY, CTAs per SM the register
// budget targets, options); variant 0 is the default.
template <int BX_, int BY_, int MINB_, int OPT_ = 0>
struct TiledShape {
    static constexpr int BX = BX_, BY = BY_, MINB = MINB_, OPT = OPT_;
};
// FP32: the approximate 1/rho is the default (measured ~1.5 % faster at
// 256^3, error far below FP32 storage rounding); variant 5 keeps the
// IEEE-rounded division, variant 6 adds the split-phase plane barrier.
template <class T, int V> struct TiledVariant { using type = TiledShape<64, 4, 2, kFastRcp>; };
template <> struct TiledVariant<float, 1> { using type = TiledShape<64, 8, 1, kFastRcp>; };
template <> struct TiledVariant<float, 2> { using type = TiledShape<96, 4, 1, kFastRcp>; };
template <> struct TiledVariant<float, 3> { using type = TiledShape<32, 8, 2, kFastRcp>; };
template <> struct TiledVariant<float, 4> { using type = TiledShape<128, 4, 1, kFastRcp>; };
template <> struct TiledVariant<float, 5> { using type = TiledShape<64, 4, 2>; };
template <> struct TiledVariant<float, 6> { using type = TiledShape<64, 4, 2, kSplit | kFastRcp>; };
template <> struct TiledVariant<float, 7> { using type = TiledShape<32, 4, 4, kFastRcp>; };
// halo-warp forms: 16 warps per SM in total keep 128 registers per thread
template <> struct TiledVariant<float, 8> { using type = TiledShape<64, 7, 1, kFastRcp | kHaloWarps>; };
template <> struct TiledVariant<float, 9> { using type = TiledShape<64, 3, 2, kFastRcp | kHaloWarps>; };
template <int V> struct TiledVariant<double, V> { using type = TiledShape<32, 8, 1>; };

// Threads of a CTA of tile shape S (the halo-warp form adds two warps).
template <class S>
constexpr int tiled_threads() { return S::BX * S::BY + ((S::OPT & kHaloWarps) ? 64 : 0); }

template <class L, class T, class St, class S>
auto tiled_kernel() {
    if constexpr ((S::OPT & kHaloWarps) != 0)
        return k_moment_tiled_hw<L, T, S::BX, S::BY, S::MINB, S::OPT, St>;
    else
        return k_moment_tiled<L, T, S::BX, S::BY, S::MINB, S::OPT, St>;
}

template <class L, class T, class St, class S>
int tiled_ctas_c(const llb_ctx& c) {
    using K = Tiled<L, T, S::BX, S::BY>;
    auto kern = tiled_kernel<L, T, St, S>();
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem_bytes) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tiled_threads<S>(), K::smem_bytes) !=
            cudaSuccess ||
        per_sm < 1)
        return 0;
    const Sched sc = plan(c.nx, c.ny, c.nz, S::BX, S::BY, per_sm * c.num_sms);
    return std::min(sc.nitems, per_sm * c.num_sms);
}

template <class L, class T, class St, class S>
cudaError_t run_tiled_c(const llb_ctx& c, const void* in, void* out) {
    using K = Tiled<L, T, S::BX, S::BY>;
    const int grid = c.tile_ctas > 0 ? c.tile_ctas : 1;
    const Sched sc = plan(c.nx, c.ny, c.nz, S::BX, S::BY, grid);
    // device clock ~2 GHz: cycles per millisecond
    const long long budget = (long long)c.params.wait_budget_ms * 2000000LL;
    if constexpr ((S::OPT & kHaloWarps) != 0)
        k_moment_tiled_hw<L, T, S::BX, S::BY, S::MINB, S::OPT, St><<<grid, tiled_threads<S>(), K::smem_bytes,
                                                                      c.stream>>>(
            static_cast<const St*>(in), static_cast<St*>(out), c.lay, (T)c.omega, sc);
    else
        k_moment_tiled<L, T, S::BX, S::BY, S::MINB, S::OPT, St><<<grid, K::NT, K::smem_bytes, c.stream>>>(
            static_cast<const St*>(in), static_cast<St*>(out), c.lay, (T)c.omega, sc, static_cast<int*>(c.err_dev),
            budget);
    return cudaGetLastError();
}

#define LLB_TILED_VARIANT(fn, ...)                                                           \
    switch (c.variant) {                                                                     \
        case 1: return fn<L, T, St, typename TiledVariant<T, 1>::type>(__VA_ARGS__);         \
        case 2: return fn<L, T, St, typename TiledVariant<T, 2>::type>(__VA_ARGS__);         \
        case 3: return fn<L, T, St, typename TiledVariant<T, 3>::type>(__VA_ARGS__);         \
        case 4: return fn<L, T, St, typename TiledVariant<T, 4>::type>(__VA_ARGS__);         \
        case 5: return fn<L, T, St, typename TiledVariant<T, 5>::type>(__VA_ARGS__);         \
        case 6: return fn<L, T, St, typename TiledVariant<T, 6>::type>(__VA_ARGS__);         \
        case 7: return fn<L, T, St, typename TiledVariant<T, 7>::type>(__VA_ARGS__);         \
        case 8: return fn<L, T, St, typename TiledVariant<T, 8>::type>(__VA_ARGS__);         \
        case 9: return fn<L, T, St, typename TiledVariant<T, 9>::type>(__VA_ARGS__);         \
        default: return fn<L, T, St, typename TiledVariant<T, 0>::type>(__VA_ARGS__);        \
    }

template <class L, class T, class St>
int tiled_ctas(const llb_ctx& c) { LLB_TILED_VARIANT(tiled_ctas_c, c) }
template <class L, class T, class St>
cudaError_t run_tiled(const llb_ctx& c, const void* in, void* out) { LLB_TILED_VARIANT(run_tiled_c, c, in, out) }

template <class L, class T, class C>
int tma_ctas_c(const llb_ctx& c) {
    if (c.variant >= kTmaVariants) return 0;  // the TMA kernel has variants 0..4 only
    if (!c.lay.ghosts || c.lay.px < C::SW || c.lay.py < C::SR) return 0;
    auto kern = k_moment_tma<L, T, C>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM) != cudaSuccess) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, C::SMEM) != cudaSuccess || per_sm < 1)
        return 0;
    const Sched sc = plan(c.nx, c.ny, c.nz, C::BX, C::BY, per_sm * c.num_sms);
    return std::min(sc.nitems, per_sm * c.num_sms);
}

template <class L, class T, class C>
cudaError_t run_tma_c(const llb_ctx& c, int in_index, void* out) {
    const int grid = c.tma_ctas > 0 ? c.tma_ctas : 1;
    const Sched sc = plan(c.nx, c.ny, c.nz, C::BX, C::BY, grid);
    // device clock ~2 GHz: cycles per millisecond
    const long long budget = (long long)c.params.wait_budget_ms * 2000000LL;
    k_moment_tma<L, T, C><<<grid, C::NT, C::SMEM, c.stream>>>(c.tmap[in_index], static_cast<T*>(out), c.lay,
                                                               (T)c.omega, sc, static_cast<int*>(c.err_dev), budget,
                                                               (c.params.debug_flags & 1) ? 1 : 0);
    return cudaGetLastError();
}

template <class L, class T, class C>
bool tma_encode_c(const llb_ctx& c, void* buf, CUtensorMap* out) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const Layout& Lo = c.lay;
    if (!Lo.ghosts) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)Lo.px, (cuuint64_t)Lo.py, (cuuint64_t)Lo.nz, 10};
    const cuuint64_t strides[3] = {(cuuint64_t)Lo.px * sizeof(T), (cuuint64_t)Lo.px * Lo.py * sizeof(T),
                                   (cuuint64_t)Lo.fs * sizeof(T)};
    const cuuint32_t box[4] = {(cuuint32_t)C::SW, (cuuint32_t)C::SR, 1, 10};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = encode(out, sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                        buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

#define LLB_TMA_VARIANT(fn, ...)                                                                  \
    switch (c.variant) {                                                                          \
        case 1: return fn<L, T, typename TmaVariant<L, T, 1>::type>(__VA_ARGS__);                 \
        case 2: return fn<L, T, typename TmaVariant<L, T, 2>::type>(__VA_ARGS__);                 \
        case 3: return fn<L, T, typename TmaVariant<L, T, 3>::type>(__VA_ARGS__);                 \
        case 4: return fn<L, T, typename TmaVariant<L, T, 4>::type>(__VA_ARGS__);                 \
        default: return fn<L, T, typename TmaVariant<L, T, 0>::type>(__VA_ARGS__);                \
    }

template <class L, class T>
int tma_ctas(const llb_ctx& c) { LLB_TMA_VARIANT(tma_ctas_c, c) }
template <class L, class T>
cudaError_t run_tma(const llb_ctx& c, int in_index, void* out) { LLB_TMA_VARIANT(run_tma_c, c, in_index, out) }
template <class L, class T>
bool tma_encode(const llb_ctx& c, void* buf, CUtensorMap* out) { LLB_TMA_VARIANT(tma_encode_c, c, buf, out) }

}  // namespace

// (lattice, element type) -> kernel instance.  16-bit states compute in FP32.
#define LLB_SDISPATCH(fn, ...)                                                                    \
    switch (c.storage) {                                                                          \
        case LLB_F64: return c.Q == 19 ? fn<D3Q19, double, double>(__VA_ARGS__)                   \
                                       : fn<D3Q27, double, double>(__VA_ARGS__);                  \
        case LLB_F16S: return c.Q == 19 ? fn<D3Q19, float, __half>(__VA_ARGS__)                   \
                                        : fn<D3Q27, float, __half>(__VA_ARGS__);                  \
        case LLB_BF16S: return c.Q == 19 ? fn<D3Q19, float, __nv_bfloat16>(__VA_ARGS__)           \
                                         : fn<D3Q27, float, __nv_bfloat16>(__VA_ARGS__);          \
        default: return c.Q == 19 ? fn<D3Q19, float, float>(__VA_ARGS__)                          \
                                  : fn<D3Q27, float, float>(__VA_ARGS__);                         \
    }

// The TMA kernel stages FP32 or FP64 boxes only.
#define LLB_MDISPATCH(fn, fallback, ...)                                                          \
    switch (c.storage) {                                                                          \
        case LLB_F64: return c.Q == 19 ? fn<D3Q19, double>(__VA_ARGS__) : fn<D3Q27, double>(__VA_ARGS__); \
        case LLB_F32: return c.Q == 19 ? fn<D3Q19, float>(__VA_ARGS__) : fn<D3Q27, float>(__VA_ARGS__);   \
        default: return fallback;                                                                 \
    }

cudaError_t launch_moment_direct(const llb_ctx& c, const void* in, void* out) {
    LLB_SDISPATCH(run_direct, c, in, out)
}
int moment_tiled_ctas(const llb_ctx& c) { LLB_SDISPATCH(tiled_ctas, c) }
cudaError_t launch_moment_tiled(const llb_ctx& c, const void* in, void* out) {
    LLB_SDISPATCH(run_tiled, c, in, out)
}
int moment_tma_ctas(const llb_ctx& c) { LLB_MDISPATCH(tma_ctas, 0, c) }
cudaError_t launch_moment_tma(const llb_ctx& c, int in_index, void* out) {
    LLB_MDISPATCH(run_tma, cudaErrorInvalidValue, c, in_index, out)
}
bool moment_tma_encode(const llb_ctx& c, void* buf, CUtensorMap* out) {
    LLB_MDISPATCH(tma_encode, false, c, buf, out)
}

}  // namespace llb
