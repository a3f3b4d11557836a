// Device pieces shared by the z-marching moment-only kernels (one component):
// moment loads and stores, the work schedule, and the shared-memory exchange
// of the populations that cross between the columns of a tile.
//
// One step maps the shifted moments m(t) to m(t+1) (Sec. II-III A):
//   1. collision at every source node y (local):  A'(y) = (1-omega) A + omega j j / rho
//   2. reconstruction of the post-collision population travelling from y
//      along c_i (Eq. (8)):  g'_i(y) = w_i [d + 3 c_i.j + 4.5 c_i c_i:A' - 1.5 tr A']
//   3. pull streaming (Eq. (9)):  g_i(x, t+1) = g'_i(x - c_i)
//   4. projection (Eqs. (1)-(3)):  d = sum g_i, j = sum g_i c_i, A = sum g_i c_i c_i - cs^2 d I
// No population is ever stored in global memory (Sec. III A, "without arrays").
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "checked.cuh"
#include "internal.h"
#include "lattice.cuh"
#include "layout.cuh"
#include "storage.cuh"
#include "tma.cuh"

namespace llb {
namespace mom {

// cycles (~50 ms) to let this CTA's copies in flight land after an abort: a
// 16 KB box arrives within microseconds even under heavy load
constexpr long long kDrainBudget = 100000000LL;

// Ten shifted moments of node idx from a state of element type S (converted to T).
// Ten shifted moments of node idx (index of the node in the state buffer p).
template <class T, class S>
__device__ __forceinline__ Mom<T> load_mom(const S* __restrict__ p, size_t idx, size_t fs) {
    using FM = FieldMap<S, 10>;
    Mom<T> m;
    m.d = ld_field<T>(p + FM::at(idx, 0, fs), 0);
    m.jx = ld_field<T>(p + FM::at(idx, 1, fs), 1);
    m.jy = ld_field<T>(p + FM::at(idx, 2, fs), 2);
    m.jz = ld_field<T>(p + FM::at(idx, 3, fs), 3);
    m.axx = ld_field<T>(p + FM::at(idx, 4, fs), 4);
    m.ayy = ld_field<T>(p + FM::at(idx, 5, fs), 5);
    m.azz = ld_field<T>(p + FM::at(idx, 6, fs), 6);
    m.axy = ld_field<T>(p + FM::at(idx, 7, fs), 7);
    m.axz = ld_field<T>(p + FM::at(idx, 8, fs), 8);
    m.ayz = ld_field<T>(p + FM::at(idx, 9, fs), 9);
    return m;
}

// The ten stored elements of one node as loaded.  A kernel that loads a plane
// ahead keeps these and converts them (from_raw) only when it collides the
// node, so that with 16-bit storage the wait for the load falls at the use and
// not right after the load.
template <class S>
struct RawMom {
    S v[10];
};

template <class S>
__device__ __forceinline__ RawMom<S> load_raw(const S* __restrict__ p, size_t idx, size_t fs) {
    RawMom<S> r;
#pragma unroll
    for (int f = 0; f < 10; ++f) r.v[f] = __ldg(p + FieldMap<S, 10>::at(idx, f, fs));
    return r;
}

template <class T, class S>
__device__ __forceinline__ Mom<T> from_raw(const RawMom<S>& r) {
    Mom<T> m;
    m.d = cv_field<T>(r.v[0], 0);
    m.jx = cv_field<T>(r.v[1], 1);
    m.jy = cv_field<T>(r.v[2], 2);
    m.jz = cv_field<T>(r.v[3], 3);
    m.axx = cv_field<T>(r.v[4], 4);
    m.ayy = cv_field<T>(r.v[5], 5);
    m.azz = cv_field<T>(r.v[6], 6);
    m.axy = cv_field<T>(r.v[7], 7);
    m.axz = cv_field<T>(r.v[8], 8);
    m.ayz = cv_field<T>(r.v[9], 9);
    return m;
}

template <class T, class S>
__device__ __forceinline__ void store_mom(S* __restrict__ p, size_t idx, size_t fs, const Mom<T>& m) {
    using FM = FieldMap<S, 10>;
    p[FM::at(idx, 0, fs)] = to_store<S>(m.d, 0);
    p[FM::at(idx, 1, fs)] = to_store<S>(m.jx, 1);
    p[FM::at(idx, 2, fs)] = to_store<S>(m.jy, 2);
    p[FM::at(idx, 3, fs)] = to_store<S>(m.jz, 3);
    p[FM::at(idx, 4, fs)] = to_store<S>(m.axx, 4);
    p[FM::at(idx, 5, fs)] = to_store<S>(m.ayy, 5);
    p[FM::at(idx, 6, fs)] = to_store<S>(m.azz, 6);
    p[FM::at(idx, 7, fs)] = to_store<S>(m.axy, 7);
    p[FM::at(idx, 8, fs)] = to_store<S>(m.axz, 8);
    p[FM::at(idx, 9, fs)] = to_store<S>(m.ayz, 9);
}

// Store node (x, y, z) and its periodic ghost copies.
template <class T, class S>
__device__ __forceinline__ void store_node(S* __restrict__ p, const Layout& L, int x, int y, int z, const Mom<T>& m) {
    for_node_and_ghosts(L, x, y, [&](int gx, int gy) {
        const size_t i = L.at(gx, gy, z);
        if (LLB_IN(i, L.fs, kChkGhost)) store_mom(p, i, L.fs, m);
    });
}

__host__ __device__ __forceinline__ int pmod(int v, int n) {
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
inline Sched plan(int nx, int ny, int nz, int BX, int BY, int grid) {
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
    if (!LLB_IN(n, HN, kChkPublish)) return;
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

// Publish the directions with c_x = sx (sx = +1 or -1 at run time) of a
// collided node of the left (sx = +1) or right (sx = -1) halo column or a
// corner: the only directions along which such a node feeds the tile.  One
// code path serves both signs, so the side and corner threads of a warp do
// not diverge.
template <class L, class T, int HN>
__device__ __forceinline__ void publish_side(T* __restrict__ G, int n, const Mom<T>& c, int sx) {
    if (!LLB_IN(n, HN, kChkPublish)) return;
    const T s = T(sx);
    const T base = g_shared(c) + T(4.5) * c.axx;
    const T sxy = s * c.axy, sxz = s * c.axz, sjx = T(3) * s * c.jx;
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy) {
            if (!L::has(1, cy, cz)) continue;
            T q = base;
            if (cy) q += T(4.5) * c.ayy;
            if (cz) q += T(4.5) * c.azz;
            if (cy) q += T(9 * cy) * sxy;
            if (cz) q += T(9 * cz) * sxz;
            if (cy * cz) q += T(9 * cy * cz) * c.ayz;
            T l = sjx;
            if (cy) l += T(3 * cy) * c.jy;
            if (cz) l += T(3 * cz) * c.jz;
            const int k = sx > 0 ? kslot<L>(1, cy, cz) : kslot<L>(-1, cy, cz);
            G[k * HN + n] = T(L::w(1, cy, cz)) * (q + l);
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
    // every neighbour slot n1 - cy HX - cx lies between these two
    if (!LLB_IN(n1 - HX - 1, HN, kChkGather) || !LLB_IN(n1 + HX + 1, HN, kChkGather)) return;
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

// Halo node handled by thread t < 2 BX + 2 BY + 4 and its role.  Threads
// [0, BX) take the row above the tile and publish only c_y = +1, threads
// [BX, 2 BX) the row below (c_y = -1); both roles are warp-uniform when BX is
// a multiple of 32.  The next 2 BY + 4 threads take the left and right
// columns and the four corners and publish only the directions with
// c_x = sx pointing into the tile (publish_side, one code path for both
// signs).
enum HaloRole { kNone, kTop, kBottom, kSide };

template <int BX, int BY>
__device__ __forceinline__ int halo_node(int t, int& hx, int& hy, int& sx) {
    sx = 1;
    if (t < BX) { hx = t + 1; hy = 0; return kTop; }
    if (t < 2 * BX) { hx = t - BX + 1; hy = BY + 1; return kBottom; }
    const int s = t - 2 * BX;
    if (s < BY) { hx = 0; hy = s + 1; sx = 1; return kSide; }
    if (s < 2 * BY) { hx = BX + 1; hy = s - BY + 1; sx = -1; return kSide; }
    switch (s - 2 * BY) {
        case 0: hx = 0; hy = 0; sx = 1; return kSide;
        case 1: hx = BX + 1; hy = 0; sx = -1; return kSide;
        case 2: hx = 0; hy = BY + 1; sx = 1; return kSide;
        case 3: hx = BX + 1; hy = BY + 1; sx = -1; return kSide;
        default: hx = 0; hy = 0; return kNone;
    }
}

// Publish a collided halo node: only the directions its role feeds.
template <class L, class T, int HN>
__device__ __forceinline__ void publish_halo(T* __restrict__ G, int n, int role, int sx, const Mom<T>& c) {
    if (role == kTop) publish<L, T, HN, kAny, 1>(G, n, c);
    else if (role == kBottom) publish<L, T, HN, kAny, -1>(G, n, c);
    else if (role == kSide) publish_side<L, T, HN>(G, n, c, sx);
}

}  // namespace mom
}  // namespace llb
