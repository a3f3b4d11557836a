// Two-component moment-only step: colour-gradient model with near-contact
// forcing (Sec. III A-B), fused into one z-marching kernel.
//
// State per node (11 fields): rho1, d = rho - 1 (total density), j, A = P - cs^2 rho I.
// Per source node y (tile plus one-node halo), from the moments at time t:
//   phi = (rho1 - rho2) / rho = 2 rho1 / rho - 1              (Sec. III B)
//   G = (1/cs^2) sum_k w_k c_k phi(y + c_k), n = G / |G| (0 if |G| < g_min);
//   with grad_eps > 0, |G| is the smooth sqrt(|G|^2 + eps^2) and n = G / |G| everywhere
//   near contact: |G| >= g_nci and phi(y + round(k n_out)) > phi(y) + 0.01 for
//   some k = 1..h_c, n_out = -n; then F = A_h G (F_rep = -A_h n_out delta_I,
//   delta_I = |G|), else F = 0
//   collision (BGK on the reconstructed populations, Guo forcing,
//   u_F = (j + F/2) / rho, colour-gradient perturbation):
//     j' = j + F
//     A' = (1 - w) A + w rho u_F u_F + (1 - w/2)(u_F F + F u_F) + A_s cs^4 |G| n n
//   post-collision populations g'_i = w_i [d + 3 c_i.j' + 4.5 c_i c_i:A' - 1.5 tr A']
//   recolouring: h1'_i = (rho1/rho)(w_i + g'_i) + beta (rho1 rho2 / rho) w_i (c_i.n)/|c_i|
// and per output node x: the total moments from sum_i g'_i(x - c_i) (Eqs. (9) and
// (1)-(3)) and rho1(x) = sum_i h1'_i(x - c_i).
//
// The CTA marches a BX x BY column through z like the one-component tiled
// kernel.  phi of the tile plus a two-node halo is kept for three planes
// (s-1, s, s+1) in shared memory, so the gradient at every source node is a
// shared-memory stencil; the near-contact probes, needed only on the
// interface band and only when A_h != 0, read phi from global memory (L2).
// Each source node publishes, for every direction that crosses to another
// column, both g'_i and h1'_i; each output thread pulls them and keeps
// rolling accumulators for the planes s-1, s, s+1.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "checked.cuh"
#include "internal.h"
#include "lattice.cuh"
#include "layout.cuh"

namespace llb {
namespace cg {

constexpr double kPhiRise = 0.01;  // phi rise at a probe that signals another interface
constexpr double kGNci = 0.05;     // |grad phi| above which a node is in the detector's interface band

template <class T>
struct CGPar {
    T omega, beta, A_s, A_h, g_min, g_nci;
    T eps2;  // > 0: smooth norm |G|_eps = sqrt(|G|^2 + eps2), normal defined everywhere
    int h_c;
};

template <class T>
struct Node2 {
    T r1;       // rho1
    Mom<T> m;   // d, j, A of the mixture
};

__device__ __forceinline__ int pmod2(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

template <class T>
__device__ __forceinline__ Node2<T> load_node2(const T* __restrict__ p, size_t i, size_t fs) {
    Node2<T> a{};
    if (!LLB_IN(i, fs, kChkLoad)) return a;
    a.r1 = __ldg(p + i);
    a.m.d = __ldg(p + fs + i);
    a.m.jx = __ldg(p + 2 * fs + i);
    a.m.jy = __ldg(p + 3 * fs + i);
    a.m.jz = __ldg(p + 4 * fs + i);
    a.m.axx = __ldg(p + 5 * fs + i);
    a.m.ayy = __ldg(p + 6 * fs + i);
    a.m.azz = __ldg(p + 7 * fs + i);
    a.m.axy = __ldg(p + 8 * fs + i);
    a.m.axz = __ldg(p + 9 * fs + i);
    a.m.ayz = __ldg(p + 10 * fs + i);
    return a;
}

template <class T>
__device__ __forceinline__ void store_node2(T* __restrict__ p, const Layout& L, int x, int y, int z, T r1,
                                            const Mom<T>& m) {
    for_node_and_ghosts(L, x, y, [&](int gx, int gy) {
        const size_t i = L.at(gx, gy, z);
        const size_t fs = L.fs;
        if (!LLB_IN(i, fs, kChkGhost)) return;
        p[i] = r1;
        p[fs + i] = m.d;
        p[2 * fs + i] = m.jx;
        p[3 * fs + i] = m.jy;
        p[4 * fs + i] = m.jz;
        p[5 * fs + i] = m.axx;
        p[6 * fs + i] = m.ayy;
        p[7 * fs + i] = m.azz;
        p[8 * fs + i] = m.axy;
        p[9 * fs + i] = m.axz;
        p[10 * fs + i] = m.ayz;
    });
}

template <class T>
__device__ __forceinline__ void store_node2_at(T* __restrict__ p, size_t fs, T r1, const Mom<T>& m) {
    p[0] = r1;
    p[fs] = m.d;
    p[2 * fs] = m.jx;
    p[3 * fs] = m.jy;
    p[4 * fs] = m.jz;
    p[5 * fs] = m.axx;
    p[6 * fs] = m.ayy;
    p[7 * fs] = m.azz;
    p[8 * fs] = m.axy;
    p[9 * fs] = m.axz;
    p[10 * fs] = m.ayz;
}

// phi = 2 rho1 / rho - 1 (FAST, FP32: approximate quotient)
template <bool FAST, class T>
__device__ __forceinline__ T phi_of(T r1, T d) {
    if constexpr (FAST && sizeof(T) == 4)
        return __fdividef(T(2) * r1, T(1) + d) - T(1);
    else
        return T(2) * r1 / (T(1) + d) - T(1);
}

template <class L>
__host__ __device__ constexpr int kslot2(int cx, int cy, int cz) {
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

__host__ __device__ constexpr double inv_len(int cx, int cy, int cz) {
    return (cx * cx + cy * cy + cz * cz) == 1 ? 1.0
         : (cx * cx + cy * cy + cz * cz) == 2 ? 0.70710678118654752440
         : (cx * cx + cy * cy + cz * cz) == 3 ? 0.57735026918962576451 : 0.0;
}

// (g'_i, h1'_i) of one direction, exchanged as one 8- (FP32) or 16-byte
// (FP64) shared-memory element so that a publish and a pull are one access.
template <class T>
struct alignas(2 * sizeof(T)) GH {
    T g, h;
};

// Collided source node: moments after collision and the colour quantities.
template <class T>
struct Src2 {
    Mom<T> c;     // d, j' = j + F, A'
    T r1;         // rho1 / rho
    T e;          // beta rho1 rho2 / rho
    T nx, ny, nz; // unit normal (0 off the interface)
};

// Normal, near-contact test, forcing and collision of one node whose phase-
// field gradient G is known.  phi0 = phi at the node; probe(ox, oy, oz)
// returns phi at the node offset by (ox, oy, oz) (periodic), read only on the
// interface band of the near-contact detector.
template <class T, bool FAST, class Probe>
__device__ __forceinline__ Src2<T> cg_collide(const Node2<T>& a, T Gx, T Gy, T Gz, T phi0, const CGPar<T>& p,
                                              Probe&& probe) {
    const T g2 = Gx * Gx + Gy * Gy + Gz * Gz;
    const bool smooth = p.eps2 > T(0);
    const T g2e = smooth ? g2 + p.eps2 : g2;
    T gn, ig;
    if constexpr (FAST && sizeof(T) == 4) {
        ig = g2e > T(0) ? rsqrtf(g2e) : T(0);
        gn = g2e * ig;
    } else {
        gn = sqrt(g2e);
        ig = gn > T(0) ? T(1) / gn : T(0);
    }
    const bool has_n = smooth || gn >= p.g_min;
    Src2<T> s;
    s.nx = s.ny = s.nz = T(0);
    if (has_n) {
        s.nx = Gx * ig;
        s.ny = Gy * ig;
        s.nz = Gz * ig;
    }
    // near-contact detector on the interface band
    T Fx = T(0), Fy = T(0), Fz = T(0);
    if (p.A_h != T(0) && gn >= p.g_nci) {
        bool near = false;
        for (int k = 1; k <= p.h_c && !near; ++k) {
            const int ox = (int)rint(-T(k) * s.nx), oy = (int)rint(-T(k) * s.ny), oz = (int)rint(-T(k) * s.nz);
            near = probe(ox, oy, oz) > phi0 + T(kPhiRise);
        }
        if (near) {
            Fx = p.A_h * Gx;
            Fy = p.A_h * Gy;
            Fz = p.A_h * Gz;
        }
    }
    const Mom<T>& m = a.m;
    const T rho = T(1) + m.d;
    const T rinv = inv_rho<FAST>(rho);
    const T ux = (m.jx + T(0.5) * Fx) * rinv, uy = (m.jy + T(0.5) * Fy) * rinv, uz = (m.jz + T(0.5) * Fz) * rinv;
    const T om = p.omega, one_m = T(1) - om, fh = T(1) - T(0.5) * om;
    const T ks = has_n ? p.A_s * gn * T(1.0 / 9.0) : T(0);
    const T orx = om * rho * ux, ory = om * rho * uy, orz = om * rho * uz;
    s.c.d = m.d;
    s.c.jx = m.jx + Fx;
    s.c.jy = m.jy + Fy;
    s.c.jz = m.jz + Fz;
    s.c.axx = one_m * m.axx + orx * ux + fh * (T(2) * ux * Fx) + ks * s.nx * s.nx;
    s.c.ayy = one_m * m.ayy + ory * uy + fh * (T(2) * uy * Fy) + ks * s.ny * s.ny;
    s.c.azz = one_m * m.azz + orz * uz + fh * (T(2) * uz * Fz) + ks * s.nz * s.nz;
    s.c.axy = one_m * m.axy + orx * uy + fh * (ux * Fy + Fx * uy) + ks * s.nx * s.ny;
    s.c.axz = one_m * m.axz + orx * uz + fh * (ux * Fz + Fx * uz) + ks * s.nx * s.nz;
    s.c.ayz = one_m * m.ayz + ory * uz + fh * (uy * Fz + Fy * uz) + ks * s.ny * s.nz;
    s.r1 = a.r1 * rinv;
    s.e = p.beta * a.r1 * (rho - a.r1) * rinv;
    return s;
}

// Gradient, near-contact test, forcing and collision of one source node of
// the z-marching kernel.  Pm, P0, Pp: phi of planes s-1, s, s+1 in shared
// memory; b = index of the node in a phi plane; the probes read phi from the
// moments in global memory (L2).
template <class L, class T, int HX2, int HN2, bool FAST>
__device__ __forceinline__ Src2<T> collide2(const Node2<T>& a, const T* __restrict__ Pm, const T* __restrict__ P0,
                                            const T* __restrict__ Pp, int b, const CGPar<T>& p,
                                            const T* __restrict__ in, const Layout& lay, int gx, int gy, int gz) {
    // isotropic gradient: sum over opposite pairs of w c (phi(+c) - phi(-c)) / cs^2
    T Gx = T(0), Gy = T(0), Gz = T(0);
    // every neighbour slot b +- (cy HX2 + cx) lies between these two
    const bool in_ring = LLB_IN(b - HX2 - 1, HN2, kChkPhi) && LLB_IN(b + HX2 + 1, HN2, kChkPhi);
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                const bool lead = cx > 0 || (cx == 0 && (cy > 0 || (cy == 0 && cz > 0)));
                if (!lead || !L::has(cx, cy, cz)) continue;
                const T* Pf = cz > 0 ? Pp : (cz < 0 ? Pm : P0);
                const T* Pb = cz > 0 ? Pm : (cz < 0 ? Pp : P0);
                if (!in_ring) continue;
                const T diff = Pf[b + cy * HX2 + cx] - Pb[b - cy * HX2 - cx];
                const T wd = T(3.0 * L::w(cx, cy, cz)) * diff;
                if (cx) Gx += T(cx) * wd;
                if (cy) Gy += T(cy) * wd;
                if (cz) Gz += T(cz) * wd;
            }
    return cg_collide<T, FAST>(a, Gx, Gy, Gz, P0[b], p, [&](int ox, int oy, int oz) {
        const size_t q = lay.at(pmod2(gx + ox, lay.nx), pmod2(gy + oy, lay.ny), pmod2(gz + oz, lay.nz));
        if (!LLB_IN(q, lay.fs, kChkProbe)) return T(0);
        return phi_of<false>(__ldg(in + q), __ldg(in + lay.fs + q));
    });
}

template <int RX, int RY>
__host__ __device__ constexpr bool wanted2(int cx, int cy) {
    return (RX == 2 || cx == RX) && (RY == 2 || cy == RY);
}

// Publish (g'_i, h1'_i) of every wanted crossing direction.  For a pair
// (c, -c): g'_{+-c} = w (q +- l) and h1'_{+-c} = r1 (w + w q) +- (r1 w l + e_c)
// with e_c = e w (c.n) / |c|.
template <class L, class T, int HN, int RX = 2, int RY = 2>
__device__ __forceinline__ void publish2(GH<T>* __restrict__ X, int n, const Src2<T>& s) {
    if (!LLB_IN(n, HN, kChkPublish)) return;
    const Mom<T>& c = s.c;
    const T s0 = g_shared(c);
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                const bool lead = cx > 0 || (cx == 0 && (cy > 0 || (cy == 0 && cz > 0)));
                if (!lead || !L::has(cx, cy, cz) || (cx == 0 && cy == 0)) continue;
                const bool wp = wanted2<RX, RY>(cx, cy), wm = wanted2<RX, RY>(-cx, -cy);
                if (!wp && !wm) continue;
                T q = s0;
                if (cx) q += T(4.5) * c.axx;
                if (cy) q += T(4.5) * c.ayy;
                if (cz) q += T(4.5) * c.azz;
                if (cx * cy) q += T(9 * cx * cy) * c.axy;
                if (cx * cz) q += T(9 * cx * cz) * c.axz;
                if (cy * cz) q += T(9 * cy * cz) * c.ayz;
                T l = T(0), cn = T(0);
                if (cx) { l += T(3 * cx) * c.jx; cn += T(cx) * s.nx; }
                if (cy) { l += T(3 * cy) * c.jy; cn += T(cy) * s.ny; }
                if (cz) { l += T(3 * cz) * c.jz; cn += T(cz) * s.nz; }
                const T w = T(L::w(cx, cy, cz));
                const T wq = w * q, wl = w * l;
                const T hb = s.r1 * (w + wq);
                const T ho = s.r1 * wl + s.e * T(L::w(cx, cy, cz) * inv_len(cx, cy, cz)) * cn;
                if (wp) X[kslot2<L>(cx, cy, cz) * HN + n] = GH<T>{wq + wl, hb + ho};
                if (wm) X[kslot2<L>(-cx, -cy, -cz) * HN + n] = GH<T>{wq - wl, hb - ho};
            }
}

// Publish the directions with c_x = sx (run-time sign) of a node of the left
// (sx = +1) or right (sx = -1) halo column or a corner: the only directions
// along which it feeds the tile.  One code path for both signs.
template <class L, class T, int HN>
__device__ __forceinline__ void publish2_side(GH<T>* __restrict__ X, int n, const Src2<T>& s, int sx) {
    if (!LLB_IN(n, HN, kChkPublish)) return;
    const Mom<T>& c = s.c;
    const T sg = T(sx);
    const T base = g_shared(c) + T(4.5) * c.axx;
    const T sxy = sg * c.axy, sxz = sg * c.axz, sjx = T(3) * sg * c.jx, snx = sg * s.nx;
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
            T l = sjx, cn = snx;
            if (cy) { l += T(3 * cy) * c.jy; cn += T(cy) * s.ny; }
            if (cz) { l += T(3 * cz) * c.jz; cn += T(cz) * s.nz; }
            const T w = T(L::w(1, cy, cz));
            const T g = w * (q + l);
            const T h = s.r1 * (w + g) + s.e * T(L::w(1, cy, cz) * inv_len(1, cy, cz)) * cn;
            const int k = sx > 0 ? kslot2<L>(1, cy, cz) : kslot2<L>(-1, cy, cz);
            X[k * HN + n] = GH<T>{g, h};
        }
}

// Accumulator of one output plane: mixture moments and rho1.
template <class T>
struct Acc2 {
    Acc<T> a;
    T r1;
    __device__ __forceinline__ void zero() {
        a.zero();
        r1 = T(0);
    }
};

template <class T, bool INIT>
__device__ __forceinline__ void acc2_to(T& a, T v) {
    if constexpr (INIT) a = v; else a += v;
}

// Pull the (g', h1') with c_z = CZ that output node n pulls from the source
// plane and add them into the accumulator of plane s + CZ (INIT: assigned).
template <class L, class T, int CZ, int HN, int HX, bool INIT = false>
__device__ __forceinline__ void add_plane2(const GH<T>* __restrict__ X, int n, T g_own, T h_own, Acc2<T>& A) {
    // every neighbour slot n - cy HX - cx lies between these two
    if (!LLB_IN(n - HX - 1, HN, kChkGather) || !LLB_IN(n + HX + 1, HN, kChkGather)) return;
#define LLB_GH(cx, cy) X[kslot2<L>(cx, cy, CZ) * HN + n - (cy) * HX - (cx)]
    static_assert(L::has(1, 0, CZ) && L::has(0, 1, CZ), "lattice without the axis-plane directions");
    const GH<T> ax = LLB_GH(1, 0), bx = LLB_GH(-1, 0), ay = LLB_GH(0, 1), by = LLB_GH(0, -1);
    const T sx = ax.g + bx.g, sy = ay.g + by.g;
    T jx = ax.g - bx.g, jy = ay.g - by.g;
    T sxx = sx, syy = sy;
    T sum = (g_own + sx) + sy;
    T r = (h_own + (ax.h + bx.h)) + (ay.h + by.h);
    T sxy = T(0);
    if constexpr (L::has(1, 1, CZ)) {
        const GH<T> pp = LLB_GH(1, 1), mm = LLB_GH(-1, -1), pm = LLB_GH(1, -1), mp = LLB_GH(-1, 1);
        const T a = pp.g + mm.g, b = pm.g + mp.g, c = pp.g - mm.g, e = pm.g - mp.g;
        const T sd = a + b;
        sum += sd;
        sxx += sd;
        syy += sd;
        sxy = a - b;
        jx += c + e;
        jy += c - e;
        r += (pp.h + mm.h) + (pm.h + mp.h);
    }
#undef LLB_GH
    acc2_to<T, INIT>(A.a.d, sum);
    acc2_to<T, INIT>(A.a.jx, jx);
    acc2_to<T, INIT>(A.a.jy, jy);
    acc2_to<T, INIT>(A.a.sxx, sxx);
    acc2_to<T, INIT>(A.a.syy, syy);
    acc2_to<T, INIT>(A.a.sxy, sxy);
    acc2_to<T, INIT>(A.r1, r);
    if constexpr (CZ != 0) {
        acc2_to<T, INIT>(A.a.szz, sum);
        if constexpr (CZ > 0) {
            acc2_to<T, INIT>(A.a.jz, sum);
            acc2_to<T, INIT>(A.a.sxz, jx);
            acc2_to<T, INIT>(A.a.syz, jy);
        } else {
            static_assert(!INIT, "only the plane ahead starts here");
            A.a.jz -= sum;
            A.a.sxz -= jx;
            A.a.syz -= jy;
        }
    } else {
        static_assert(!INIT, "only the plane ahead starts here");
    }
}

template <int BX, int BY>
__device__ __forceinline__ int halo_role2(int t, int& hx, int& hy, int& sx) {
    // 0 none, 1 top (c_y = +1 only), 2 bottom (c_y = -1 only), 3 side/corner (c_x = sx only)
    sx = 1;
    if (t < BX) { hx = t + 1; hy = 0; return 1; }
    if (t < 2 * BX) { hx = t - BX + 1; hy = BY + 1; return 2; }
    const int s = t - 2 * BX;
    if (s < BY) { hx = 0; hy = s + 1; return 3; }
    if (s < 2 * BY) { hx = BX + 1; hy = s - BY + 1; sx = -1; return 3; }
    switch (s - 2 * BY) {
        case 0: hx = 0; hy = 0; return 3;
        case 1: hx = BX + 1; hy = 0; sx = -1; return 3;
        case 2: hx = 0; hy = BY + 1; return 3;
        case 3: hx = BX + 1; hy = BY + 1; sx = -1; return 3;
        default: hx = 0; hy = 0; return 0;
    }
}

struct Sched2 {
    int ncx, ntiles, zc, nitems;
};
static_assert(sizeof(Sched2) == 4 * sizeof(int), "schedule layout");

template <class L, class T, int BX, int BY>
struct CGCfg {
    static constexpr int NT = BX * BY;
    static constexpr int HX1 = BX + 2, HY1 = BY + 2, HN1 = HX1 * HY1;  // sources: tile + 1 halo
    static constexpr int HX2 = BX + 4, HY2 = BY + 4, HN2 = HX2 * HY2;  // phi: tile + 2 halo
    static constexpr int NS = n_xy_shifted<L>();
    static constexpr size_t smem_bytes = sizeof(GH<T>) * (size_t)NS * HN1 + sizeof(T) * 3 * (size_t)HN2;
    static_assert(2 * BX + 2 * BY + 4 <= NT, "halo must fit one node per thread");
    static constexpr int NJ = (HN2 + NT - 1) / NT;  // phi nodes per thread
    static_assert(NJ <= 3, "phi region must fit three nodes per thread");
};

// One work item (z-chunk of one tile) of the two-component step; the items
// cover output planes zlo .. zlo + nzr - 1 (the whole box: 0, nz).  Called by
// every thread of the CTA (it synchronises the CTA).
template <class L, class T, int BX, int BY, bool FAST, bool ROLLED>
__device__ __forceinline__ void cg_item(const T* __restrict__ in, T* __restrict__ out, const Layout& lay,
                                        const CGPar<T>& prm, const Sched2& sc, int it, int zlo, int nzr) {
    using C = CGCfg<L, T, BX, BY>;
    constexpr int NT = C::NT, HX1 = C::HX1, HN1 = C::HN1, HX2 = C::HX2, HN2 = C::HN2, NS = C::NS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GH<T>* const XG = reinterpret_cast<GH<T>*>(smem_raw);
    T* const PH = reinterpret_cast<T*>(XG + NS * HN1);  // 3 planes of phi
    const int nx = lay.nx, ny = lay.ny, nz = lay.nz;
    const size_t plane = (size_t)lay.px * lay.py, fs = lay.fs;

    const int t = threadIdx.x;
    const int tx = t % BX, ty = t / BX;
    const int n1 = (ty + 1) * HX1 + (tx + 1);
    const int b1 = (ty + 2) * HX2 + (tx + 2);  // own node in a phi plane
    int hx2, hy2, sx2;
    const int role2 = halo_role2<BX, BY>(t, hx2, hy2, sx2);
    const int n2 = hy2 * HX1 + hx2;
    const int b2 = (hy2 + 1) * HX2 + (hx2 + 1);
    // phi nodes of this thread: j = t + q NT (q < NJ) inside the tile + 2 halo
    constexpr int NJ = C::NJ;

    const int chunk = it / sc.ntiles, tile = it - chunk * sc.ntiles;
    const int x0 = (tile % sc.ncx) * BX, y0 = (tile / sc.ncx) * BY;
    const int za = zlo + chunk * sc.zc, zb = min(zlo + nzr, za + sc.zc);
    const bool store_ok = (x0 + tx < nx) && (y0 + ty < ny);
    const int gx1 = pmod2(x0 + tx, nx), gy1 = pmod2(y0 + ty, ny);
    const int gx2 = pmod2(x0 - 1 + hx2, nx), gy2 = pmod2(y0 - 1 + hy2, ny);
    const size_t off1 = lay.at(gx1, gy1, 0), off2 = lay.at(gx2, gy2, 0);
    size_t offj[NJ];
#pragma unroll
    for (int q = 0; q < NJ; ++q) {
        const int j = t + q * NT;
        offj[q] = j < HN2 ? lay.at(pmod2(x0 - 2 + j % HX2, nx), pmod2(y0 - 2 + j / HX2, ny), 0) : 0;
    }

    // phi of planes za-2, za-1, za into ring slots 0, 1, 2 (slot of plane p: (p - za + 2) % 3)
    for (int pz = 0; pz < 3; ++pz) {
        const size_t zo = (size_t)pmod2(za - 2 + pz, nz) * plane;
#pragma unroll
        for (int q = 0; q < NJ; ++q)
            if (t + q * NT < HN2 && LLB_IN(zo + offj[q], fs, kChkLoad))
                PH[pz * HN2 + t + q * NT] = phi_of<FAST>(__ldg(in + zo + offj[q]), __ldg(in + fs + zo + offj[q]));
    }
    // registers: phi inputs of plane za+1, moments of source plane za-1
    T pr1[NJ], pd[NJ];
    {
        const size_t zo = (size_t)pmod2(za + 1, nz) * plane;
#pragma unroll
        for (int q = 0; q < NJ; ++q) {
            pr1[q] = T(0);
            pd[q] = T(0);
            if (t + q * NT < HN2 && LLB_IN(zo + offj[q], fs, kChkLoad)) {
                pr1[q] = __ldg(in + zo + offj[q]);
                pd[q] = __ldg(in + fs + zo + offj[q]);
            }
        }
    }
    // wrapped plane indices, advanced without division: zs = source plane s,
    // z1 = s + 1, z3 = s + 3; ring slots of planes s - 1, s, s + 1
    int zs = pmod2(za - 1, nz);
    int z1 = zs + 1 == nz ? 0 : zs + 1;
    int z3 = pmod2(za + 2, nz);
    Node2<T> m1 = load_node2(in, (size_t)zs * plane + off1, fs);
    Node2<T> m2 = m1;
    if (role2) m2 = load_node2(in, (size_t)zs * plane + off2, fs);
    int sm = 0, s0i = 1, sp = 2;
    const int ox = x0 + tx, oy = y0 + ty;
    const bool ghost = store_ok && (ox < kGhostX || ox >= nx - kGhostX || oy < lay.yo || oy >= ny - lay.yo);
    T* out1 = out + (store_ok ? lay.at(ox, oy, za) : 0);

    Acc2<T> a0, a1, a2;
    a0.zero();
    a1.zero();
    a2.zero();
    __syncthreads();

    // One source plane s: X, Y, Z accumulate output planes s-1, s, s+1 (Z starts here).
    //   (a) collide the source nodes of plane s (phi of planes s-1, s, s+1 are
    //       in the ring) and publish; the moments of plane s+1 are loaded into
    //       the registers just freed, a whole step ahead of their use;
    //   barrier: the exchange buffer is complete;
    //   (b) phi of plane s+2 into the ring slot of plane s-1 (no longer read),
    //       and the loads of plane s+3's phi inputs;
    //   (c) pull and store;
    //   barrier: the exchange buffer is free and phi of plane s+2 is visible.
    auto plane_step = [&](int s, Acc2<T>& X, Acc2<T>& Y, Acc2<T>& Z) {
        const bool more = s + 1 <= zb;
        const T* Pm = PH + sm * HN2;
        const T* P0 = PH + s0i * HN2;
        const T* Pp = PH + sp * HN2;
        const Src2<T> c1 = collide2<L, T, HX2, HN2, FAST>(m1, Pm, P0, Pp, b1, prm, in, lay, gx1, gy1, zs);
        if (more) m1 = load_node2(in, (size_t)z1 * plane + off1, fs);
        publish2<L, T, HN1>(XG, n1, c1);
        // own column (c_x = c_y = 0)
        const T s0 = g_shared(c1.c);
        const T wz = T(L::w(0, 0, 1)), w0 = T(L::w(0, 0, 0));
        const T wq = wz * (s0 + T(4.5) * c1.c.azz), wl = wz * (T(3) * c1.c.jz);
        const T g_p = wq + wl, g_m = wq - wl, g_0 = w0 * s0;
        const T ez = c1.e * wz * c1.nz;
        const T hb = c1.r1 * (wz + wq), ho = c1.r1 * wl + ez;
        const T h_p = hb + ho, h_m = hb - ho, h_0 = c1.r1 * (w0 + g_0);
        if (role2) {
            const Src2<T> c2 = collide2<L, T, HX2, HN2, FAST>(m2, Pm, P0, Pp, b2, prm, in, lay, gx2, gy2, zs);
            if (more) m2 = load_node2(in, (size_t)z1 * plane + off2, fs);
            if (role2 == 1) publish2<L, T, HN1, 2, 1>(XG, n2, c2);
            else if (role2 == 2) publish2<L, T, HN1, 2, -1>(XG, n2, c2);
            else publish2_side<L, T, HN1>(XG, n2, c2, sx2);
        }
        __syncthreads();
        if (more) {  // step s+1 exists and needs phi of plane s+2
#pragma unroll
            for (int q = 0; q < NJ; ++q)
                if (t + q * NT < HN2) PH[sm * HN2 + t + q * NT] = phi_of<FAST>(pr1[q], pd[q]);
            if (s + 2 <= zb) {  // step s+2 exists and needs phi of plane s+3
                const size_t zq = (size_t)z3 * plane;
#pragma unroll
                for (int q = 0; q < NJ; ++q)
                    if (t + q * NT < HN2 && LLB_IN(zq + offj[q], fs, kChkLoad)) {
                        pr1[q] = __ldg(in + zq + offj[q]);
                        pd[q] = __ldg(in + fs + zq + offj[q]);
                    }
            }
        }
        add_plane2<L, T, -1, HN1, HX1>(XG, n1, g_m, h_m, X);
        add_plane2<L, T, 0, HN1, HX1>(XG, n1, g_0, h_0, Y);
        add_plane2<L, T, 1, HN1, HX1, true>(XG, n1, g_p, h_p, Z);
        if (s - 1 >= za && store_ok) {
            const Mom<T> r = X.a.finish();
            if (LLB_IN(out1 - out, fs, kChkStore)) store_node2_at(out1, fs, X.r1, r);
            if (ghost) store_node2(out, lay, ox, oy, s - 1, X.r1, r);
            out1 += plane;
        }
        __syncthreads();
        zs = z1;
        z1 = z1 + 1 == nz ? 0 : z1 + 1;
        z3 = z3 + 1 == nz ? 0 : z3 + 1;
        const int tmp = sm;
        sm = s0i;
        s0i = sp;
        sp = tmp;
    };

    int s = za - 1;
    if constexpr (ROLLED) {
        // one copy of the plane step in the loop (a third of the code of the
        // unrolled form, for the instruction cache), accumulators rotated by copies
        for (;;) {
            plane_step(s, a0, a1, a2);
            if (++s > zb) break;
            a0 = a1;
            a1 = a2;
        }
    } else {
        for (;;) {
            plane_step(s, a0, a1, a2);
            if (++s > zb) break;
            plane_step(s, a1, a2, a0);
            if (++s > zb) break;
            plane_step(s, a2, a0, a1);
            if (++s > zb) break;
        }
    }
}

template <class L, class T, int BX, int BY, int MINB, bool FAST, bool ROLLED>
__global__ void __launch_bounds__(BX * BY, MINB)
    k_cg_tiled(const T* __restrict__ in, T* __restrict__ out, Layout lay, CGPar<T> prm, Sched2 sc, int zlo, int nzr) {
    for (int it = blockIdx.x; it < sc.nitems; it += gridDim.x)
        cg_item<L, T, BX, BY, FAST, ROLLED>(in, out, lay, prm, sc, it, zlo, nzr);
}

// Batched ensemble: the items of every box, box after box, in one persistent
// launch; a CTA finds the box of each item by binary search on item_begin.
template <class L, class T, int BX, int BY, int MINB, bool FAST, bool ROLLED>
__global__ void __launch_bounds__(BX * BY, MINB)
    k_cg_batch(const BatchDom* __restrict__ doms, int ndom, int total, CGPar<T> prm, int* __restrict__ next) {
    // work queue: each CTA takes the next item when it is done with one, so that
    // items of different lengths (boxes of different sizes) even out over the grid
    __shared__ int s_it;
    for (;;) {
        if (threadIdx.x == 0) s_it = atomicAdd(next, 1);
        __syncthreads();
        const int it = s_it;
        __syncthreads();  // every thread has read s_it before it is overwritten
        if (it >= total) break;
        int lo = 0, hi = ndom - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (doms[mid].item_begin <= it) lo = mid;
            else hi = mid - 1;
        }
        const BatchDom d = doms[lo];
        Sched2 sc;
        sc.ncx = d.ncx;
        sc.ntiles = d.ntiles;
        sc.zc = d.zc;
        sc.nitems = d.nitems;
        cg_item<L, T, BX, BY, FAST, ROLLED>(static_cast<const T*>(d.in), static_cast<T*>(d.out), d.lay, prm, sc,
                                    it - d.item_begin, 0, d.lay.nz);
    }
}

inline Sched2 plan2(int nx, int ny, int nz, int BX, int BY, int grid) {
    Sched2 s;
    s.ncx = (nx + BX - 1) / BX;
    s.ntiles = s.ncx * ((ny + BY - 1) / BY);
    long long best = -1;
    for (int nch = 1; nch <= nz; ++nch) {
        const int zc = (nz + nch - 1) / nch;
        const int chunks = (nz + zc - 1) / zc;
        const long long items = (long long)s.ntiles * chunks;
        if (items > (1LL << 30)) break;
        const long long rounds = (items + grid - 1) / grid;
        const long long cost = rounds * (zc + 3);
        if (best < 0 || cost < best) {
            best = cost;
            s.zc = zc;
            s.nitems = (int)items;
        }
    }
    return s;
}

// Two-component kernel shapes: tile BX x BY, CTAs per SM, approximate FP32
// divisions (phi, 1/rho, 1/|G|).  Variant 0 is the default.
template <int BX_, int BY_, int MINB_, bool FAST_, bool ROLLED_ = false>
struct CGShape {
    static constexpr int BX = BX_, BY = BY_, MINB = MINB_;
    static constexpr bool FAST = FAST_, ROLLED = ROLLED_;
};
// The approximate quotients measured 18 % (D3Q27) to 23 % (D3Q19) faster on
// the 384 x 192 x 192 droplet pair and stay within the FP32 parity bound; the
// rolled plane loop a further 10 % on D3Q27 (fewer instruction-cache misses)
// and 1 % slower on D3Q19.
template <class T, int V> struct CGVariant { using type = CGShape<32, 8, 2, true, true>; };
template <> struct CGVariant<float, 1> { using type = CGShape<64, 4, 2, false>; };
template <> struct CGVariant<float, 2> { using type = CGShape<32, 8, 2, false>; };
template <> struct CGVariant<float, 3> { using type = CGShape<32, 16, 1, false>; };
template <> struct CGVariant<float, 4> { using type = CGShape<32, 8, 2, true>; };
template <> struct CGVariant<float, 5> { using type = CGShape<64, 4, 2, true, true>; };
// FP64 (parity runs): one shape, one CTA per SM (its exchange buffers take
// more than half of an SM's shared memory), so the full register file is there
template <int V> struct CGVariant<double, V> { using type = CGShape<32, 8, 1, false>; };

template <class T>
CGPar<T> cg_params(const llb_ctx& c) {
    CGPar<T> p;
    p.omega = (T)c.omega;
    p.beta = (T)c.params.beta;
    p.A_s = (T)c.params.A_s;
    p.A_h = (T)c.params.A_h;
    p.g_min = (T)c.params.g_min;
    p.g_nci = (T)kGNci;
    p.eps2 = (T)(c.params.grad_eps * c.params.grad_eps);
    p.h_c = c.params.h_c;
    return p;
}

// (lattice, element type, variant) -> instance.
#define LLB_CG_V(fn, L, T, ...)                                                                    \
    switch (c.variant) {                                                                           \
        case 1: return fn<L, T, typename CGVariant<T, 1>::type>(__VA_ARGS__);                      \
        case 2: return fn<L, T, typename CGVariant<T, 2>::type>(__VA_ARGS__);                      \
        case 3: return fn<L, T, typename CGVariant<T, 3>::type>(__VA_ARGS__);                      \
        case 4: return fn<L, T, typename CGVariant<T, 4>::type>(__VA_ARGS__);                      \
        case 5: return fn<L, T, typename CGVariant<T, 5>::type>(__VA_ARGS__);                      \
        default: return fn<L, T, typename CGVariant<T, 0>::type>(__VA_ARGS__);                     \
    }
#define LLB_CG(fn, ...)                                                                            \
    if (c.Q == 19) {                                                                               \
        if (c.storage == LLB_F64) { LLB_CG_V(fn, D3Q19, double, __VA_ARGS__) }                     \
        LLB_CG_V(fn, D3Q19, float, __VA_ARGS__)                                                    \
    }                                                                                              \
    if (c.storage == LLB_F64) { LLB_CG_V(fn, D3Q27, double, __VA_ARGS__) }                         \
    LLB_CG_V(fn, D3Q27, float, __VA_ARGS__)

}  // namespace cg
}  // namespace llb
