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
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "lattice.cuh"
#include "layout.cuh"

namespace llb {
namespace {

constexpr float kPhiRise = 0.01f;  // phi rise at a probe that signals another interface
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
    Node2<T> a;
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

template <class T>
__device__ __forceinline__ T phi_of(T r1, T d) {
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

// Collided source node: moments after collision and the colour quantities.
template <class T>
struct Src2 {
    Mom<T> c;     // d, j' = j + F, A'
    T r1;         // rho1 / rho
    T e;          // beta rho1 rho2 / rho
    T nx, ny, nz; // unit normal (0 off the interface)
};

// Gradient, near-contact test, forcing and collision of one source node.
// P: phi of planes s-1, s, s+1 (HN2 each), b = index of the node in a phi plane.
template <class L, class T, int HX2, int HN2>
__device__ __forceinline__ Src2<T> collide2(const Node2<T>& a, const T* __restrict__ Pm, const T* __restrict__ P0,
                                            const T* __restrict__ Pp, int b, const CGPar<T>& p,
                                            const T* __restrict__ in, const Layout& lay, int gx, int gy, int gz) {
    // isotropic gradient: sum over opposite pairs of w c (phi(+c) - phi(-c)) / cs^2
    T Gx = T(0), Gy = T(0), Gz = T(0);
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
                const T diff = Pf[b + cy * HX2 + cx] - Pb[b - cy * HX2 - cx];
                const T wd = T(3.0 * L::w(cx, cy, cz)) * diff;
                if (cx) Gx += T(cx) * wd;
                if (cy) Gy += T(cy) * wd;
                if (cz) Gz += T(cz) * wd;
            }
    const T g2 = Gx * Gx + Gy * Gy + Gz * Gz;
    const bool smooth = p.eps2 > T(0);
    const T gn = sqrt(smooth ? g2 + p.eps2 : g2);
    const bool has_n = smooth || gn >= p.g_min;
    Src2<T> s;
    s.nx = s.ny = s.nz = T(0);
    if (has_n) {
        const T ig = T(1) / gn;
        s.nx = Gx * ig;
        s.ny = Gy * ig;
        s.nz = Gz * ig;
    }
    // near-contact detector on the interface band (phi read from L2 for the probes)
    T Fx = T(0), Fy = T(0), Fz = T(0);
    if (p.A_h != T(0) && gn >= p.g_nci) {
        const T phi0 = P0[b];
        bool near = false;
        for (int k = 1; k <= p.h_c && !near; ++k) {
            const int ox = (int)rint(-T(k) * s.nx), oy = (int)rint(-T(k) * s.ny), oz = (int)rint(-T(k) * s.nz);
            const size_t q = lay.at(pmod2(gx + ox, lay.nx), pmod2(gy + oy, lay.ny), pmod2(gz + oz, lay.nz));
            const T ph = phi_of(__ldg(in + q), __ldg(in + lay.fs + q));
            near = ph > phi0 + T(kPhiRise);
        }
        if (near) {
            Fx = p.A_h * Gx;
            Fy = p.A_h * Gy;
            Fz = p.A_h * Gz;
        }
    }
    const Mom<T>& m = a.m;
    const T rho = T(1) + m.d;
    const T rinv = T(1) / rho;
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

template <int RX, int RY>
__host__ __device__ constexpr bool wanted2(int cx, int cy) {
    return (RX == 2 || cx == RX) && (RY == 2 || cy == RY);
}

// Publish g'_i and h1'_i of every wanted crossing direction.
template <class L, class T, int HN, int RX = 2, int RY = 2>
__device__ __forceinline__ void publish2(T* __restrict__ Gg, T* __restrict__ Gh, int n, const Src2<T>& s) {
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
                const T gp = wq + wl, gm = wq - wl;
                const T ec = s.e * w * T(inv_len(cx, cy, cz)) * cn;
                if (wp) {
                    const int k = kslot2<L>(cx, cy, cz);
                    Gg[k * HN + n] = gp;
                    Gh[k * HN + n] = s.r1 * (w + gp) + ec;
                }
                if (wm) {
                    const int k = kslot2<L>(-cx, -cy, -cz);
                    Gg[k * HN + n] = gm;
                    Gh[k * HN + n] = s.r1 * (w + gm) - ec;
                }
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

// Pull the populations with c_z = CZ that output node n pulls from the
// source plane and add them into the accumulator of plane s + CZ.
template <class L, class T, int CZ, int HN, int HX>
__device__ __forceinline__ void add_plane2(const T* __restrict__ Gg, const T* __restrict__ Gh, int n, T g_own,
                                           T h_own, Acc2<T>& A) {
#define LLB_G(cx, cy) Gg[kslot2<L>(cx, cy, CZ) * HN + n - (cy) * HX - (cx)]
#define LLB_H(cx, cy) Gh[kslot2<L>(cx, cy, CZ) * HN + n - (cy) * HX - (cx)]
    T sum = g_own, jx = T(0), jy = T(0), sxx = T(0), syy = T(0), sxy = T(0), r = h_own;
    if (L::has(1, 0, CZ)) {
        const T a = LLB_G(1, 0), b = LLB_G(-1, 0);
        sum += a + b;
        sxx += a + b;
        jx += a - b;
        r += LLB_H(1, 0) + LLB_H(-1, 0);
    }
    if (L::has(0, 1, CZ)) {
        const T a = LLB_G(0, 1), b = LLB_G(0, -1);
        sum += a + b;
        syy += a + b;
        jy += a - b;
        r += LLB_H(0, 1) + LLB_H(0, -1);
    }
    if (L::has(1, 1, CZ)) {
        const T pp = LLB_G(1, 1), mm = LLB_G(-1, -1), pm = LLB_G(1, -1), mp = LLB_G(-1, 1);
        const T a = pp + mm, b = pm + mp, c = pp - mm, e = pm - mp;
        const T s = a + b;
        sum += s;
        sxx += s;
        syy += s;
        sxy += a - b;
        jx += c + e;
        jy += c - e;
        r += (LLB_H(1, 1) + LLB_H(-1, -1)) + (LLB_H(1, -1) + LLB_H(-1, 1));
    }
#undef LLB_G
#undef LLB_H
    A.a.d += sum;
    A.a.jx += jx;
    A.a.jy += jy;
    A.a.sxx += sxx;
    A.a.syy += syy;
    A.a.sxy += sxy;
    A.r1 += r;
    if (CZ != 0) {
        A.a.szz += sum;
        if (CZ > 0) {
            A.a.jz += sum;
            A.a.sxz += jx;
            A.a.syz += jy;
        } else {
            A.a.jz -= sum;
            A.a.sxz -= jx;
            A.a.syz -= jy;
        }
    }
}

template <int BX, int BY>
__device__ __forceinline__ int halo_role2(int t, int& hx, int& hy) {
    // 0 none, 1 top (c_y = +1 only), 2 bottom (c_y = -1 only), 3 side/corner (all)
    if (t < BX) { hx = t + 1; hy = 0; return 1; }
    if (t < 2 * BX) { hx = t - BX + 1; hy = BY + 1; return 2; }
    const int s = t - 2 * BX;
    if (s < BY) { hx = 0; hy = s + 1; return 3; }
    if (s < 2 * BY) { hx = BX + 1; hy = s - BY + 1; return 3; }
    switch (s - 2 * BY) {
        case 0: hx = 0; hy = 0; return 3;
        case 1: hx = BX + 1; hy = 0; return 3;
        case 2: hx = 0; hy = BY + 1; return 3;
        case 3: hx = BX + 1; hy = BY + 1; return 3;
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
    static constexpr size_t smem_bytes = sizeof(T) * (2 * (size_t)NS * HN1 + 3 * (size_t)HN2);
    static_assert(2 * BX + 2 * BY + 4 <= NT, "halo must fit one node per thread");
    static constexpr int NJ = (HN2 + NT - 1) / NT;  // phi nodes per thread
    static_assert(NJ <= 3, "phi region must fit three nodes per thread");
};

// One work item (z-chunk of one tile) of the two-component step.  Called by
// every thread of the CTA (it synchronises the CTA).
template <class L, class T, int BX, int BY>
__device__ __forceinline__ void cg_item(const T* __restrict__ in, T* __restrict__ out, const Layout& lay,
                                        const CGPar<T>& prm, const Sched2& sc, int it) {
    using C = CGCfg<L, T, BX, BY>;
    constexpr int NT = C::NT, HX1 = C::HX1, HN1 = C::HN1, HX2 = C::HX2, HN2 = C::HN2, NS = C::NS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* const Gg = reinterpret_cast<T*>(smem_raw);
    T* const Gh = Gg + NS * HN1;
    T* const PH = Gh + NS * HN1;  // 3 planes of phi
    const int nx = lay.nx, ny = lay.ny, nz = lay.nz;
    const size_t plane = (size_t)lay.px * lay.py, fs = lay.fs;

    const int t = threadIdx.x;
    const int tx = t % BX, ty = t / BX;
    const int n1 = (ty + 1) * HX1 + (tx + 1);
    const int b1 = (ty + 2) * HX2 + (tx + 2);  // own node in a phi plane
    int hx2, hy2;
    const int role2 = halo_role2<BX, BY>(t, hx2, hy2);
    const int n2 = hy2 * HX1 + hx2;
    const int b2 = (hy2 + 1) * HX2 + (hx2 + 1);
    // phi nodes of this thread: j = t + q NT (q < NJ) inside the tile + 2 halo
    constexpr int NJ = C::NJ;

    {
        const int chunk = it / sc.ntiles, tile = it - chunk * sc.ntiles;
        const int x0 = (tile % sc.ncx) * BX, y0 = (tile / sc.ncx) * BY;
        const int za = chunk * sc.zc, zb = min(nz, za + sc.zc);
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

        // phi of planes za-2 and za-1 into ring slots 0 and 1 (slot of plane p: (p - za + 2) % 3)
        for (int pz = 0; pz < 2; ++pz) {
            const size_t zo = (size_t)pmod2(za - 2 + pz, nz) * plane;
#pragma unroll
            for (int q = 0; q < NJ; ++q)
                if (t + q * NT < HN2)
                    PH[pz * HN2 + t + q * NT] = phi_of(__ldg(in + zo + offj[q]), __ldg(in + fs + zo + offj[q]));
        }
        // registers: phi inputs of plane za, moments of source plane za-1
        size_t zo = (size_t)pmod2(za, nz) * plane;
        T pr1[NJ], pd[NJ];
#pragma unroll
        for (int q = 0; q < NJ; ++q) {
            pr1[q] = T(0);
            pd[q] = T(0);
            if (t + q * NT < HN2) {
                pr1[q] = __ldg(in + zo + offj[q]);
                pd[q] = __ldg(in + fs + zo + offj[q]);
            }
        }
        zo = (size_t)pmod2(za - 1, nz) * plane;
        Node2<T> m1 = load_node2(in, zo + off1, fs);
        Node2<T> m2 = m1;
        if (role2) m2 = load_node2(in, zo + off2, fs);

        Acc2<T> X, Y, Z;
        X.zero(); Y.zero(); Z.zero();
        // wrapped plane indices, advanced without division: zs = source plane s,
        // z1 = s + 1, z2 = s + 2; ring slots of planes s - 1, s, s + 1
        int zs = pmod2(za - 1, nz);
        int z1 = zs + 1 == nz ? 0 : zs + 1;
        int z2 = z1 + 1 == nz ? 0 : z1 + 1;
        int sm = 0, s0i = 1, sp = 2;
        const int ox = x0 + tx, oy = y0 + ty;
        const bool ghost = store_ok && (ox < kGhostX || ox >= nx - kGhostX || oy < lay.yo || oy >= ny - lay.yo);
        T* out1 = out + (store_ok ? lay.at(ox, oy, za) : 0);
        for (int s = za - 1; s <= zb; ++s) {
            // (a) phi of plane s+1 from registers; prefetch for the next plane
#pragma unroll
            for (int q = 0; q < NJ; ++q)
                if (t + q * NT < HN2) PH[sp * HN2 + t + q * NT] = phi_of(pr1[q], pd[q]);
            Node2<T> n1next = m1, n2next = m2;
            if (s + 1 <= zb) {
                const size_t zq = (size_t)z2 * plane;
#pragma unroll
                for (int q = 0; q < NJ; ++q)
                    if (t + q * NT < HN2) {
                        pr1[q] = __ldg(in + zq + offj[q]);
                        pd[q] = __ldg(in + fs + zq + offj[q]);
                    }
                const size_t zn = (size_t)z1 * plane;
                n1next = load_node2(in, zn + off1, fs);
                if (role2) n2next = load_node2(in, zn + off2, fs);
            }
            __syncthreads();
            // (b) collide the source nodes of plane s and publish
            const T* Pm = PH + sm * HN2;
            const T* P0 = PH + s0i * HN2;
            const T* Pp = PH + sp * HN2;
            const Src2<T> c1 = collide2<L, T, HX2, HN2>(m1, Pm, P0, Pp, b1, prm, in, lay, gx1, gy1, zs);
            publish2<L, T, HN1>(Gg, Gh, n1, c1);
            // own column (c_x = c_y = 0)
            const T s0 = g_shared(c1.c);
            const T wz = T(L::w(0, 0, 1)), w0 = T(L::w(0, 0, 0));
            const T wq = wz * (s0 + T(4.5) * c1.c.azz), wl = wz * (T(3) * c1.c.jz);
            const T g_p = wq + wl, g_m = wq - wl, g_0 = w0 * s0;
            const T ez = c1.e * wz * c1.nz;
            const T h_p = c1.r1 * (wz + g_p) + ez, h_m = c1.r1 * (wz + g_m) - ez, h_0 = c1.r1 * (w0 + g_0);
            if (role2) {
                const Src2<T> c2 = collide2<L, T, HX2, HN2>(m2, Pm, P0, Pp, b2, prm, in, lay, gx2, gy2, zs);
                if (role2 == 1) publish2<L, T, HN1, 2, 1>(Gg, Gh, n2, c2);
                else if (role2 == 2) publish2<L, T, HN1, 2, -1>(Gg, Gh, n2, c2);
                else publish2<L, T, HN1>(Gg, Gh, n2, c2);
            }
            __syncthreads();
            // (c) pull into the accumulators of planes s-1 (X), s (Y), s+1 (Z)
            Z.zero();
            add_plane2<L, T, -1, HN1, HX1>(Gg, Gh, n1, g_m, h_m, X);
            add_plane2<L, T, 0, HN1, HX1>(Gg, Gh, n1, g_0, h_0, Y);
            add_plane2<L, T, 1, HN1, HX1>(Gg, Gh, n1, g_p, h_p, Z);
            if (s - 1 >= za && store_ok) {
                const Mom<T> r = X.a.finish();
                store_node2_at(out1, fs, X.r1, r);
                if (ghost) store_node2(out, lay, ox, oy, s - 1, X.r1, r);
                out1 += plane;
            }
            X = Y;
            Y = Z;
            m1 = n1next;
            m2 = n2next;
            zs = z1;
            z1 = z2;
            z2 = z2 + 1 == nz ? 0 : z2 + 1;
            const int tmp = sm;
            sm = s0i;
            s0i = sp;
            sp = tmp;
        }
        __syncthreads();  // the phi ring and exchange buffers are reused by the next item
    }
}

template <class L, class T, int BX, int BY>
__global__ void __launch_bounds__(BX * BY, 2)
    k_cg_tiled(const T* __restrict__ in, T* __restrict__ out, Layout lay, CGPar<T> prm, Sched2 sc) {
    for (int it = blockIdx.x; it < sc.nitems; it += gridDim.x) cg_item<L, T, BX, BY>(in, out, lay, prm, sc, it);
}

// Batched ensemble: the items of every box, box after box, in one persistent
// launch; a CTA finds the box of each item by binary search on item_begin.
template <class L, class T, int BX, int BY>
__global__ void __launch_bounds__(BX * BY, 2)
    k_cg_batch(const BatchDom* __restrict__ doms, int ndom, int total, CGPar<T> prm) {
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
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
        cg_item<L, T, BX, BY>(static_cast<const T*>(d.in), static_cast<T*>(d.out), d.lay, prm, sc,
                              it - d.item_begin);
    }
}

Sched2 plan2(int nx, int ny, int nz, int BX, int BY, int grid) {
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

template <class L, class T, int kBX2, int kBY2>
int cg_ctas_v(const llb_ctx& c) {
    using C = CGCfg<L, T, kBX2, kBY2>;
    auto kern = k_cg_tiled<L, T, kBX2, kBY2>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_bytes) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, C::smem_bytes) != cudaSuccess ||
        per_sm < 1)
        return 0;
    const Sched2 sc = plan2(c.nx, c.ny, c.nz, kBX2, kBY2, per_sm * c.num_sms);
    return std::min(sc.nitems, per_sm * c.num_sms);
}

template <class L, class T, int kBX2, int kBY2>
cudaError_t cg_run_v(const llb_ctx& c, const void* in, void* out) {
    using C = CGCfg<L, T, kBX2, kBY2>;
    const int grid = c.tile_ctas > 0 ? c.tile_ctas : 1;
    const Sched2 sc = plan2(c.nx, c.ny, c.nz, kBX2, kBY2, grid);
    CGPar<T> p;
    p.omega = (T)c.omega;
    p.beta = (T)c.params.beta;
    p.A_s = (T)c.params.A_s;
    p.A_h = (T)c.params.A_h;
    p.g_min = (T)c.params.g_min;
    p.g_nci = (T)kGNci;
    p.eps2 = (T)(c.params.grad_eps * c.params.grad_eps);
    p.h_c = c.params.h_c;
    k_cg_tiled<L, T, kBX2, kBY2><<<grid, C::NT, C::smem_bytes, c.stream>>>(
        static_cast<const T*>(in), static_cast<T*>(out), c.lay, p, sc);
    return cudaGetLastError();
}

template <class L, class T, int kBX2, int kBY2>
int cg_batch_ctas_v(const llb_ctx& c) {
    using C = CGCfg<L, T, kBX2, kBY2>;
    auto kern = k_cg_batch<L, T, kBX2, kBY2>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_bytes) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, C::smem_bytes) != cudaSuccess ||
        per_sm < 1)
        return 0;
    return per_sm * c.num_sms;
}

template <class L, class T, int kBX2, int kBY2>
void cg_batch_plan_v(int nx, int ny, int nz, int grid, BatchDom* d) {
    const Sched2 sc = plan2(nx, ny, nz, kBX2, kBY2, grid);
    d->ncx = sc.ncx;
    d->ntiles = sc.ntiles;
    d->zc = sc.zc;
    d->nitems = sc.nitems;
}

template <class L, class T, int kBX2, int kBY2>
cudaError_t cg_batch_run_v(const llb_ctx& c, const BatchDom* doms, int ndom, int total, int grid) {
    using C = CGCfg<L, T, kBX2, kBY2>;
    CGPar<T> p;
    p.omega = (T)c.omega;
    p.beta = (T)c.params.beta;
    p.A_s = (T)c.params.A_s;
    p.A_h = (T)c.params.A_h;
    p.g_min = (T)c.params.g_min;
    p.g_nci = (T)kGNci;
    p.eps2 = (T)(c.params.grad_eps * c.params.grad_eps);
    p.h_c = c.params.h_c;
    k_cg_batch<L, T, kBX2, kBY2><<<grid, C::NT, C::smem_bytes, c.stream>>>(doms, ndom, total, p);
    return cudaGetLastError();
}

// Tile shapes: variant 0 = 64 x 4 (default), 1 = 32 x 8.
template <class L, class T>
int cg_ctas_t(const llb_ctx& c) {
    return c.variant == 1 ? cg_ctas_v<L, T, 32, 8>(c) : cg_ctas_v<L, T, 64, 4>(c);
}
template <class L, class T>
cudaError_t cg_run_t(const llb_ctx& c, const void* in, void* out) {
    return c.variant == 1 ? cg_run_v<L, T, 32, 8>(c, in, out) : cg_run_v<L, T, 64, 4>(c, in, out);
}

}  // namespace

int cg_tiled_ctas(const llb_ctx& c) {
    if (c.Q == 19) return c.storage == LLB_F64 ? cg_ctas_t<D3Q19, double>(c) : cg_ctas_t<D3Q19, float>(c);
    return c.storage == LLB_F64 ? cg_ctas_t<D3Q27, double>(c) : cg_ctas_t<D3Q27, float>(c);
}

#define LLB_CG_BATCH(fn, ...)                                                                          \
    if (c.Q == 19) {                                                                                   \
        if (c.storage == LLB_F64)                                                                      \
            return c.variant == 1 ? fn<D3Q19, double, 32, 8>(__VA_ARGS__) : fn<D3Q19, double, 64, 4>(__VA_ARGS__); \
        return c.variant == 1 ? fn<D3Q19, float, 32, 8>(__VA_ARGS__) : fn<D3Q19, float, 64, 4>(__VA_ARGS__);       \
    }                                                                                                  \
    if (c.storage == LLB_F64)                                                                          \
        return c.variant == 1 ? fn<D3Q27, double, 32, 8>(__VA_ARGS__) : fn<D3Q27, double, 64, 4>(__VA_ARGS__);     \
    return c.variant == 1 ? fn<D3Q27, float, 32, 8>(__VA_ARGS__) : fn<D3Q27, float, 64, 4>(__VA_ARGS__);

int cg_batch_ctas(const llb_ctx& c) { LLB_CG_BATCH(cg_batch_ctas_v, c) }
void cg_batch_plan(const llb_ctx& c, int grid, BatchDom* d) {
    LLB_CG_BATCH(cg_batch_plan_v, c.nx, c.ny, c.nz, grid, d)
}
cudaError_t launch_cg_batch(const llb_ctx& c, const BatchDom* doms, int ndom, int total, int grid) {
    LLB_CG_BATCH(cg_batch_run_v, c, doms, ndom, total, grid)
}

cudaError_t launch_cg_tiled(const llb_ctx& c, const void* in, void* out) {
    if (c.Q == 19) return c.storage == LLB_F64 ? cg_run_t<D3Q19, double>(c, in, out) : cg_run_t<D3Q19, float>(c, in, out);
    return c.storage == LLB_F64 ? cg_run_t<D3Q27, double>(c, in, out) : cg_run_t<D3Q27, float>(c, in, out);
}

}  // namespace llb
