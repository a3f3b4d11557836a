// Lattice definitions and the per-node arithmetic of the moment-only step.
//
// Velocities are not tabulated: a lattice is a predicate on c in {-1,0,1}^3
// plus a weight per shell |c|^2, so every loop over directions below is
// fully unrolled and every c component is a compile-time constant.
//   D3Q19 (the paper's lattice, Sec. III A): |c|^2 <= 2, w = 1/3, 1/18, 1/36
//   D3Q27: all 27 vectors, w = 8/27, 2/27, 1/54, 1/216
// Sound speed cs^2 = 1/3 (Sec. II).
//
// Shifted storage.  The device keeps, per node,
//   d = rho - 1,  j = rho u,  A = P - cs^2 rho I  (six entries)
// and works with g_i = h_i - w_i.  Because sum_i w_i (1, c_i, c_i c_i) =
// (1, 0, cs^2 I), the constant w_i part never has to be added into the
// sums, which keeps FP32 rounding relative to the flow's deviations from rest.
//
// With A' the post-collision value of A, Eq. (8) reduces to
//   h'_i = w_i [rho + 3 c_i.j + 4.5 c_i c_i : A' - 1.5 tr A'],
//   A' = (1 - omega) A + omega j j / rho,
// because P^eq = cs^2 rho I + rho u u makes the u u terms of Eq. (5)
// and Eq. (6) cancel.  rho and j are unchanged by the collision.
#pragma once

#include <cstdint>

namespace llb {

constexpr double kCs2 = 1.0 / 3.0;

struct D3Q19 {
    static constexpr int Q = 19;
    __host__ __device__ static constexpr bool has(int cx, int cy, int cz) {
        return cx * cx + cy * cy + cz * cz <= 2;
    }
    __host__ __device__ static constexpr double w(int cx, int cy, int cz) {
        return (cx * cx + cy * cy + cz * cz) == 0 ? 1.0 / 3.0
             : (cx * cx + cy * cy + cz * cz) == 1 ? 1.0 / 18.0
             : (cx * cx + cy * cy + cz * cz) == 2 ? 1.0 / 36.0 : 0.0;
    }
};

struct D3Q27 {
    static constexpr int Q = 27;
    __host__ __device__ static constexpr bool has(int, int, int) { return true; }
    __host__ __device__ static constexpr double w(int cx, int cy, int cz) {
        return (cx * cx + cy * cy + cz * cz) == 0 ? 8.0 / 27.0
             : (cx * cx + cy * cy + cz * cz) == 1 ? 2.0 / 27.0
             : (cx * cx + cy * cy + cz * cz) == 2 ? 1.0 / 54.0 : 1.0 / 216.0;
    }
};

// Number of directions whose (cx, cy) is not (0, 0): those cross between
// columns of a z-marching tile.
template <class L>
__host__ __device__ constexpr int n_xy_shifted() { return L::Q - 3; }

// Ten shifted moments of one node.
template <class T>
struct Mom {
    T d, jx, jy, jz, axx, ayy, azz, axy, axz, ayz;
};

// 1/rho.  FAST (FP32 only): the hardware approximate division (__fdividef,
// within 2 ulp for rho of order one) instead of the IEEE-rounded quotient;
// it enters only the non-linear term omega j j / rho.
template <bool FAST, class T>
__device__ __forceinline__ T inv_rho(T rho) {
    if constexpr (FAST && sizeof(T) == 4)
        return __fdividef(1.0f, rho);
    else
        return T(1) / rho;
}

// Collision: A' = (1 - omega) A + omega j j / rho; d and j are kept.
template <class T, bool FAST = false>
__device__ __forceinline__ Mom<T> collide(const Mom<T>& m, T omega) {
    const T one_m = T(1) - omega;
    const T rinv = inv_rho<FAST>(T(1) + m.d);
    const T ox = omega * m.jx * rinv, oy = omega * m.jy * rinv, oz = omega * m.jz * rinv;
    Mom<T> c;
    c.d = m.d;
    c.jx = m.jx; c.jy = m.jy; c.jz = m.jz;
    c.axx = one_m * m.axx + ox * m.jx;
    c.ayy = one_m * m.ayy + oy * m.jy;
    c.azz = one_m * m.azz + oz * m.jz;
    c.axy = one_m * m.axy + ox * m.jy;
    c.axz = one_m * m.axz + ox * m.jz;
    c.ayz = one_m * m.ayz + oy * m.jz;
    return c;
}

// g'_i = h'_i - w_i for direction (cx, cy, cz) from collided moments.
// s0 = d - 1.5 tr A' is shared by all directions of a node.
template <class L, class T>
__device__ __forceinline__ T g_dir(const Mom<T>& c, T s0, int cx, int cy, int cz) {
    T q = s0;
    if (cx) q += T(4.5) * c.axx;
    if (cy) q += T(4.5) * c.ayy;
    if (cz) q += T(4.5) * c.azz;
    if (cx * cy) q += T(9 * cx * cy) * c.axy;
    if (cx * cz) q += T(9 * cx * cz) * c.axz;
    if (cy * cz) q += T(9 * cy * cz) * c.ayz;
    T lin = T(0);
    if (cx) lin += T(3 * cx) * c.jx;
    if (cy) lin += T(3 * cy) * c.jy;
    if (cz) lin += T(3 * cz) * c.jz;
    return T(L::w(cx, cy, cz)) * (q + lin);
}

template <class T>
__device__ __forceinline__ T g_shared(const Mom<T>& c) {
    return c.d - T(1.5) * (c.axx + c.ayy + c.azz);
}

// Accumulator of streamed g's into (d, j, S = sum g c c) of one node.
template <class T>
struct Acc {
    T d, jx, jy, jz, sxx, syy, szz, sxy, sxz, syz;
    __device__ __forceinline__ void zero() {
        d = jx = jy = jz = sxx = syy = szz = sxy = sxz = syz = T(0);
    }
    __device__ __forceinline__ void add(T g, int cx, int cy, int cz) {
        d += g;
        if (cx > 0) { jx += g; sxx += g; } else if (cx < 0) { jx -= g; sxx += g; }
        if (cy > 0) { jy += g; syy += g; } else if (cy < 0) { jy -= g; syy += g; }
        if (cz > 0) { jz += g; szz += g; } else if (cz < 0) { jz -= g; szz += g; }
        if (cx * cy > 0) sxy += g; else if (cx * cy < 0) sxy -= g;
        if (cx * cz > 0) sxz += g; else if (cx * cz < 0) sxz -= g;
        if (cy * cz > 0) syz += g; else if (cy * cz < 0) syz -= g;
    }
    // New shifted moments: A = S - cs^2 d I (Eqs. (1)-(3) on h = w + g).
    __device__ __forceinline__ Mom<T> finish() const {
        Mom<T> m;
        const T t = T(kCs2) * d;
        m.d = d; m.jx = jx; m.jy = jy; m.jz = jz;
        m.axx = sxx - t; m.ayy = syy - t; m.azz = szz - t;
        m.axy = sxy; m.axz = sxz; m.ayz = syz;
        return m;
    }
};

__host__ __device__ __forceinline__ int wrap_idx(int v, int n) {
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

}  // namespace llb
