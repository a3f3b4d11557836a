// Hand-written adjoint of the one-component moment-only step.
//
// One step is m_new = S(C(m)) with
//   C (pointwise collision): (d, j, A) -> (d, j, A' = (1 - omega) A + omega j j / rho), rho = 1 + d
//   S (linear pull stencil): m_new(x) = sum_i e_i g_i(x - c_i),
//       g_i = r_i . m' = w_i [d + 3 c_i.j + 4.5 c_i c_i : A' - 1.5 tr A'],
//       e_i = (1, c_i, c_i c_i - cs^2 I) (the moments one unit of g_i carries).
// Its adjoint maps a cotangent lam_new of m_new to the cotangent of m:
//   lam'(y) = S^T lam_new (y) = sum_i r_i s_i,  s_i = e_i . lam_new(y + c_i)
//   lam(y)  = J_C(m(y))^T lam'(y)
// and accumulates dL/domega = sum_y lam'_A(y) : (j j / rho - A)(y).
// The state A is stored as six entries; a cotangent of an off-diagonal entry
// is the derivative with respect to that stored entry.
//
// Two components (A_h = 0, smooth normal |G|_eps): the state is (rho1, d, j,
// A) and a source node y emits g'_i (as above, with A' gaining
// ks n n, ks = A_s |G|_eps / 9, n = G / |G|_eps) and the colour population
//   h1'_i = (rho1 / rho)(w_i + g'_i) + e w_i (c_i.n) / |c_i|,  e = beta rho1 (rho - rho1) / rho,
// where G(y) = 3 sum_k w_k c_k phi(y + c_k), phi = 2 rho1 / rho - 1.  The
// adjoint runs in two passes: per node y, the cotangents of y's own fields
// and of G(y) (pull transposed, then the node's collision, perturbation and
// recolouring transposed); then per node z, the transposed gradient stencil
// lam_phi(z) = 3 sum_k w_k c_k . lam_G(z - c_k), added through phi(z) to
// lam_rho1(z) and lam_d(z).
//
// For two components the first pass (everything but the transposed gradient
// stencil) runs tiled by default (k_adjoint_cg_tiled, below); one component
// keeps the one-thread-per-node k_adjoint_step, a plain linear gather whose
// neighbour loads hit L1 (a tiled form of it measured 13-18 % slower).
//
// llb_adjoint runs the forward steps once, keeping the state every K steps
// (moments only), then walks the segments backwards: each segment is
// recomputed from its checkpoint with its K states kept, and the adjoint
// steps run through it in reverse (memory: ~N/K + K state copies).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "checked.cuh"
#include "internal.h"
#include "lattice.cuh"
#include "layout.cuh"
#include "moment_common.cuh"

namespace llb {
namespace {

constexpr int kAdjThreads = 128;

// The ten fields of node i of a one-component buffer (state or cotangent; the
// field order of FieldMap).
template <class T>
__device__ __forceinline__ void load10(const T* __restrict__ p, size_t i, size_t fs, T* v) {
#pragma unroll
    for (int f = 0; f < 10; ++f) v[f] = p[FieldMap<T, 10>::at(i, f, fs)];
}

// Adjoint of one step at source node y (one thread per node).  lam_new, m and
// lam share the context's Layout; neighbours are addressed with the periodic
// wrap (no ghost copies are needed in the cotangent arrays).
template <class L, class T>
__global__ void __launch_bounds__(kAdjThreads) k_adjoint_step(const T* __restrict__ lam_new, const T* __restrict__ m,
                                                              T* __restrict__ lam, Layout lay, T omega,
                                                              double* __restrict__ domega_rows) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    double part = 0.0;
    if (x < lay.nx) {
        // lam' = sum_i r_i (e_i . lam_new(y + c_i))
        T ld = T(0), lj[3] = {T(0), T(0), T(0)}, la[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
            for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
                for (int cx = -1; cx <= 1; ++cx) {
                    if (!L::has(cx, cy, cz)) continue;
                    const size_t q = lay.at(wrap_idx(x + cx, lay.nx), wrap_idx(y + cy, lay.ny), wrap_idx(z + cz, lay.nz));
                    T v[10];
                    load10(lam_new, q, lay.fs, v);
                    const T cxx = T(cx * cx) - T(kCs2), cyy = T(cy * cy) - T(kCs2), czz = T(cz * cz) - T(kCs2);
                    // e_i . lam_new: the stored A entries carry (c_a c_b - cs^2 delta_ab)
                    const T si = v[0] + T(cx) * v[1] + T(cy) * v[2] + T(cz) * v[3] + cxx * v[4] + cyy * v[5] +
                                 czz * v[6] + T(cx * cy) * v[7] + T(cx * cz) * v[8] + T(cy * cz) * v[9];
                    const T ws = T(L::w(cx, cy, cz)) * si;
                    // r_i: dg/dd = w, dg/dj = 3 w c, dg/dA_aa = w (4.5 c_a^2 - 1.5), dg/dA_ab = 9 w c_a c_b
                    ld += ws;
                    lj[0] += T(3 * cx) * ws;
                    lj[1] += T(3 * cy) * ws;
                    lj[2] += T(3 * cz) * ws;
                    la[0] += (T(4.5 * cx * cx) - T(1.5)) * ws;
                    la[1] += (T(4.5 * cy * cy) - T(1.5)) * ws;
                    la[2] += (T(4.5 * cz * cz) - T(1.5)) * ws;
                    la[3] += T(9 * cx * cy) * ws;
                    la[4] += T(9 * cx * cz) * ws;
                    la[5] += T(9 * cy * cz) * ws;
                }
        // J_C^T at y
        const size_t i0 = lay.at(x, y, z);
        T s[10];
        load10(m, i0, lay.fs, s);
        const T rinv = T(1) / (T(1) + s[0]);
        const T jx = s[1], jy = s[2], jz = s[3];
        const T om = omega;
        // A'_aa = (1-w) A_aa + w j_a^2 / rho ; A'_ab = (1-w) A_ab + w j_a j_b / rho
        const T jj[6] = {jx * jx, jy * jy, jz * jz, jx * jy, jx * jz, jy * jz};
        T dsum = T(0);
        for (int k = 0; k < 6; ++k) dsum += la[k] * jj[k];
        T out[10];
        out[0] = ld - om * rinv * rinv * dsum;
        out[1] = lj[0] + om * rinv * (T(2) * jx * la[0] + jy * la[3] + jz * la[4]);
        out[2] = lj[1] + om * rinv * (T(2) * jy * la[1] + jx * la[3] + jz * la[5]);
        out[3] = lj[2] + om * rinv * (T(2) * jz * la[2] + jx * la[4] + jy * la[5]);
        for (int k = 0; k < 6; ++k) out[4 + k] = (T(1) - om) * la[k];
#pragma unroll
        for (int f = 0; f < 10; ++f) lam[FieldMap<T, 10>::at(i0, f, lay.fs)] = out[f];
        // dL/domega: lam'_A : (j j / rho - A)
        for (int k = 0; k < 6; ++k) part += (double)la[k] * ((double)jj[k] * (double)rinv - (double)s[4 + k]);
    }
    // block sum of the omega derivative (fixed order: warp shuffles then lanes of warp 0)
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    __shared__ double wsum[kAdjThreads / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sacc = 0.0;
        for (int w = 0; w < kAdjThreads / 32; ++w) sacc += wsum[w];
        const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        domega_rows[b] = sacc;
    }
}

template <class T>
struct CGAdjPar {
    T omega, beta, A_s, eps2;
};

__host__ __device__ constexpr double inv_len_c(int cx, int cy, int cz) {
    return (cx * cx + cy * cy + cz * cz) == 1 ? 1.0
         : (cx * cx + cy * cy + cz * cz) == 2 ? 0.70710678118654752440
         : (cx * cx + cy * cy + cz * cz) == 3 ? 0.57735026918962576451 : 0.0;
}

// Pass 1 of the two-component adjoint step at source node y: writes the
// cotangents of y's 11 fields (before the phase-field chain) to lam and of
// G(y) to lam_g (3 fields), and the block's dL/domega to domega_rows.
template <class L, class T>
__global__ void __launch_bounds__(kAdjThreads) k_adjoint_cg_local(const T* __restrict__ lam_new,
                                                                  const T* __restrict__ m, T* __restrict__ lam,
                                                                  T* __restrict__ lam_g, Layout lay, CGAdjPar<T> p,
                                                                  double* __restrict__ domega_rows) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    const size_t fs = lay.fs;
    double part = 0.0;
    if (x < lay.nx) {
        const size_t i0 = lay.at(x, y, z);
        T s[11];
#pragma unroll
        for (int f = 0; f < 11; ++f) s[f] = m[f * fs + i0];
        const T r1 = s[0], d = s[1], jx = s[2], jy = s[3], jz = s[4];
        const T* A = s + 5;  // xx, yy, zz, xy, xz, yz
        // G(y) from phi of the neighbours
        T G[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
            for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
                for (int cx = -1; cx <= 1; ++cx) {
                    if (!L::has(cx, cy, cz) || (cx == 0 && cy == 0 && cz == 0)) continue;
                    const size_t q = lay.at(wrap_idx(x + cx, lay.nx), wrap_idx(y + cy, lay.ny), wrap_idx(z + cz, lay.nz));
                    const T ph = T(2) * m[q] / (T(1) + m[fs + q]) - T(1);
                    const T wp = T(3.0 * L::w(cx, cy, cz)) * ph;
                    G[0] += T(cx) * wp;
                    G[1] += T(cy) * wp;
                    G[2] += T(cz) * wp;
                }
        // forward quantities of the node
        const T rho = T(1) + d, rinv = T(1) / rho, om = p.omega;
        const T gn = sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2] + p.eps2);
        const T n[3] = {G[0] / gn, G[1] / gn, G[2] / gn};
        const T ks = p.A_s * gn * T(1.0 / 9.0);
        const T jj[6] = {jx * jx, jy * jy, jz * jz, jx * jy, jx * jz, jy * jz};
        const T nn[6] = {n[0] * n[0], n[1] * n[1], n[2] * n[2], n[0] * n[1], n[0] * n[2], n[1] * n[2]};
        T Ap[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) Ap[k] = (T(1) - om) * A[k] + om * jj[k] * rinv + ks * nn[k];
        const T s0 = d - T(1.5) * (Ap[0] + Ap[1] + Ap[2]);
        const T r1r = r1 * rinv;
        const T e = p.beta * r1 * (rho - r1) * rinv;
        // pull transposed: per direction, the cotangents of g'_i and h1'_i
        T ld = T(0), lj[3] = {T(0), T(0), T(0)}, la[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        T l_r1r = T(0), l_e = T(0), ln[3] = {T(0), T(0), T(0)};
#pragma unroll
        for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
            for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
                for (int cx = -1; cx <= 1; ++cx) {
                    if (!L::has(cx, cy, cz)) continue;
                    const size_t q = lay.at(wrap_idx(x + cx, lay.nx), wrap_idx(y + cy, lay.ny), wrap_idx(z + cz, lay.nz));
                    T v[11];
#pragma unroll
                    for (int f = 0; f < 11; ++f) v[f] = lam_new[f * fs + q];
                    const T cxx = T(cx * cx) - T(kCs2), cyy = T(cy * cy) - T(kCs2), czz = T(cz * cz) - T(kCs2);
                    const T si = v[1] + T(cx) * v[2] + T(cy) * v[3] + T(cz) * v[4] + cxx * v[5] + cyy * v[6] +
                                 czz * v[7] + T(cx * cy) * v[8] + T(cx * cz) * v[9] + T(cy * cz) * v[10];
                    const T ti = v[0];
                    const T w = T(L::w(cx, cy, cz));
                    T qd = s0;
                    if (cx) qd += T(4.5) * Ap[0];
                    if (cy) qd += T(4.5) * Ap[1];
                    if (cz) qd += T(4.5) * Ap[2];
                    if (cx * cy) qd += T(9 * cx * cy) * Ap[3];
                    if (cx * cz) qd += T(9 * cx * cz) * Ap[4];
                    if (cy * cz) qd += T(9 * cy * cz) * Ap[5];
                    const T gi = w * (qd + T(3 * cx) * jx + T(3 * cy) * jy + T(3 * cz) * jz);
                    l_r1r += ti * (w + gi);
                    if (cx || cy || cz) {
                        const T il = T(inv_len_c(cx, cy, cz));
                        const T cn = T(cx) * n[0] + T(cy) * n[1] + T(cz) * n[2];
                        l_e += ti * w * cn * il;
                        const T f = ti * e * w * il;
                        ln[0] += f * T(cx);
                        ln[1] += f * T(cy);
                        ln[2] += f * T(cz);
                    }
                    const T ws = w * (si + ti * r1r);
                    ld += ws;
                    lj[0] += T(3 * cx) * ws;
                    lj[1] += T(3 * cy) * ws;
                    lj[2] += T(3 * cz) * ws;
                    la[0] += (T(4.5 * cx * cx) - T(1.5)) * ws;
                    la[1] += (T(4.5 * cy * cy) - T(1.5)) * ws;
                    la[2] += (T(4.5 * cz * cz) - T(1.5)) * ws;
                    la[3] += T(9 * cx * cy) * ws;
                    la[4] += T(9 * cx * cz) * ws;
                    la[5] += T(9 * cy * cz) * ws;
                }
        // collision transposed: A' = (1 - w) A + w j j / rho + ks n n
        T l_rinv = T(0), l_ks = T(0);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            l_rinv += om * la[k] * jj[k];
            l_ks += la[k] * nn[k];
        }
        T out[11];
        out[2] = lj[0] + om * rinv * (T(2) * jx * la[0] + jy * la[3] + jz * la[4]);
        out[3] = lj[1] + om * rinv * (T(2) * jy * la[1] + jx * la[3] + jz * la[5]);
        out[4] = lj[2] + om * rinv * (T(2) * jz * la[2] + jx * la[4] + jy * la[5]);
#pragma unroll
        for (int k = 0; k < 6; ++k) out[5 + k] = (T(1) - om) * la[k];
        ln[0] += ks * (T(2) * n[0] * la[0] + n[1] * la[3] + n[2] * la[4]);
        ln[1] += ks * (T(2) * n[1] * la[1] + n[0] * la[3] + n[2] * la[5]);
        ln[2] += ks * (T(2) * n[2] * la[2] + n[0] * la[4] + n[1] * la[5]);
        // ks = A_s gn / 9, n = G / gn, gn = sqrt(|G|^2 + eps^2)
        T l_gn = p.A_s * T(1.0 / 9.0) * l_ks - (ln[0] * G[0] + ln[1] * G[1] + ln[2] * G[2]) / (gn * gn);
        T lg[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) lg[a] = ln[a] / gn + l_gn * G[a] / gn;
        // colour split: r1r = r1 / rho, e = beta (r1 - r1^2 / rho)
        l_rinv += l_r1r * r1 - l_e * p.beta * r1 * r1;
        out[0] = l_r1r * rinv + l_e * p.beta * (T(1) - T(2) * r1 * rinv);
        out[1] = ld - l_rinv * rinv * rinv;
#pragma unroll
        for (int f = 0; f < 11; ++f) lam[f * fs + i0] = out[f];
#pragma unroll
        for (int a = 0; a < 3; ++a) lam_g[a * fs + i0] = lg[a];
        for (int k = 0; k < 6; ++k) part += (double)la[k] * ((double)jj[k] * (double)rinv - (double)A[k]);
    }
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    __shared__ double wsum[kAdjThreads / 32];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sacc = 0.0;
        for (int w = 0; w < kAdjThreads / 32; ++w) sacc += wsum[w];
        const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        domega_rows[b] = sacc;
    }
}

// Pass 2: the phase-field chain at node z.  G(y) = 3 sum_k w_k c_k phi(y + c_k)
// transposed gives lam_phi(z) = 3 sum_k w_k c_k . lam_G(z - c_k); phi = 2 rho1 / rho - 1.
template <class L, class T>
__global__ void __launch_bounds__(kAdjThreads) k_adjoint_cg_phi(const T* __restrict__ m, const T* __restrict__ lam_g,
                                                                T* __restrict__ lam, Layout lay) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= lay.nx) return;
    const size_t fs = lay.fs;
    T lphi = T(0);
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz) || (cx == 0 && cy == 0 && cz == 0)) continue;
                const size_t q = lay.at(wrap_idx(x - cx, lay.nx), wrap_idx(y - cy, lay.ny), wrap_idx(z - cz, lay.nz));
                lphi += T(3.0 * L::w(cx, cy, cz)) *
                        (T(cx) * lam_g[q] + T(cy) * lam_g[fs + q] + T(cz) * lam_g[2 * fs + q]);
            }
    const size_t i0 = lay.at(x, y, z);
    const T rinv = T(1) / (T(1) + m[fs + i0]);
    lam[i0] += lphi * T(2) * rinv;
    lam[fs + i0] -= lphi * T(2) * m[i0] * rinv * rinv;
}

// ---------------------------------------------------------------------------
// Tiled pass 1 of the two-component adjoint (the default).  Receiver y needs,
// for every direction c, s_c(y + c) = e_c . lam_new(y + c) and
// t(y + c) = lam_new_rho1(y + c), and phi(y + c) for G(y).  Instead of loading
// the 11 cotangent fields of each of its Q neighbours (k_adjoint_cg_local), a
// persistent CTA marches a BX x BY tile through z: for each plane, every node
// of the tile plus a one-node halo computes its Q projections once and
// publishes them, with t and phi, into a ring of three planes in shared
// memory; each receiver of the middle plane then reads two values per
// direction.  Two barriers per plane (published; ring slot free again).
template <class L, class T, int BX, int BY>
struct AdjTile {
    static constexpr int NT = BX * BY, HX = BX + 2, HY = BY + 2, HN = HX * HY;
    static constexpr int NF = L::Q + 2;  // Q projections, t, phi
    static constexpr int SLOT = NF * HN;  // elements of one plane of the ring
    static constexpr size_t smem_bytes = 3 * (size_t)SLOT * sizeof(T);
    static constexpr int MINB = sizeof(T) == 4 ? 3 : 1;  // CTAs per SM the register budget targets
    static_assert(NT % 32 == 0, "whole warps");
};
constexpr int kAdjBX = 32, kAdjBY = 4;

// Index of direction (cx, cy, cz) in the lattice, enumerated over cz, cy, cx.
template <class L>
__host__ __device__ constexpr int dir_index(int cx, int cy, int cz) {
    int k = 0;
    for (int z = -1; z <= 1; ++z)
        for (int y = -1; y <= 1; ++y)
            for (int x = -1; x <= 1; ++x) {
                if (!L::has(x, y, z)) continue;
                if (x == cx && y == cy && z == cz) return k;
                ++k;
            }
    return -1;
}

// Publish node j of the tile-plus-halo region (plane index zq, wrapped) into slot S.
template <class L, class T, int HN>
__device__ __forceinline__ void adj_publish(const T* __restrict__ lam_new, const T* __restrict__ m, const Layout& lay,
                                            size_t i, int j, T* __restrict__ S) {
    const size_t fs = lay.fs;
    if (!LLB_IN(i, fs, kChkLoad) || !LLB_IN(j, HN, kChkPublish)) return;
    T v[11];
#pragma unroll
    for (int f = 0; f < 11; ++f) v[f] = lam_new[f * fs + i];
    const T r1 = m[i], d = m[fs + i];
    S[(L::Q + 1) * HN + j] = T(2) * r1 / (T(1) + d) - T(1);
    S[L::Q * HN + j] = v[0];
    // s(+-c) = even +- odd, even = v1 + (cc - cs^2 I) : vP, odd = c . vj
    const T ev0 = v[1] - T(kCs2) * (v[5] + v[6] + v[7]);
    S[dir_index<L>(0, 0, 0) * HN + j] = ev0;
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                const bool lead = cx > 0 || (cx == 0 && (cy > 0 || (cy == 0 && cz > 0)));
                if (!lead || !L::has(cx, cy, cz)) continue;
                T ev = ev0;
                if (cx) ev += v[5];
                if (cy) ev += v[6];
                if (cz) ev += v[7];
                if (cx * cy) ev += T(cx * cy) * v[8];
                if (cx * cz) ev += T(cx * cz) * v[9];
                if (cy * cz) ev += T(cy * cz) * v[10];
                T od = T(0);
                if (cx) od += T(cx) * v[2];
                if (cy) od += T(cy) * v[3];
                if (cz) od += T(cz) * v[4];
                S[dir_index<L>(cx, cy, cz) * HN + j] = ev + od;
                S[dir_index<L>(-cx, -cy, -cz) * HN + j] = ev - od;
            }
}

// Receiver y (node n of the region, own 11 fields in s): the direct kernel's
// arithmetic with the neighbour quantities read from the ring planes Sm, S0, Sp
// (planes z - 1, z, z + 1).  Writes lam(y), lam_g(y); returns y's dL/domega term.
template <class L, class T, int HX, int HN>
__device__ __forceinline__ double adj_receive(const T* __restrict__ Sm, const T* __restrict__ S0,
                                              const T* __restrict__ Sp, int n, const T* s, const CGAdjPar<T>& p,
                                              T* __restrict__ lam, T* __restrict__ lam_g, size_t i0, size_t fs) {
    if (!LLB_IN(n - HX - 1, HN, kChkGather) || !LLB_IN(n + HX + 1, HN, kChkGather) || !LLB_IN(i0, fs, kChkStore))
        return 0.0;
    constexpr int Q = L::Q;
    const T r1 = s[0], d = s[1], jx = s[2], jy = s[3], jz = s[4];
    const T* A = s + 5;  // xx, yy, zz, xy, xz, yz
    T G[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz) || (cx == 0 && cy == 0 && cz == 0)) continue;
                const T* P = cz > 0 ? Sp : (cz < 0 ? Sm : S0);
                const T wp = T(3.0 * L::w(cx, cy, cz)) * P[(Q + 1) * HN + n + cy * HX + cx];
                G[0] += T(cx) * wp;
                G[1] += T(cy) * wp;
                G[2] += T(cz) * wp;
            }
    const T rho = T(1) + d, rinv = T(1) / rho, om = p.omega;
    const T gn = sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2] + p.eps2);
    const T nv[3] = {G[0] / gn, G[1] / gn, G[2] / gn};
    const T ks = p.A_s * gn * T(1.0 / 9.0);
    const T jj[6] = {jx * jx, jy * jy, jz * jz, jx * jy, jx * jz, jy * jz};
    const T nn[6] = {nv[0] * nv[0], nv[1] * nv[1], nv[2] * nv[2], nv[0] * nv[1], nv[0] * nv[2], nv[1] * nv[2]};
    T Ap[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) Ap[k] = (T(1) - om) * A[k] + om * jj[k] * rinv + ks * nn[k];
    const T s0 = d - T(1.5) * (Ap[0] + Ap[1] + Ap[2]);
    const T r1r = r1 * rinv;
    const T e = p.beta * r1 * (rho - r1) * rinv;
    T ld = T(0), lj[3] = {T(0), T(0), T(0)}, la[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    T l_r1r = T(0), l_e = T(0), ln[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                if (!L::has(cx, cy, cz)) continue;
                const T* P = cz > 0 ? Sp : (cz < 0 ? Sm : S0);
                const int o = n + cy * HX + cx;
                const T si = P[dir_index<L>(cx, cy, cz) * HN + o];
                const T ti = P[Q * HN + o];
                const T w = T(L::w(cx, cy, cz));
                T qd = s0;
                if (cx) qd += T(4.5) * Ap[0];
                if (cy) qd += T(4.5) * Ap[1];
                if (cz) qd += T(4.5) * Ap[2];
                if (cx * cy) qd += T(9 * cx * cy) * Ap[3];
                if (cx * cz) qd += T(9 * cx * cz) * Ap[4];
                if (cy * cz) qd += T(9 * cy * cz) * Ap[5];
                const T gi = w * (qd + T(3 * cx) * jx + T(3 * cy) * jy + T(3 * cz) * jz);
                l_r1r += ti * (w + gi);
                if (cx || cy || cz) {
                    const T il = T(inv_len_c(cx, cy, cz));
                    const T cn = T(cx) * nv[0] + T(cy) * nv[1] + T(cz) * nv[2];
                    l_e += ti * w * cn * il;
                    const T f = ti * e * w * il;
                    ln[0] += f * T(cx);
                    ln[1] += f * T(cy);
                    ln[2] += f * T(cz);
                }
                const T ws = w * (si + ti * r1r);
                ld += ws;
                lj[0] += T(3 * cx) * ws;
                lj[1] += T(3 * cy) * ws;
                lj[2] += T(3 * cz) * ws;
                la[0] += (T(4.5 * cx * cx) - T(1.5)) * ws;
                la[1] += (T(4.5 * cy * cy) - T(1.5)) * ws;
                la[2] += (T(4.5 * cz * cz) - T(1.5)) * ws;
                la[3] += T(9 * cx * cy) * ws;
                la[4] += T(9 * cx * cz) * ws;
                la[5] += T(9 * cy * cz) * ws;
            }
    T l_rinv = T(0), l_ks = T(0);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        l_rinv += om * la[k] * jj[k];
        l_ks += la[k] * nn[k];
    }
    T out[11];
    out[2] = lj[0] + om * rinv * (T(2) * jx * la[0] + jy * la[3] + jz * la[4]);
    out[3] = lj[1] + om * rinv * (T(2) * jy * la[1] + jx * la[3] + jz * la[5]);
    out[4] = lj[2] + om * rinv * (T(2) * jz * la[2] + jx * la[4] + jy * la[5]);
#pragma unroll
    for (int k = 0; k < 6; ++k) out[5 + k] = (T(1) - om) * la[k];
    ln[0] += ks * (T(2) * nv[0] * la[0] + nv[1] * la[3] + nv[2] * la[4]);
    ln[1] += ks * (T(2) * nv[1] * la[1] + nv[0] * la[3] + nv[2] * la[5]);
    ln[2] += ks * (T(2) * nv[2] * la[2] + nv[0] * la[4] + nv[1] * la[5]);
    const T l_gn = p.A_s * T(1.0 / 9.0) * l_ks - (ln[0] * G[0] + ln[1] * G[1] + ln[2] * G[2]) / (gn * gn);
    l_rinv += l_r1r * r1 - l_e * p.beta * r1 * r1;
    out[0] = l_r1r * rinv + l_e * p.beta * (T(1) - T(2) * r1 * rinv);
    out[1] = ld - l_rinv * rinv * rinv;
#pragma unroll
    for (int f = 0; f < 11; ++f) lam[f * fs + i0] = out[f];
#pragma unroll
    for (int a = 0; a < 3; ++a) lam_g[a * fs + i0] = ln[a] / gn + l_gn * G[a] / gn;
    double part = 0.0;
    for (int k = 0; k < 6; ++k) part += (double)la[k] * ((double)jj[k] * (double)rinv - (double)A[k]);
    return part;
}

template <class L, class T, int BX, int BY>
__global__ void __launch_bounds__(BX * BY, (AdjTile<L, T, BX, BY>::MINB))
    k_adjoint_cg_tiled(const T* __restrict__ lam_new, const T* __restrict__ m, T* __restrict__ lam,
                       T* __restrict__ lam_g, Layout lay, CGAdjPar<T> p, mom::Sched sc,
                       double* __restrict__ domega_rows) {
    using C = AdjTile<L, T, BX, BY>;
    constexpr int NT = C::NT, HX = C::HX, HN = C::HN, SLOT = C::SLOT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* const ring = reinterpret_cast<T*>(smem_raw);
    const int nx = lay.nx, ny = lay.ny, nz = lay.nz;
    const size_t fs = lay.fs, plane = (size_t)lay.px * lay.py;
    const int t = threadIdx.x, tx = t % BX, ty = t / BX;
    const int n_own = (ty + 1) * HX + (tx + 1);
    double part = 0.0;

    for (int it = blockIdx.x; it < sc.nitems; it += gridDim.x) {
        int x0, y0, za, zb;  // receivers of planes za .. zb-1 of the tile at (x0, y0)
        sc.item(it, BX, BY, nz, x0, y0, za, zb);
        // region nodes of this thread: j = t and j = t + NT (if inside the tile plus halo)
        const int j1 = t + NT;
        const size_t off0 = lay.at(mom::pmod(x0 - 1 + t % HX, nx), mom::pmod(y0 - 1 + t / HX, ny), 0);
        const size_t off1 = j1 < HN ? lay.at(mom::pmod(x0 - 1 + j1 % HX, nx), mom::pmod(y0 - 1 + j1 / HX, ny), 0) : 0;
        const int ox = x0 + tx, oy = y0 + ty;
        const bool ok = ox < nx && oy < ny;
        const size_t own = ok ? lay.at(ox, oy, 0) : 0;
        auto slot = [&](int q) { return ring + (size_t)((q - za + 1) % 3) * SLOT; };  // q >= za - 1
        auto publish = [&](int q) {
            T* S = slot(q);
            const size_t zo = (size_t)mom::pmod(q, nz) * plane;
            adj_publish<L, T, HN>(lam_new, m, lay, off0 + zo, t, S);
            if (j1 < HN) adj_publish<L, T, HN>(lam_new, m, lay, off1 + zo, j1, S);
        };
        publish(za - 1);
        publish(za);
        for (int q = za; q < zb; ++q) {  // receivers of plane q
            publish(q + 1);
            T sv[11];
            const size_t iy = own + (size_t)mom::pmod(q, nz) * plane;
            if (ok && LLB_IN(iy, fs, kChkLoad)) {
#pragma unroll
                for (int f = 0; f < 11; ++f) sv[f] = m[f * fs + iy];
            }
            __syncthreads();  // planes q - 1, q, q + 1 published
            if (ok) part += adj_receive<L, T, HX, HN>(slot(q - 1), slot(q), slot(q + 1), n_own, sv, p, lam, lam_g, iy, fs);
            __syncthreads();  // the slot of plane q - 1 may be refilled
        }
    }
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    __shared__ double wsum[NT / 32];
    if ((t & 31) == 0) wsum[t >> 5] = part;
    __syncthreads();
    if (t == 0) {
        double sacc = 0.0;
        for (int w = 0; w < NT / 32; ++w) sacc += wsum[w];
        domega_rows[blockIdx.x] = sacc;
    }
}

// acc += sum of rows (one block, fixed order).
__global__ void k_sum_rows(const double* __restrict__ rows, size_t n, double* __restrict__ acc) {
    __shared__ double sh[256];
    double s = 0.0;
    for (size_t i = threadIdx.x; i < n; i += 256) s += rows[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *acc += sh[0];
}

// Cotangents: canonical (rho, j, P) <-> shifted (d, j, A).  The forward maps are
// d = rho - 1, A_aa = P_aa - cs^2 rho, A_ab = P_ab and back rho = 1 + d,
// P_aa = A_aa + cs^2 (1 + d); the cotangent maps are their transposes.
template <class T>
__global__ void k_cot_canon_to_shifted(const void* __restrict__ g, int dt, T* __restrict__ lam, Layout L) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        double v[10];
        for (int f = 0; f < 10; ++f)
            v[f] = dt == LLB_F64 ? static_cast<const double*>(g)[f * N + i] : (double)static_cast<const float*>(g)[f * N + i];
        const int x = (int)(i % L.nx);
        const size_t r = i / L.nx;
        const size_t j = L.at(x, (int)(r % L.ny), (int)(r / L.ny));
        lam[FieldMap<T, 10>::at(j, 0, L.fs)] = (T)(v[0] + kCs2 * (v[4] + v[5] + v[6]));
        for (int f = 1; f < 10; ++f) lam[FieldMap<T, 10>::at(j, f, L.fs)] = (T)v[f];
    }
}

template <class T>
__global__ void k_cot_shifted_to_canon(const T* __restrict__ lam, void* __restrict__ g, int dt, Layout L) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % L.nx);
        const size_t r = i / L.nx;
        const size_t j = L.at(x, (int)(r % L.ny), (int)(r / L.ny));
        double v[10];
        for (int f = 0; f < 10; ++f) v[f] = (double)lam[FieldMap<T, 10>::at(j, f, L.fs)];
        v[0] -= kCs2 * (v[4] + v[5] + v[6]);
        for (int f = 0; f < 10; ++f) {
            if (dt == LLB_F64) static_cast<double*>(g)[f * N + i] = v[f];
            else static_cast<float*>(g)[f * N + i] = (float)v[f];
        }
    }
}

// Two components: canonical (rho1, rho2, j, P) <-> internal (rho1, d, j, A) with
// rho2 = 1 + d - rho1, P_aa = A_aa + cs^2 (1 + d); cotangents map by the transposes.
template <class T>
__global__ void k_cot2_canon_to_internal(const void* __restrict__ g, int dt, T* __restrict__ lam, Layout L) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        double v[11];
        for (int f = 0; f < 11; ++f)
            v[f] = dt == LLB_F64 ? static_cast<const double*>(g)[f * N + i] : (double)static_cast<const float*>(g)[f * N + i];
        const int x = (int)(i % L.nx);
        const size_t r = i / L.nx;
        const size_t j = L.at(x, (int)(r % L.ny), (int)(r / L.ny));
        lam[j] = (T)(v[0] - v[1]);
        lam[L.fs + j] = (T)(v[1] + kCs2 * (v[5] + v[6] + v[7]));
        for (int f = 2; f < 11; ++f) lam[f * L.fs + j] = (T)v[f];
    }
}

template <class T>
__global__ void k_cot2_internal_to_canon(const T* __restrict__ lam, void* __restrict__ g, int dt, Layout L) {
    const size_t N = (size_t)L.nx * L.ny * L.nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % L.nx);
        const size_t r = i / L.nx;
        const size_t j = L.at(x, (int)(r % L.ny), (int)(r / L.ny));
        double v[11];
        for (int f = 0; f < 11; ++f) v[f] = (double)lam[f * L.fs + j];
        const double tr = kCs2 * (v[5] + v[6] + v[7]);
        const double g1 = v[0] + v[1] - tr, g2 = v[1] - tr;
        v[0] = g1;
        v[1] = g2;
        for (int f = 0; f < 11; ++f) {
            if (dt == LLB_F64) static_cast<double*>(g)[f * N + i] = v[f];
            else static_cast<float*>(g)[f * N + i] = (float)v[f];
        }
    }
}

dim3 adj_grid(const llb_ctx& c) { return dim3((c.nx + kAdjThreads - 1) / kAdjThreads, c.ny, c.nz); }

template <class L, class T>
cudaError_t adj_step_t(const llb_ctx& c, const void* lam_new, const void* m, void* lam, double* rows) {
    k_adjoint_step<L, T><<<adj_grid(c), kAdjThreads, 0, c.stream>>>(static_cast<const T*>(lam_new),
                                                                     static_cast<const T*>(m), static_cast<T*>(lam),
                                                                     c.lay, (T)c.omega, rows);
    return cudaGetLastError();
}

cudaError_t adj_step(const llb_ctx& c, const void* lam_new, const void* m, void* lam, double* rows) {
    if (c.Q == 19)
        return c.storage == LLB_F64 ? adj_step_t<D3Q19, double>(c, lam_new, m, lam, rows)
                                    : adj_step_t<D3Q19, float>(c, lam_new, m, lam, rows);
    return c.storage == LLB_F64 ? adj_step_t<D3Q27, double>(c, lam_new, m, lam, rows)
                                : adj_step_t<D3Q27, float>(c, lam_new, m, lam, rows);
}

// CTAs of the tiled first pass for this context (0 if it cannot run).
template <class L, class T>
int adj_tiled_ctas(const llb_ctx& c) {
    using C = AdjTile<L, T, kAdjBX, kAdjBY>;
    auto kern = k_adjoint_cg_tiled<L, T, kAdjBX, kAdjBY>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_bytes) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, C::smem_bytes) != cudaSuccess || per_sm < 1)
        return 0;
    const mom::Sched sc = mom::plan(c.nx, c.ny, c.nz, kAdjBX, kAdjBY, per_sm * c.num_sms);
    return std::min(sc.nitems, per_sm * c.num_sms);
}

// One two-component adjoint step; *nrows: rows of dL/domega partial sums written.
template <class L, class T>
cudaError_t adj_cg_step_t(const llb_ctx& c, const void* lam_new, const void* m, void* lam, void* lam_g,
                          double* rows, size_t* nrows) {
    CGAdjPar<T> p;
    p.omega = (T)c.omega;
    p.beta = (T)c.params.beta;
    p.A_s = (T)c.params.A_s;
    p.eps2 = (T)(c.params.grad_eps * c.params.grad_eps);
    const int grid = (c.params.debug_flags & 2) ? 0 : adj_tiled_ctas<L, T>(c);
    if (grid > 0) {
        using C = AdjTile<L, T, kAdjBX, kAdjBY>;
        const mom::Sched sc = mom::plan(c.nx, c.ny, c.nz, kAdjBX, kAdjBY, grid);
        k_adjoint_cg_tiled<L, T, kAdjBX, kAdjBY><<<grid, C::NT, C::smem_bytes, c.stream>>>(
            static_cast<const T*>(lam_new), static_cast<const T*>(m), static_cast<T*>(lam), static_cast<T*>(lam_g),
            c.lay, p, sc, rows);
        *nrows = (size_t)grid;
    } else {  // reference form: one thread per node, neighbour fields loaded directly
        k_adjoint_cg_local<L, T><<<adj_grid(c), kAdjThreads, 0, c.stream>>>(
            static_cast<const T*>(lam_new), static_cast<const T*>(m), static_cast<T*>(lam), static_cast<T*>(lam_g),
            c.lay, p, rows);
        *nrows = (size_t)adj_grid(c).x * c.ny * c.nz;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adjoint_cg_phi<L, T><<<adj_grid(c), kAdjThreads, 0, c.stream>>>(static_cast<const T*>(m),
                                                                       static_cast<const T*>(lam_g),
                                                                       static_cast<T*>(lam), c.lay);
    return cudaGetLastError();
}

cudaError_t adj_cg_step(const llb_ctx& c, const void* lam_new, const void* m, void* lam, void* lam_g, double* rows,
                        size_t* nrows) {
    if (c.Q == 19)
        return c.storage == LLB_F64 ? adj_cg_step_t<D3Q19, double>(c, lam_new, m, lam, lam_g, rows, nrows)
                                    : adj_cg_step_t<D3Q19, float>(c, lam_new, m, lam, lam_g, rows, nrows);
    return c.storage == LLB_F64 ? adj_cg_step_t<D3Q27, double>(c, lam_new, m, lam, lam_g, rows, nrows)
                                : adj_cg_step_t<D3Q27, float>(c, lam_new, m, lam, lam_g, rows, nrows);
}

int grid_n(const llb_ctx& c) {
    const size_t want = (c.N + 255) / 256;
    const size_t cap = (size_t)(c.num_sms > 0 ? c.num_sms : 148) * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

// Advance the context by one step (same kernels as llb_step), flipping cur.
cudaError_t fwd_one(llb_ctx* c) {
    const void* in = c->buf[c->cur];
    void* out = c->buf[1 - c->cur];
    const cudaError_t e = c->ncomp == 2                   ? launch_cg_tiled(*c, in, out)
                          : c->kernel == LLB_KERNEL_TMA   ? launch_moment_tma(*c, c->cur, out)
                          : c->kernel == LLB_KERNEL_TILED ? launch_moment_tiled(*c, c->cur, in, out)
                                                          : launch_moment_direct(*c, in, out);
    if (e == cudaSuccess) c->cur = 1 - c->cur;
    return e;
}

}  // namespace

LLB_CHK_TU(adjoint)

}  // namespace llb

extern "C" int llb_adjoint(llb_ctx* c, int nsteps, int every, const void* dev_gfinal, void* dev_ginit, int dtype,
                           double* dtau) {
    using namespace llb;
    if (!c) return LLB_EINVAL;
    if (c->sticky != LLB_OK) return LLB_ESTATE;
    if (c->in_batch || c->scheme != LLB_SCHEME_MOMENT || (c->storage != LLB_F32 && c->storage != LLB_F64) ||
        nsteps < 0 || !dev_gfinal || !dev_ginit || (dtype != LLB_F64 && dtype != LLB_F32))
        return LLB_EINVAL;
    // two components: differentiable only without the near-contact switch and with the smooth normal
    const bool two = c->ncomp == 2;
    if (two && (c->params.A_h != 0.0 || !(c->params.grad_eps > 0.0))) return LLB_EINVAL;
    const int K = every > 0 ? every : (int)std::fmax(1.0, std::round(std::sqrt((double)nsteps)));
    const int nseg = nsteps > 0 ? (nsteps + K - 1) / K : 0;
    const size_t sb = c->state_bytes;
    // rows of dL/domega partial sums: one per block of the one-thread-per-node kernels,
    // or one per CTA of the tiled first pass (at most 32 per SM)
    const size_t nrows = std::max((size_t)adj_grid(*c).x * c->ny * c->nz, (size_t)32 * (c->num_sms > 0 ? c->num_sms : 1));
    // scratch: nseg checkpoints, K segment states, two cotangents, omega rows, accumulator
    std::vector<void*> ptrs;
    auto grab = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        return p;
    };
    auto release = [&]() {
        cudaStreamSynchronize(c->stream);
        for (void* p : ptrs) cudaFree(p);
        cudaGetLastError();
    };
    char* ck = static_cast<char*>(grab(sb * (size_t)(nseg > 0 ? nseg : 1)));
    char* seg = static_cast<char*>(grab(sb * (size_t)K));
    void* lamA = grab(sb);
    void* lamB = grab(sb);
    void* lamG = two ? grab(sb) : lamA;  // cotangent of G (3 fields), two components only
    double* rows = static_cast<double*>(grab(nrows * sizeof(double)));
    double* acc = static_cast<double*>(grab(sizeof(double)));
    if (!ck || !seg || !lamA || !lamB || !lamG || !rows || !acc) {
        release();
        return LLB_ENOMEM;
    }
    const int cur0 = c->cur;
    const long long t0 = c->t;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double), c->stream);
    // forward with checkpoints (checkpoint k = state at step k K)
    for (int s = 0; s < nsteps && e == cudaSuccess; ++s) {
        if (s % K == 0)
            e = cudaMemcpyAsync(ck + (size_t)(s / K) * sb, c->buf[c->cur], sb, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = fwd_one(c);
    }
    // cotangent of the final state
    if (e == cudaSuccess) {
        if (two && c->storage == LLB_F64)
            k_cot2_canon_to_internal<double><<<grid_n(*c), 256, 0, c->stream>>>(dev_gfinal, dtype, static_cast<double*>(lamA), c->lay);
        else if (two)
            k_cot2_canon_to_internal<float><<<grid_n(*c), 256, 0, c->stream>>>(dev_gfinal, dtype, static_cast<float*>(lamA), c->lay);
        else if (c->storage == LLB_F64)
            k_cot_canon_to_shifted<double><<<grid_n(*c), 256, 0, c->stream>>>(dev_gfinal, dtype, static_cast<double*>(lamA), c->lay);
        else
            k_cot_canon_to_shifted<float><<<grid_n(*c), 256, 0, c->stream>>>(dev_gfinal, dtype, static_cast<float*>(lamA), c->lay);
        e = cudaGetLastError();
    }
    void* lam_in = lamA;
    void* lam_out = lamB;
    for (int k = nseg - 1; k >= 0 && e == cudaSuccess; --k) {
        const int s0 = k * K, s1 = s0 + K < nsteps ? s0 + K : nsteps;
        // recompute the states s0 .. s1-1 of this segment from its checkpoint
        if (two) {
            // the two-component step takes any pair of state buffers: step slot to slot
            e = cudaMemcpyAsync(seg, ck + (size_t)k * sb, sb, cudaMemcpyDeviceToDevice, c->stream);
            for (int s = s0; s + 1 < s1 && e == cudaSuccess; ++s)
                e = launch_cg_tiled(*c, seg + (size_t)(s - s0) * sb, seg + (size_t)(s + 1 - s0) * sb);
        } else {
            e = cudaMemcpyAsync(c->buf[c->cur], ck + (size_t)k * sb, sb, cudaMemcpyDeviceToDevice, c->stream);
            for (int s = s0; s < s1 && e == cudaSuccess; ++s) {
                e = cudaMemcpyAsync(seg + (size_t)(s - s0) * sb, c->buf[c->cur], sb, cudaMemcpyDeviceToDevice,
                                    c->stream);
                if (e == cudaSuccess && s + 1 < s1) e = fwd_one(c);
            }
        }
        for (int s = s1 - 1; s >= s0 && e == cudaSuccess; --s) {
            size_t used = (size_t)adj_grid(*c).x * c->ny * c->nz;
            e = two ? adj_cg_step(*c, lam_in, seg + (size_t)(s - s0) * sb, lam_out, lamG, rows, &used)
                    : adj_step(*c, lam_in, seg + (size_t)(s - s0) * sb, lam_out, rows);
            if (e == cudaSuccess) {
                k_sum_rows<<<1, 256, 0, c->stream>>>(rows, used, acc);
                e = cudaGetLastError();
            }
            void* tmp = lam_in;
            lam_in = lam_out;
            lam_out = tmp;
        }
    }
    // cotangent of the initial state, in canonical form
    if (e == cudaSuccess) {
        if (two && c->storage == LLB_F64)
            k_cot2_internal_to_canon<double><<<grid_n(*c), 256, 0, c->stream>>>(static_cast<const double*>(lam_in), dev_ginit, dtype, c->lay);
        else if (two)
            k_cot2_internal_to_canon<float><<<grid_n(*c), 256, 0, c->stream>>>(static_cast<const float*>(lam_in), dev_ginit, dtype, c->lay);
        else if (c->storage == LLB_F64)
            k_cot_shifted_to_canon<double><<<grid_n(*c), 256, 0, c->stream>>>(static_cast<const double*>(lam_in), dev_ginit, dtype, c->lay);
        else
            k_cot_shifted_to_canon<float><<<grid_n(*c), 256, 0, c->stream>>>(static_cast<const float*>(lam_in), dev_ginit, dtype, c->lay);
        e = cudaGetLastError();
    }
    double domega = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&domega, acc, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    // restore the initial state
    if (e == cudaSuccess && nseg > 0) e = cudaMemcpyAsync(c->buf[cur0], ck, sb, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->cur = cur0;
    c->t = t0;
    release();
    if (e != cudaSuccess) {
        c->sticky = LLB_ECUDA;
        c->msg = std::string("adjoint: ") + cudaGetErrorString(e);
        return LLB_ECUDA;
    }
    // omega = 1 / tau
    if (dtau) *dtau = -domega / (c->tau * c->tau);
    return LLB_OK;
}
