// Tiled z-marching moment-only kernel (one component), plain loads.
//
// A persistent CTA owns a BX x BY column of output nodes and walks it plane
// by plane.  For every source plane it collides each node of the tile plus a
// one-node halo ONCE, evaluates the Q-3 populations that cross to another
// column and publishes them in shared memory; each output thread then pulls
// one scalar per direction (instead of ten moments) and adds it into one of
// three rolling per-plane accumulators (planes s-1, s, s+1).  Each moment is
// read from and written to HBM once per step.
//
// Loads: the moments of the next source plane are loaded into the registers
// of the node just collided (one plane ahead).  With kPrefetch, one thread
// of the CTA also asks the TMA unit to prefetch the tile-plus-halo box of
// the source plane PD steps ahead into L2 (cp.async.bulk.prefetch.tensor),
// so that those register loads hit L2 instead of waiting on HBM; the
// prefetch cursor runs on into the CTA's next work item.
//
// This header holds the kernel and its host-side launch templates; each
// storage type instantiates them in its own translation unit.
#pragma once

#include <algorithm>

#include "moment_common.cuh"

namespace llb {
namespace mom {

// Options of the tiled kernel (bit flags):
//   kSplit    -- split-phase plane barrier: each thread arrives on an mbarrier
//                as soon as its populations are published, stores the plane
//                finished one step earlier while the others catch up, and only
//                then waits (bounded) before pulling; replaces __syncthreads.
//   kFastRcp  -- FP32 collision with the approximate division for 1/rho.
//   kPrefetch -- TMA prefetch of the source plane PD steps ahead into L2.
constexpr int kSplit = 1, kFastRcp = 2, kPrefetch = 4;

__device__ __forceinline__ void tma_prefetch_l2_4d(const CUtensorMap* map, int c0, int c1, int c2, int c3) {
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}

template <class L, class T, int BX, int BY>
struct Tiled {
    static constexpr int NT = BX * BY;             // threads = output columns of a tile
    static constexpr int HX = BX + 2, HY = BY + 2; // tile plus one-node halo
    static constexpr int HN = HX * HY;
    static constexpr int NH = 2 * BX + 2 * BY + 4; // halo nodes, one per thread t < NH
    static constexpr int NS = n_xy_shifted<L>();   // directions crossing columns
    static constexpr size_t g_bytes = sizeof(T) * 2 * NS * HN;
    static constexpr size_t smem_bytes = g_bytes + 16;  // + two mbarriers (split-phase option)
    static_assert(NH <= NT, "halo must fit one node per thread");
    static_assert(NT % 32 == 0, "whole warps");
    static_assert(g_bytes % 8 == 0, "mbarriers need 8-byte alignment");
};

// Columns of padding on each side of the prefetch box, so that its x start
// times the element size is a multiple of 16 bytes.
template <class S>
constexpr int pf_pad() { return 16 / (int)sizeof(S) > 4 ? 16 / (int)sizeof(S) : 4; }

// Moments of a node of plane offset zoff: field-major storage addresses them
// from the node's own pointer p (kept per work item); the interleaved FP32
// state needs the node's absolute index o + zoff (its field offsets depend on
// it).  Likewise for the store of an output node at q (absolute index q - out).
template <class S>
__device__ __forceinline__ RawMom<S> load_node_raw(const S* __restrict__ in, const S* __restrict__ p, long long o,
                                                   size_t zoff, size_t fs) {
    if constexpr (FieldMap<S, 10>::kInterleaved)
        return load_raw(in, (size_t)o + zoff, fs);
    else
        return load_raw(p + zoff, 0, fs);
}

template <class T, class S>
__device__ __forceinline__ void store_node_mom(S* __restrict__ out, S* __restrict__ q, size_t fs, const Mom<T>& m) {
    if constexpr (FieldMap<S, 10>::kInterleaved)
        store_mom(out, (size_t)(q - out), fs, m);
    else
        store_mom(q, 0, fs, m);
}

template <class L, class T, int BX, int BY, int MINB, int OPT, int PD, class S>
__global__ void __launch_bounds__(BX * BY, MINB)
    k_moment_tiled(const S* __restrict__ in, S* __restrict__ out, Layout lay, T omega, Sched sc, int zlo, int nzr,
                   int* err, long long budget, const __grid_constant__ CUtensorMap pmap, int pf_enable) {
    using K = Tiled<L, T, BX, BY>;
    constexpr int HX = K::HX, HN = K::HN, NS = K::NS;
    constexpr bool SPLIT = (OPT & kSplit) != 0, FAST = (OPT & kFastRcp) != 0, PF = (OPT & kPrefetch) != 0;
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
    int hx2, hy2, sx2;
    const int role2 = halo_node<BX, BY>(t, hx2, hy2, sx2);
    const bool has2 = role2 != kNone;
    const int n2 = hy2 * HX + hx2;
    const size_t plane = (size_t)lay.px * lay.py;
    int buf = 0;

    // L2 prefetch cursor: item and source plane of the next box to prefetch
    // (used by lane 0 of the last warp, which has no halo node to collide;
    // off when the context could not encode the prefetch map).
    const bool pf_thread = PF && pf_enable && t == K::NT - 32;
    int p_it = blockIdx.x, p_x0 = 0, p_y0 = 0, p_s = 0, p_zb = -1;
    auto pf_issue = [&]() {
        if (p_it >= sc.nitems) return;
        if (p_s > p_zb) return;
        tma_prefetch_l2_4d(&pmap, p_x0 + lay.xo - pf_pad<S>(), p_y0 + lay.yo - 1, pmod(p_s, nz), 0);
        if (++p_s > p_zb) {
            p_it += gridDim.x;
            if (p_it < sc.nitems) {
                int za2, zb2;
                sc.item(p_it, BX, BY, nzr, p_x0, p_y0, za2, zb2);
                p_s = zlo + za2 - 1;
                p_zb = zlo + zb2;
            }
        }
    };
    if (pf_thread && p_it < sc.nitems) {
        int za2, zb2;
        sc.item(p_it, BX, BY, nzr, p_x0, p_y0, za2, zb2);
        p_s = zlo + za2 - 1;
        p_zb = zlo + zb2;
        for (int k = 0; k <= PD; ++k) pf_issue();
    }

    for (int it = blockIdx.x; it < sc.nitems; it += gridDim.x) {
        int x0, y0, za, zb;  // outputs za .. zb-1 of the tile at (x0, y0)
        sc.item(it, BX, BY, nzr, x0, y0, za, zb);
        za += zlo;            // the items cover output planes zlo .. zlo + nzr - 1
        zb += zlo;
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
        const long long o1 = in1 - in, o2 = in2 - in;  // node offsets within a field (plane 0)
        RawMom<S> m1{}, m2{};  // converted at the collision
        if (LLB_IN(o1 + (long long)zn_off, lay.fs, kChkLoad)) m1 = load_node_raw(in, in1, o1, zn_off, lay.fs);
        if (has2 && LLB_IN(o2 + (long long)zn_off, lay.fs, kChkLoad)) m2 = load_node_raw(in, in2, o2, zn_off, lay.fs);

        Acc<T> a0, a1, a2;
        a0.zero(); a1.zero(); a2.zero();

        auto put = [&](const Acc<T>& A, int z) {
            const Mom<T> r = A.finish();
            if (LLB_IN(out1 - out, lay.fs, kChkStore)) store_node_mom(out, out1, lay.fs, r);
            if (ghost) store_node(out, lay, ox, oy, z, r);
            out1 += plane;
        };

        // One source plane s: X, Y, Z accumulate output planes s-1, s, s+1.
        // Without kSplit, plane s-1 is finished and stored here; with kSplit
        // it is stored in the next step (from Z, before Z restarts as s+2).
        auto plane_step = [&](int s, Acc<T>& X, Acc<T>& Y, Acc<T>& Z) -> bool {
            T* const G = Gbase + buf * (NS * HN);
            if constexpr (PF) {
                if (pf_thread) pf_issue();
            }
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
            const Mom<T> c1 = collide<T, FAST>(from_raw<T>(m1), omega);
            if (more && LLB_IN(o1 + (long long)zn_off, lay.fs, kChkLoad)) m1 = load_node_raw(in, in1, o1, zn_off, lay.fs);
            publish<L, T, HN>(G, n1, c1);
            T g_m, g_0, g_p;
            own_column<L, T>(c1, g_m, g_0, g_p);
            if (has2) {
                const Mom<T> c2 = collide<T, FAST>(from_raw<T>(m2), omega);
                if (more && LLB_IN(o2 + (long long)zn_off, lay.fs, kChkLoad)) m2 = load_node_raw(in, in2, o2, zn_off, lay.fs);
                publish_halo<L, T, HN>(G, n2, role2, sx2, c2);
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

// Plain-load tiled kernel shapes: tile BX x BY, CTAs per SM the register
// budget targets, options, prefetch distance in planes.
template <int BX_, int BY_, int MINB_, int OPT_ = 0, int PD_ = 2>
struct TiledShape {
    static constexpr int BX = BX_, BY = BY_, MINB = MINB_, OPT = OPT_, PD = PD_;
};

// FP32 variants (0 = default).  The approximate 1/rho is used by all but
// variant 2 (measured ~1.5 % faster at 256^3, error far below FP32 storage
// rounding).  The L2 prefetch (variant 1) measured 5 % slower than plain
// loads on GB300 and is kept for the autotuner.
constexpr int kTiledVariants = kTiledVariants32;
template <class T, int V> struct TiledVariant { using type = TiledShape<64, 4, 2, kFastRcp>; };
template <> struct TiledVariant<float, 1> { using type = TiledShape<64, 4, 2, kFastRcp | kPrefetch, 2>; };
template <> struct TiledVariant<float, 2> { using type = TiledShape<64, 4, 2, 0>; };
template <> struct TiledVariant<float, 3> { using type = TiledShape<64, 8, 1, kFastRcp>; };
template <> struct TiledVariant<float, 4> { using type = TiledShape<32, 8, 2, kFastRcp>; };
template <> struct TiledVariant<float, 5> { using type = TiledShape<64, 4, 2, kSplit | kFastRcp>; };
// FP64: one shape (32 x 8, one CTA per SM, IEEE division).
template <int V> struct TiledVariant<double, V> { using type = TiledShape<32, 8, 1, 0>; };

template <class L, class T, class St, class S>
int tiled_ctas_c(const llb_ctx& c) {
    using K = Tiled<L, T, S::BX, S::BY>;
    auto kern = k_moment_tiled<L, T, S::BX, S::BY, S::MINB, S::OPT, S::PD, St>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem_bytes) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, K::NT, K::smem_bytes) != cudaSuccess ||
        per_sm < 1)
        return 0;
    const Sched sc = plan(c.nx, c.ny, c.nz, S::BX, S::BY, per_sm * c.num_sms);
    return std::min(sc.nitems, per_sm * c.num_sms);
}

// Output planes zlo .. zhi-1 (all of them: 0, nz) on `stream`.
template <class L, class T, class St, class S>
cudaError_t run_tiled_c(const llb_ctx& c, int in_index, const void* in, void* out, int zlo, int zhi,
                        cudaStream_t stream) {
    using K = Tiled<L, T, S::BX, S::BY>;
    const int grid = c.tile_ctas > 0 ? c.tile_ctas : 1;
    const Sched sc = plan(c.nx, c.ny, zhi - zlo, S::BX, S::BY, grid);
    // device clock ~2 GHz: cycles per millisecond
    const long long budget = (long long)c.params.wait_budget_ms * 2000000LL;
    k_moment_tiled<L, T, S::BX, S::BY, S::MINB, S::OPT, S::PD, St><<<grid, K::NT, K::smem_bytes, stream>>>(
        static_cast<const St*>(in), static_cast<St*>(out), c.lay, (T)c.omega, sc, zlo, zhi - zlo,
        static_cast<int*>(c.err_dev), budget, c.pmap[in_index], c.pmap_ok ? 1 : 0);
    return cudaGetLastError();
}

// Box of the L2 prefetch of variant S: the tile plus its halo, widened in x
// to 16-byte boundaries.
template <class St, class S>
void tiled_box(int* w, int* h) {
    *w = S::BX + 2 * pf_pad<St>();
    *h = S::BY + 2;
}

}  // namespace mom
}  // namespace llb

// Instantiate the per-storage entry points of the tiled kernel for compute
// type T and storage type St (VMAX: number of variants this storage offers).
#define LLB_TILED_ENTRY(SUFFIX, T, St, VMAX)                                                                   \
    namespace llb {                                                                                            \
    namespace {                                                                                                \
    template <class L>                                                                                         \
    int ctas_l(const llb_ctx& c) {                                                                             \
        switch (c.variant < VMAX ? c.variant : 0) {                                                            \
            case 1: return mom::tiled_ctas_c<L, T, St, typename mom::TiledVariant<T, 1 % VMAX>::type>(c);      \
            case 2: return mom::tiled_ctas_c<L, T, St, typename mom::TiledVariant<T, 2 % VMAX>::type>(c);      \
            case 3: return mom::tiled_ctas_c<L, T, St, typename mom::TiledVariant<T, 3 % VMAX>::type>(c);      \
            case 4: return mom::tiled_ctas_c<L, T, St, typename mom::TiledVariant<T, 4 % VMAX>::type>(c);      \
            case 5: return mom::tiled_ctas_c<L, T, St, typename mom::TiledVariant<T, 5 % VMAX>::type>(c);      \
            default: return mom::tiled_ctas_c<L, T, St, typename mom::TiledVariant<T, 0>::type>(c);            \
        }                                                                                                      \
    }                                                                                                          \
    template <class L>                                                                                         \
    cudaError_t run_l(const llb_ctx& c, int in_index, const void* in, void* out, int zlo, int zhi,         \
                      cudaStream_t st) {                             \
        switch (c.variant < VMAX ? c.variant : 0) {                                                            \
            case 1: return mom::run_tiled_c<L, T, St, typename mom::TiledVariant<T, 1 % VMAX>::type>(c, in_index, in, out, zlo, zhi, st); \
            case 2: return mom::run_tiled_c<L, T, St, typename mom::TiledVariant<T, 2 % VMAX>::type>(c, in_index, in, out, zlo, zhi, st); \
            case 3: return mom::run_tiled_c<L, T, St, typename mom::TiledVariant<T, 3 % VMAX>::type>(c, in_index, in, out, zlo, zhi, st); \
            case 4: return mom::run_tiled_c<L, T, St, typename mom::TiledVariant<T, 4 % VMAX>::type>(c, in_index, in, out, zlo, zhi, st); \
            case 5: return mom::run_tiled_c<L, T, St, typename mom::TiledVariant<T, 5 % VMAX>::type>(c, in_index, in, out, zlo, zhi, st); \
            default: return mom::run_tiled_c<L, T, St, typename mom::TiledVariant<T, 0>::type>(c, in_index, in, out, zlo, zhi, st); \
        }                                                                                                      \
    }                                                                                                          \
    template <class L>                                                                                         \
    void box_l(const llb_ctx& c, int* w, int* h) {                                                             \
        switch (c.variant < VMAX ? c.variant : 0) {                                                            \
            case 1: return mom::tiled_box<St, typename mom::TiledVariant<T, 1 % VMAX>::type>(w, h);            \
            case 2: return mom::tiled_box<St, typename mom::TiledVariant<T, 2 % VMAX>::type>(w, h);            \
            case 3: return mom::tiled_box<St, typename mom::TiledVariant<T, 3 % VMAX>::type>(w, h);            \
            case 4: return mom::tiled_box<St, typename mom::TiledVariant<T, 4 % VMAX>::type>(w, h);            \
            case 5: return mom::tiled_box<St, typename mom::TiledVariant<T, 5 % VMAX>::type>(w, h);            \
            default: return mom::tiled_box<St, typename mom::TiledVariant<T, 0>::type>(w, h);                  \
        }                                                                                                      \
    }                                                                                                          \
    }                                                                                                          \
    int moment_tiled_ctas_##SUFFIX(const llb_ctx& c) {                                                         \
        return c.Q == 19 ? ctas_l<D3Q19>(c) : ctas_l<D3Q27>(c);                                                \
    }                                                                                                          \
    cudaError_t launch_moment_tiled_##SUFFIX(const llb_ctx& c, int in_index, const void* in, void* out,        \
                                             int zlo, int zhi, cudaStream_t st) {                              \
        return c.Q == 19 ? run_l<D3Q19>(c, in_index, in, out, zlo, zhi, st)                                    \
                         : run_l<D3Q27>(c, in_index, in, out, zlo, zhi, st);                                   \
    }                                                                                                          \
    void moment_tiled_box_##SUFFIX(const llb_ctx& c, int* w, int* h) {                                         \
        if (c.Q == 19) box_l<D3Q19>(c, w, h); else box_l<D3Q27>(c, w, h);                                      \
    }                                                                                                          \
    LLB_CHK_TU(tiled_##SUFFIX)                                                                                 \
    }
