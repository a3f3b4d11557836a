// TMA-staged z-marching moment-only kernel (one component), and the TMA
// tensor maps of the moment state.
//
// The computation is that of the tiled kernel (moment_tiled.cuh): per source
// plane, every node of the tile plus a one-node halo is collided once and
// publishes its column-crossing populations in shared memory, and each output
// thread pulls one scalar per direction into three rolling accumulators.
// Here the tile-plus-halo moments of each source plane are fetched by one TMA
// box load into an NST-deep ring of shared-memory stages (mbarrier
// completion), so that several planes of loads are in flight per CTA without
// holding registers.  Needs the padded layout (periodic ghosts, 16-byte
// aligned tile start).  Every mbarrier wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "moment_common.cuh"

namespace llb {
namespace {

using namespace mom;

template <class L, class T, int BX_, int BY_, int NST_, int MINB_>
struct TmaCfg {
    static constexpr int BX = BX_, BY = BY_, NST = NST_;
    static constexpr int NT = BX * BY;
    static constexpr int HX = BX + 2, HY = BY + 2, HN = HX * HY, NH = 2 * BX + 2 * BY + 4;
    static constexpr int NS = n_xy_shifted<L>();
    // the interleaved FP32 state (FieldMap) is staged in whole 32-node blocks:
    // NB blocks cover the padded columns x0+7 .. x0+BX+8 of the tile and halo
    static constexpr bool IL = FieldMap<T, 10>::kInterleaved;
    static constexpr int NB = BX / 32 + 1;
    static constexpr int SW = IL ? 32 * NB : BX + 8;  // staged row: blocks, or x0-4 .. x0+BX+3
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
    static_assert(!IL || BX % 32 == 0, "interleaved boxes need tiles of whole 32-node blocks");
};

// Moments of staged node (hx, hy) of the tile plus halo.  Field-major stage:
// [field][row][x0-4 ..]; interleaved stage: [row][block][field][lane], node
// hx at padded column x0+7+hx.
template <class T, class C>
__device__ __forceinline__ Mom<T> stage_mom(const T* __restrict__ S, int hx, int hy) {
    constexpr int SF = C::SF, SW = C::SW;
    Mom<T> m{};
    int o, fstep;
    if constexpr (C::IL) {
        const int rel = 7 + hx;
        o = ((hy * C::NB + (rel >> 5)) * 10) * 32 + (rel & 31);
        fstep = 32;
    } else {
        o = hy * SW + hx + 3;
        fstep = SF;
    }
    if (!LLB_IN(o + 9 * fstep, 10 * SF, kChkStage)) return m;
    const T* p = S + o;
    m.d = p[0];
    m.jx = p[fstep];
    m.jy = p[2 * fstep];
    m.jz = p[3 * fstep];
    m.axx = p[4 * fstep];
    m.ayy = p[5 * fstep];
    m.azz = p[6 * fstep];
    m.axy = p[7 * fstep];
    m.axz = p[8 * fstep];
    m.ayz = p[9 * fstep];
    return m;
}

// One stage load: the tile-plus-halo box of plane z.
template <class C>
__device__ __forceinline__ void stage_load(uint32_t dst, const CUtensorMap* map, const Layout& lay, int x0, int y0, int z,
                                           uint32_t bar) {
    if constexpr (C::IL)
        tma_load_5d(dst, map, 0, 0, (x0 + lay.xo - 1) / 32, y0 + lay.yo - 1, z, bar);
    else
        tma_load_4d(dst, map, x0 + lay.xo - 4, y0 + lay.yo - 1, z, 0, bar);
}

template <class L, class T, class C>
__global__ void __launch_bounds__(C::NT, C::MINB)
    k_moment_tma(const __grid_constant__ CUtensorMap tmap, T* __restrict__ out, Layout lay, T omega, Sched sc,
                 int* __restrict__ err, long long wait_budget, int extra_tx) {
    constexpr int BX = C::BX, BY = C::BY, NST = C::NST, HX = C::HX, HN = C::HN, NS = C::NS;
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
    int hx2, hy2, sx2;
    const int role2 = halo_node<BX, BY>(t, hx2, hy2, sx2);
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
                stage_load<C>(stage0 + (qq % NST) * C::STAGE_STRIDE, &tmap, lay, x0, y0, pmod(za - 1 + i, nz), bar);
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
                const Mom<T> c1 = collide<T, true>(stage_mom<T, C>(S, tx + 1, ty + 1), omega);
                publish<L, T, HN>(G, n1, c1);
                own_column<L, T>(c1, g_m, g_0, g_p);
                if (has2)
                    publish_halo<L, T, HN>(G, n2, role2, sx2,
                                           collide<T, true>(stage_mom<T, C>(S, hx2, hy2), omega));
            }
            if (__syncthreads_or(!ok)) return false;
            // every thread is done with stage k: refill it with plane s + NST
            if (t == 0 && (int)(q - q0) + NST < P) {
                fence_proxy_async();
                const unsigned qq = q + NST;
                const uint32_t bar = bar0 + 8 * k;
                mbar_arrive_expect_tx(bar, C::STAGE_BYTES + extra_tx);
                stage_load<C>(stage0 + k * C::STAGE_STRIDE, &tmap, lay, x0, y0, pmod(s + NST, nz), bar);
                issued = qq + 1;
            }
            gather<L, T, HN, HX>(G, n1, g_m, g_0, g_p, X, Y, Z);
            if (s - 1 >= za && store_ok) {
                const Mom<T> r = X.finish();
                if (LLB_IN(out1 - out, lay.fs, kChkStore)) {
                    if constexpr (C::IL)
                        store_mom(out, (size_t)(out1 - out), lay.fs, r);  // absolute index (interleaved)
                    else
                        store_mom(out1, 0, lay.fs, r);
                }
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

// TMA kernel variants (tile BX x BY, ring depth, CTAs per SM).  Variant 0 is
// the default.  Ring depths are chosen so that two CTAs of the 256-thread
// tiles fit in the shared memory of one SM (2-3 x 17 KB stages + 51 KB
// exchange buffers); the 2-deep ring measured fastest on 256^3.
template <class L, class T, int V>
struct TmaVariant;
template <class L> struct TmaVariant<L, float, 0> { using type = TmaCfg<L, float, 64, 4, 2, 2>; };
template <class L> struct TmaVariant<L, float, 1> { using type = TmaCfg<L, float, 64, 4, 3, 2>; };
template <class L> struct TmaVariant<L, float, 2> { using type = TmaCfg<L, float, 32, 8, 3, 2>; };
template <class L, int V> struct TmaVariant<L, double, V> { using type = TmaCfg<L, double, 32, 8, 2, 1>; };

template <class L, class T, class C>
int tma_ctas_c(const llb_ctx& c) {
    if (c.variant >= kTmaVariants) return 0;
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
    return encode_box_map(c, buf, C::SW, C::SR, out);
}

#define LLB_TMA_VARIANT(fn, ...)                                                                  \
    switch (c.variant) {                                                                          \
        case 1: return fn<L, T, typename TmaVariant<L, T, 1>::type>(__VA_ARGS__);                 \
        case 2: return fn<L, T, typename TmaVariant<L, T, 2>::type>(__VA_ARGS__);                 \
        default: return fn<L, T, typename TmaVariant<L, T, 0>::type>(__VA_ARGS__);                \
    }

template <class L, class T>
int tma_ctas(const llb_ctx& c) { LLB_TMA_VARIANT(tma_ctas_c, c) }
template <class L, class T>
cudaError_t run_tma(const llb_ctx& c, int in_index, void* out) { LLB_TMA_VARIANT(run_tma_c, c, in_index, out) }
template <class L, class T>
bool tma_encode(const llb_ctx& c, void* buf, CUtensorMap* out) { LLB_TMA_VARIANT(tma_encode_c, c, buf, out) }

}  // namespace

// 4D tensor map (x, y, z, field) of a moment state buffer with a box of
// box_w x box_h nodes of one plane and all ten fields, element type of the
// context's storage.  False if the driver entry point or the encoding fails.
bool encode_box_map(const llb_ctx& c, void* buf, int box_w, int box_h, CUtensorMap* out) {
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
    if (!Lo.ghosts || c.ncomp != 1 || box_w > 256 || box_h > 256) return false;
    CUtensorMapDataType dt;
    switch (c.storage) {
        case LLB_F64: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; break;
        case LLB_F32: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
        case LLB_F16S: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
        case LLB_BF16S: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
        default: return false;
    }
    const size_t es = elem_size(c.storage);
    if (c.storage == LLB_F32) {
        // interleaved state (FieldMap): dims (lane, field, 32-node block, y, z);
        // a box of box_w / 32 whole blocks, all ten fields
        if (box_w % 32 != 0 || Lo.px % 32 != 0) return false;
        const cuuint64_t dims[5] = {32, 10, (cuuint64_t)Lo.px / 32, (cuuint64_t)Lo.py, (cuuint64_t)Lo.nz};
        const cuuint64_t strides[4] = {32 * es, 320 * es, (cuuint64_t)Lo.px * 10 * es,
                                       (cuuint64_t)Lo.px * Lo.py * 10 * es};
        const cuuint32_t box[5] = {32, 10, (cuuint32_t)box_w / 32, (cuuint32_t)box_h, 1};
        const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        return encode(out, dt, 5, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    if ((size_t)box_w * es % 16 != 0) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)Lo.px, (cuuint64_t)Lo.py, (cuuint64_t)Lo.nz, 10};
    const cuuint64_t strides[3] = {(cuuint64_t)Lo.px * es, (cuuint64_t)Lo.px * Lo.py * es, (cuuint64_t)Lo.fs * es};
    const cuuint32_t box[4] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1, 10};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = encode(out, dt, 4, buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The TMA kernel stages FP32 or FP64 boxes only.
#define LLB_MDISPATCH(fn, fallback, ...)                                                          \
    switch (c.storage) {                                                                          \
        case LLB_F64: return c.Q == 19 ? fn<D3Q19, double>(__VA_ARGS__) : fn<D3Q27, double>(__VA_ARGS__); \
        case LLB_F32: return c.Q == 19 ? fn<D3Q19, float>(__VA_ARGS__) : fn<D3Q27, float>(__VA_ARGS__);   \
        default: return fallback;                                                                 \
    }

int moment_tma_ctas(const llb_ctx& c) { LLB_MDISPATCH(tma_ctas, 0, c) }
cudaError_t launch_moment_tma(const llb_ctx& c, int in_index, void* out) {
    LLB_MDISPATCH(run_tma, cudaErrorInvalidValue, c, in_index, out)
}
bool moment_tma_encode(const llb_ctx& c, void* buf, CUtensorMap* out) {
    LLB_MDISPATCH(tma_encode, false, c, buf, out)
}

LLB_CHK_TU(tma)

}  // namespace llb
