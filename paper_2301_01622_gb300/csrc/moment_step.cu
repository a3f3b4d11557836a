// Moment-only lattice Boltzmann step, one component (Sec. II-III A): the
// direct kernel and the dispatch of the three kernels.
//
//   * k_moment_direct: one thread per output node, gathers the ten moments of
//     each of its Q neighbours and repeats the collision per neighbour.
//     Shape-agnostic; the reference GPU path.
//   * k_moment_tiled (moment_tiled.cuh, one translation unit per storage
//     type): persistent z-marching kernel with plain loads and a TMA L2
//     prefetch of the planes ahead; the default.
//   * k_moment_tma (moment_tma.cu): the same march with the planes staged in
//     shared memory by TMA box loads.
#include <cuda_runtime.h>

#include "moment_common.cuh"

namespace llb {
namespace {

using namespace mom;

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
                if (!LLB_IN(s, lay.fs, kChkLoad)) continue;
                const Mom<T> c = collide(load_mom<T>(in, s, lay.fs), omega);
                acc.add(g_dir<L, T>(c, g_shared(c), cx, cy, cz), cx, cy, cz);
            }
    store_node(out, lay, x, y, z, acc.finish());
}

template <class L, class T, class S>
cudaError_t run_direct(const llb_ctx& c, const void* in, void* out) {
    dim3 block(128), grid((c.nx + 127) / 128, c.ny, c.nz);
    k_moment_direct<L, T, S><<<grid, block, 0, c.stream>>>(static_cast<const S*>(in), static_cast<S*>(out), c.lay,
                                                            (T)c.omega);
    return cudaGetLastError();
}

}  // namespace

// (lattice, element type) -> kernel instance.  16-bit states compute in FP32.
cudaError_t launch_moment_direct(const llb_ctx& c, const void* in, void* out) {
    switch (c.storage) {
        case LLB_F64: return c.Q == 19 ? run_direct<D3Q19, double, double>(c, in, out)
                                       : run_direct<D3Q27, double, double>(c, in, out);
        case LLB_F16S: return c.Q == 19 ? run_direct<D3Q19, float, __half>(c, in, out)
                                        : run_direct<D3Q27, float, __half>(c, in, out);
        case LLB_BF16S: return c.Q == 19 ? run_direct<D3Q19, float, __nv_bfloat16>(c, in, out)
                                         : run_direct<D3Q27, float, __nv_bfloat16>(c, in, out);
        default: return c.Q == 19 ? run_direct<D3Q19, float, float>(c, in, out)
                                  : run_direct<D3Q27, float, float>(c, in, out);
    }
}

int moment_tiled_ctas(const llb_ctx& c) {
    switch (c.storage) {
        case LLB_F64: return moment_tiled_ctas_f64(c);
        case LLB_F16S: return moment_tiled_ctas_f16(c);
        case LLB_BF16S: return moment_tiled_ctas_bf16(c);
        default: return moment_tiled_ctas_f32(c);
    }
}

cudaError_t launch_moment_tiled_range(const llb_ctx& c, int in_index, const void* in, void* out, int zlo, int zhi,
                                      cudaStream_t st) {
    switch (c.storage) {
        case LLB_F64: return launch_moment_tiled_f64(c, in_index, in, out, zlo, zhi, st);
        case LLB_F16S: return launch_moment_tiled_f16(c, in_index, in, out, zlo, zhi, st);
        case LLB_BF16S: return launch_moment_tiled_bf16(c, in_index, in, out, zlo, zhi, st);
        default: return launch_moment_tiled_f32(c, in_index, in, out, zlo, zhi, st);
    }
}

cudaError_t launch_moment_tiled(const llb_ctx& c, int in_index, const void* in, void* out) {
    return launch_moment_tiled_range(c, in_index, in, out, 0, c.nz, c.stream);
}

bool moment_tiled_encode(const llb_ctx& c, void* buf, CUtensorMap* out) {
    int w = 0, h = 0;
    switch (c.storage) {
        case LLB_F64: moment_tiled_box_f64(c, &w, &h); break;
        case LLB_F16S: moment_tiled_box_f16(c, &w, &h); break;
        case LLB_BF16S: moment_tiled_box_bf16(c, &w, &h); break;
        default: moment_tiled_box_f32(c, &w, &h); break;
    }
    return encode_box_map(c, buf, w, h, out);
}

LLB_CHK_TU(step)

}  // namespace llb
