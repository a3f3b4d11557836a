// Two-component moment-only step (colour gradient, near-contact force,
// recolouring): instances of the single-box kernel and their launch.
#include "cg_kernel.cuh"

namespace llb {
namespace {

using namespace cg;

template <class L, class T, class V>
int cg_ctas_v(const llb_ctx& c) {
    using C = CGCfg<L, T, V::BX, V::BY>;
    auto kern = k_cg_tiled<L, T, V::BX, V::BY, V::MINB, V::FAST, V::ROLLED>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_bytes) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, C::smem_bytes) != cudaSuccess ||
        per_sm < 1)
        return 0;
    const Sched2 sc = plan2(c.nx, c.ny, c.nz, V::BX, V::BY, per_sm * c.num_sms);
    return std::min(sc.nitems, per_sm * c.num_sms);
}

// Output planes zlo .. zhi-1 (all of them: 0, nz) on `st`.
template <class L, class T, class V>
cudaError_t cg_run_v(const llb_ctx& c, const void* in, void* out, int zlo, int zhi, cudaStream_t st) {
    using C = CGCfg<L, T, V::BX, V::BY>;
    const int grid = c.tile_ctas > 0 ? c.tile_ctas : 1;
    const Sched2 sc = plan2(c.nx, c.ny, zhi - zlo, V::BX, V::BY, grid);
    k_cg_tiled<L, T, V::BX, V::BY, V::MINB, V::FAST, V::ROLLED><<<grid, C::NT, C::smem_bytes, st>>>(
        static_cast<const T*>(in), static_cast<T*>(out), c.lay, cg_params<T>(c), sc, zlo, zhi - zlo);
    return cudaGetLastError();
}

}  // namespace

int cg_tiled_ctas(const llb_ctx& c) { LLB_CG(cg_ctas_v, c) }
cudaError_t launch_cg_tiled_range(const llb_ctx& c, const void* in, void* out, int zlo, int zhi, cudaStream_t st) {
    LLB_CG(cg_run_v, c, in, out, zlo, zhi, st)
}
cudaError_t launch_cg_tiled(const llb_ctx& c, const void* in, void* out) {
    return launch_cg_tiled_range(c, in, out, 0, c.nz, c.stream);
}

LLB_CHK_TU(cg)

}  // namespace llb
