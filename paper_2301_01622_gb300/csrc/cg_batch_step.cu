// Two-component moment-only step for batched ensembles: instances of the
// kernel that walks the work items of every box of a batch, and their launch.
#include "cg_kernel.cuh"

namespace llb {
namespace {

using namespace cg;

template <class L, class T, class V>
int cg_batch_ctas_v(const llb_ctx& c) {
    using C = CGCfg<L, T, V::BX, V::BY>;
    auto kern = k_cg_batch<L, T, V::BX, V::BY, V::MINB, V::FAST, V::ROLLED>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem_bytes) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, C::smem_bytes) != cudaSuccess ||
        per_sm < 1)
        return 0;
    return per_sm * c.num_sms;
}

template <class L, class T, class V>
void cg_batch_plan_v(const llb_ctx& c, int grid, BatchDom* d) {
    const Sched2 sc = plan2(c.nx, c.ny, c.nz, V::BX, V::BY, grid);
    d->ncx = sc.ncx;
    d->ntiles = sc.ntiles;
    d->zc = sc.zc;
    d->nitems = sc.nitems;
}

template <class L, class T, class V>
cudaError_t cg_batch_run_v(const llb_ctx& c, const BatchDom* doms, int ndom, int total, int grid, int* next) {
    using C = CGCfg<L, T, V::BX, V::BY>;
    k_cg_batch<L, T, V::BX, V::BY, V::MINB, V::FAST, V::ROLLED><<<grid, C::NT, C::smem_bytes, c.stream>>>(
        doms, ndom, total, cg_params<T>(c), next);
    return cudaGetLastError();
}

}  // namespace

int cg_batch_ctas(const llb_ctx& c) { LLB_CG(cg_batch_ctas_v, c) }
void cg_batch_plan(const llb_ctx& c, int grid, BatchDom* d) { LLB_CG(cg_batch_plan_v, c, grid, d) }
cudaError_t launch_cg_batch(const llb_ctx& c, const BatchDom* doms, int ndom, int total, int grid, int* next) {
    LLB_CG(cg_batch_run_v, c, doms, ndom, total, grid, next)
}

LLB_CHK_TU(cg_batch)

}  // namespace llb
