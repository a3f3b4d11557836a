// Bounds checks of the LLB_CHECKED build.
//
// Compiled with -DLLB_CHECKED, every shared-memory and global-memory index of
// the stencil kernels is compared with the extent of its buffer before the
// access; an index out of range skips the access and is recorded, together
// with a site code, in a device word of the translation unit (the first one
// wins).  Nothing traps: the kernel carries on and the host reads the record
// with llb_checked_status.  In the normal build the checks compile to nothing.
#pragma once

#include <cuda_runtime.h>

namespace llb {

// Site codes of the checked accesses.
enum ChkSite {
    kChkNone = 0,
    kChkPublish = 1,   // exchange-buffer write (node slot of a tile or halo node)
    kChkGather = 2,    // exchange-buffer read (neighbour slots of an output node)
    kChkLoad = 3,      // state load (node offset within one field)
    kChkStore = 4,     // state store of an output node
    kChkGhost = 5,     // state store of a periodic ghost copy
    kChkStage = 6,     // TMA stage read
    kChkPhi = 7,       // phase-field ring read or write
    kChkProbe = 8,     // near-contact probe read
    kChkPop = 9,       // population or phase-field array access
};

struct ChkWord {
    int site;
    int pad;
    long long index;
};

#ifdef LLB_CHECKED
namespace {
__device__ ChkWord g_chk;  // one per translation unit
}

__device__ __forceinline__ bool chk_in(long long i, long long n, int site) {
    if (i >= 0 && i < n) return true;
    if (atomicCAS(&g_chk.site, 0, site) == 0) g_chk.index = i;
    return false;
}

#define LLB_IN(i, n, site) ::llb::chk_in((long long)(i), (long long)(n), (site))
// index i, or 0 (recorded) when it is out of [0, n)
#define LLB_CLAMP(i, n, site) (LLB_IN((i), (n), (site)) ? (i) : decltype(i)(0))

// Read and clear this translation unit's record (host side, after a device sync).
#define LLB_CHK_TU(name)                                                                    \
    int chk_take_##name(int* site, long long* index) {                                     \
        ChkWord w{};                                                                       \
        if (cudaMemcpyFromSymbol(&w, g_chk, sizeof(w)) != cudaSuccess) return -1;          \
        const ChkWord z{};                                                                 \
        if (w.site && cudaMemcpyToSymbol(g_chk, &z, sizeof(z)) != cudaSuccess) return -1;  \
        *site = w.site;                                                                    \
        *index = w.index;                                                                  \
        return 0;                                                                          \
    }
#else
#define LLB_IN(i, n, site) true
#define LLB_CLAMP(i, n, site) (i)
#define LLB_CHK_TU(name)                                  \
    int chk_take_##name(int* site, long long* index) {   \
        *site = 0;                                       \
        *index = 0;                                      \
        return 0;                                        \
    }
#endif

}  // namespace llb
