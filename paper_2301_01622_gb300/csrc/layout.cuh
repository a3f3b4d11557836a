// Memory layout of moment fields on the device.
//
// A moment buffer is field-major: field f starts at f * fs elements.  Inside
// a field, node (x, y, z) sits at ((z * py) + (y + yo)) * px + (x + xo).
//
// Dense layout (xo = yo = 0, px = nx, py = ny): used for temporaries of the
// population-storing schemes.
//
// Padded layout (moment-only state): xo = 8, yo = gy (1 or 2), px = nx + 16
// rounded up to a multiple of 8, py = ny + 2 gy.  Node x = 0 then starts a
// 32-byte sector in FP32 (64 bytes in FP64), so a warp that stores 32
// consecutive nodes writes whole sectors and HBM never has to read a sector
// back to merge a partial write.  The eight columns on each side and the gy
// rows above and below hold periodic ghost copies: columns x = -8..-1 hold
// x = nx-8..nx-1, columns x = nx..nx+7 hold x = 0..7, rows y = -gy..-1 hold
// y = ny-gy..ny-1 and rows y = ny..ny+gy-1 hold y = 0..gy-1 (corners
// likewise), written by every kernel that writes the state.  Whole sectors
// of ghosts are written for the same reason.  With them the tile plus halo a
// CTA needs is one rectangular box with a 16-byte aligned x start, so one
// TMA load fetches it without wrapping.
//
// Field order inside a buffer (FieldMap): field-major, f * fs + i, for every
// state except the one-component FP32 state, which interleaves its ten
// fields per block of 32 consecutive node indices: field f of node i sits at
// (i & ~31) * 10 + 32 f + (i & 31).  A thread then reaches every field of
// its node at a constant offset from one address, and the ten fields of a
// warp's 32 nodes are one contiguous 1280-byte run.  That state's row pitch
// is a multiple of 32 (blocks never straddle rows).  Every field stride fs is
// a multiple of 32, so the last block of an interleaved buffer stays inside
// NF * fs elements.
#pragma once

#include <cstddef>
#include <type_traits>

namespace llb {

struct Layout {
    int nx, ny, nz;
    int px, py;   // row pitch (elements) and rows per plane
    int xo, yo;   // offset of node (0, 0) inside a plane; yo = ghost rows per side
    size_t fs;    // field stride in elements
    int ghosts;   // 1: periodic ghost copies are maintained

    __host__ __device__ __forceinline__ size_t at(int x, int y, int z) const {
        return ((size_t)z * py + (y + yo)) * (size_t)px + (x + xo);
    }
};

constexpr int kGhostX = 8;  // ghost columns per side (one FP32 sector)

// Element offset of field f of node i in a buffer of NF fields of type S.
template <class S, int NF>
struct FieldMap {
    static constexpr bool kInterleaved = std::is_same<S, float>::value && NF == 10;
    __host__ __device__ __forceinline__ static size_t at(size_t i, int f, size_t fs) {
        if constexpr (kInterleaved)
            return (i & ~size_t(31)) * NF + (size_t)f * 32 + (i & 31);
        else
            return (size_t)f * fs + i;
    }
};

// row_align: multiple the padded row pitch is rounded up to (8; 32 for the
// interleaved one-component FP32 state).
inline Layout make_layout(int nx, int ny, int nz, bool padded, int ghost_rows = 1, int row_align = 8) {
    Layout L;
    L.nx = nx; L.ny = ny; L.nz = nz;
    if (padded) {
        L.xo = kGhostX; L.yo = ghost_rows;
        L.px = ((nx + 2 * kGhostX + row_align - 1) / row_align) * row_align;
        L.py = ny + 2 * ghost_rows;
        L.ghosts = 1;
    } else {
        L.xo = 0; L.yo = 0;
        L.px = nx; L.py = ny;
        L.ghosts = 0;
    }
    L.fs = ((size_t)L.px * L.py * nz + 31) / 32 * 32;
    return L;
}

// Call fn(x', y') for (x, y) and, in a padded layout, for every ghost
// position that mirrors (x, y) under the periodic wrap: x' = x -+ nx inside
// the ghost columns [-8, nx + 8), y' = y -+ ny inside the ghost rows.
template <class F>
__device__ __forceinline__ void for_node_and_ghosts(const Layout& L, int x, int y, F&& fn) {
    fn(x, y);
    if (!L.ghosts) return;
    const bool gxr = x < kGhostX, gxl = x >= L.nx - kGhostX;
    const bool gyb = y < L.yo, gyt = y >= L.ny - L.yo;
    if (!(gxr || gxl || gyb || gyt)) return;
    int xs[3], ys[3];
    int nxs = 0, nys = 0;
    xs[nxs++] = x;
    if (gxr) xs[nxs++] = x + L.nx;
    if (gxl) xs[nxs++] = x - L.nx;
    ys[nys++] = y;
    if (gyb) ys[nys++] = y + L.ny;
    if (gyt) ys[nys++] = y - L.ny;
    for (int a = 0; a < nys; ++a)
        for (int b = 0; b < nxs; ++b)
            if (a || b) fn(xs[b], ys[a]);
}

}  // namespace llb
