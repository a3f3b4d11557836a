// Memory layout of moment fields on the device.
//
// A moment buffer is field-major: field f starts at f * fs elements.  Inside
// a field, node (x, y, z) sits at ((z * py) + (y + yo)) * px + (x + xo).
//
// Dense layout (xo = yo = 0, px = nx, py = ny): used for temporaries of the
// population-storing schemes.
//
// Padded layout (moment-only state): xo = 4, yo = 1, px = nx + 8 rounded up
// to a multiple of 8, py = ny + 2.  The extra columns and rows hold periodic
// ghost copies -- column x = -1 holds x = nx-1, column x = nx holds x = 0,
// row y = -1 holds y = ny-1, row y = ny holds y = 0 (corners likewise) --
// written by every kernel that writes the state.  With them, the tile plus
// halo that a CTA needs is one rectangular box whose x start is 16-byte
// aligned, so one TMA load fetches it without wrapping; the three columns
// x = -4..-2 and x > nx are padding that is never read as data.
#pragma once

#include <cstddef>

namespace llb {

struct Layout {
    int nx, ny, nz;
    int px, py;   // row pitch (elements) and rows per plane
    int xo, yo;   // offset of node (0, 0) inside a plane
    size_t fs;    // field stride in elements
    int ghosts;   // 1: periodic ghost copies are maintained

    __host__ __device__ __forceinline__ size_t at(int x, int y, int z) const {
        return ((size_t)z * py + (y + yo)) * (size_t)px + (x + xo);
    }
};

inline Layout make_layout(int nx, int ny, int nz, bool padded) {
    Layout L;
    L.nx = nx; L.ny = ny; L.nz = nz;
    if (padded) {
        L.xo = 4; L.yo = 1;
        L.px = ((nx + 8 + 7) / 8) * 8;
        L.py = ny + 2;
        L.ghosts = 1;
    } else {
        L.xo = 0; L.yo = 0;
        L.px = nx; L.py = ny;
        L.ghosts = 0;
    }
    L.fs = (size_t)L.px * L.py * nz;
    return L;
}

// Call fn(x', y') for (x, y) and, in a padded layout, for every ghost
// position that mirrors (x, y) under the periodic wrap.
template <class F>
__device__ __forceinline__ void for_node_and_ghosts(const Layout& L, int x, int y, F&& fn) {
    fn(x, y);
    if (!L.ghosts) return;
    const bool gx0 = (x == 0), gx1 = (x == L.nx - 1);
    const bool gy0 = (y == 0), gy1 = (y == L.ny - 1);
    if (!(gx0 || gx1 || gy0 || gy1)) return;
    int xs[3], ys[3];
    int nxs = 0, nys = 0;
    xs[nxs++] = x;
    if (gx0) xs[nxs++] = L.nx;
    if (gx1) xs[nxs++] = -1;
    ys[nys++] = y;
    if (gy0) ys[nys++] = L.ny;
    if (gy1) ys[nys++] = -1;
    for (int a = 0; a < nys; ++a)
        for (int b = 0; b < nxs; ++b)
            if (a || b) fn(xs[b], ys[a]);
}

}  // namespace llb
