// Host check of the state layouts (compiled and run by tests/test_layout_host.py):
// the field map is a bijection from (node index < fs, field) onto the buffer's
// NF * fs elements for both field orders, field strides are multiples of 32, and
// the interleaved state's rows are whole 32-node blocks.
#include <cstdio>
#include <vector>

#include "layout.cuh"

using namespace llb;

template <class S, int NF>
static int check(const Layout& L, const char* what) {
    std::vector<unsigned char> seen((size_t)NF * L.fs, 0);
    for (size_t i = 0; i < L.fs; ++i)
        for (int f = 0; f < NF; ++f) {
            const size_t o = FieldMap<S, NF>::at(i, f, L.fs);
            if (o >= seen.size() || seen[o]) {
                std::printf("FAIL %s: node %zu field %d -> %zu\n", what, i, f, o);
                return 1;
            }
            seen[o] = 1;
        }
    return 0;
}

int main() {
    int bad = 0;
    const int dims[][3] = {{1, 1, 1}, {2, 3, 1}, {4, 4, 4}, {9, 6, 5}, {37, 11, 7}, {70, 10, 3}};
    for (auto& d : dims) {
        for (int padded = 0; padded < 2; ++padded) {
            const Layout a = make_layout(d[0], d[1], d[2], padded, 1, 32);  // one-component FP32
            const Layout b = make_layout(d[0], d[1], d[2], padded, 2, 8);   // two components
            if (a.fs % 32 || b.fs % 32) { std::printf("FAIL fs not a multiple of 32\n"); ++bad; }
            if (padded && a.px % 32) { std::printf("FAIL interleaved row pitch %d\n", a.px); ++bad; }
            if (a.fs < (size_t)a.px * a.py * a.nz) { std::printf("FAIL fs below the node count\n"); ++bad; }
            bad += check<float, 10>(a, "interleaved");
            bad += check<double, 10>(a, "field-major FP64");
            bad += check<float, 11>(b, "field-major two components");
            // the node index of the last node lies below fs
            if (a.at(d[0] - 1, d[1] - 1, d[2] - 1) >= a.fs) { std::printf("FAIL last node\n"); ++bad; }
        }
    }
    static_assert(FieldMap<float, 10>::kInterleaved && !FieldMap<double, 10>::kInterleaved &&
                      !FieldMap<float, 11>::kInterleaved, "field orders");
    std::printf(bad ? "layout check failed\n" : "layout check ok\n");
    return bad ? 1 : 0;
}
