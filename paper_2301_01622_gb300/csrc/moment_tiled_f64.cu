// Tiled moment-only kernel instances for double storage (double arithmetic).
#include "moment_tiled.cuh"

LLB_TILED_ENTRY(f64, double, double, 1)
