// Tiled moment-only kernel instances for float storage (float arithmetic).
#include "moment_tiled.cuh"

LLB_TILED_ENTRY(f32, float, float, kTiledVariants32)
