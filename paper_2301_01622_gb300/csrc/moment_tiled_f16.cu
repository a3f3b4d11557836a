// Tiled moment-only kernel instances for __half storage (float arithmetic).
#include "moment_tiled.cuh"

LLB_TILED_ENTRY(f16, float, __half, 1)
