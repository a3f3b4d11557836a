// Tiled moment-only kernel instances for __nv_bfloat16 storage (float arithmetic).
#include "moment_tiled.cuh"

LLB_TILED_ENTRY(bf16, float, __nv_bfloat16, 1)
