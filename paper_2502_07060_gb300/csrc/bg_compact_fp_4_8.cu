// Compact kernel instances: field fp, D = 4, D_s = 8 (both metrics).
#include "bg_instances.cuh"
BG_DEFINE_COMPACT(4, 8, FpOps, fp)
