// Compact kernel instances: field fp, D = 6, D_s = 8 (both metrics).
#include "bg_instances.cuh"
BG_DEFINE_COMPACT(6, 8, FpOps, fp)
