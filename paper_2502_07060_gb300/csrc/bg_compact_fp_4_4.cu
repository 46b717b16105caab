// Compact kernel instances: field fp, D = 4, D_s = 4 (both metrics).
#include "bg_instances.cuh"
BG_DEFINE_COMPACT(4, 4, FpOps, fp)
