// Compact kernel instances: field fp, D = 6, D_s = 6 (both metrics).
#include "bg_instances.cuh"
BG_DEFINE_COMPACT(6, 6, FpOps, fp)
