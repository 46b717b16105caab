// Compact kernel instances: field c64, D = 4, D_s = 6 (both metrics).
#include "bg_instances.cuh"
BG_DEFINE_COMPACT(4, 6, C64Ops, c64)
