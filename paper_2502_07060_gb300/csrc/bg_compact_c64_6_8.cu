// Compact kernel instances: field c64, D = 6, D_s = 8 (both metrics).
#include "bg_instances.cuh"
BG_DEFINE_COMPACT(6, 8, C64Ops, c64)
