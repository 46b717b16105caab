// Compact kernel instances: field c64 with real momenta, D = 4, D_s = 8 (both metrics).
#include "bg_instances.cuh"
BG_DEFINE_COMPACT(4, 8, C64ROps, c64r)
