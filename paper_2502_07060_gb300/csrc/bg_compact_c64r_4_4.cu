// Compact kernel instances: field c64 with real momenta, D = 4, D_s = 4 (both metrics).
#include "bg_instances.cuh"
BG_DEFINE_COMPACT(4, 4, C64ROps, c64r)
