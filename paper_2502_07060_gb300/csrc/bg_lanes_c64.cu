// Lane-group kernel instances (small batches): field c64, L = 4 and 8, both metrics.
#include "bg_lanes.cuh"
BG_DEFINE_LANES(C64Ops, c64)
