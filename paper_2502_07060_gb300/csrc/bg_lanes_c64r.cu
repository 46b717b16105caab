// Lane-group kernel instances (small batches): field c64r, L = 4 and 8, both metrics.
#include "bg_lanes.cuh"
BG_DEFINE_LANES(C64ROps, c64r)
