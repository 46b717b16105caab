// Lane-group kernel instances (small batches): field fp, L = 4 and 8, both metrics.
#include "bg_lanes.cuh"
BG_DEFINE_LANES(FpOps, fp)
