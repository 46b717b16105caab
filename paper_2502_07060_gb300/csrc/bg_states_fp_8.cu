// All-assignment (states) kernel instances: field fp, D = 8, every D_s >= D (both metrics).
#include "bg_states.cuh"
BG_DEFINE_STATES(8, FpOps, fp)
