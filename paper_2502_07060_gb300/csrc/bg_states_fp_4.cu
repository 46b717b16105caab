// All-assignment (states) kernel instances: field fp, D = 4, every D_s >= D (both metrics).
#include "bg_states.cuh"
BG_DEFINE_STATES(4, FpOps, fp)
