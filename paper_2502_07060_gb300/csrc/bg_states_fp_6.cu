// All-assignment (states) kernel instances: field fp, D = 6, every D_s >= D (both metrics).
#include "bg_states.cuh"
BG_DEFINE_STATES(6, FpOps, fp)
