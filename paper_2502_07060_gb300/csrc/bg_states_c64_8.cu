// All-assignment (states) kernel instances: field c64, D = 8, every D_s >= D (both metrics).
#include "bg_states.cuh"
BG_DEFINE_STATES(8, C64Ops, c64)
