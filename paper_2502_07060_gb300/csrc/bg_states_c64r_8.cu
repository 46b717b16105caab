// All-assignment (states) kernel instances: field c64r, D = 8, every D_s >= D (both metrics).
#include "bg_states.cuh"
BG_DEFINE_STATES(8, C64ROps, c64r)
