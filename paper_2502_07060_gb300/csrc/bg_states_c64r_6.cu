// All-assignment (states) kernel instances: field c64r, D = 6, every D_s >= D (both metrics).
#include "bg_states.cuh"
BG_DEFINE_STATES(6, C64ROps, c64r)
