// All-assignment (states) kernel instances: field c64r, D = 4, every D_s >= D (both metrics).
#include "bg_states.cuh"
BG_DEFINE_STATES(4, C64ROps, c64r)
