// Kernel instances: field c64, n = 7 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(7, false, c64)
