// Kernel instances: field c64, n = 9 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(9, false, c64)
