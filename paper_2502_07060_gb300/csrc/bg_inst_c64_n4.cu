// Kernel instances: field c64, n = 4 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(4, false, c64)
