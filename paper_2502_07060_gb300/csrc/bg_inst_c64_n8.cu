// Kernel instances: field c64, n = 8 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(8, false, c64)
