// Kernel instances: field c64, n = 12 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(12, false, c64)
