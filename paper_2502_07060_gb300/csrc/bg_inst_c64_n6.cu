// Kernel instances: field c64, n = 6 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(6, false, c64)
