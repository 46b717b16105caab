// Kernel instances: field c64, n = 10 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(10, false, c64)
