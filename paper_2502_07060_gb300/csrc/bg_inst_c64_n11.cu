// Kernel instances: field c64, n = 11 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(11, false, c64)
