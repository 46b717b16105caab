// Kernel instances: field fp, n = 8 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(8, true, fp)
