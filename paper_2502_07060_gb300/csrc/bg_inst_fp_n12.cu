// Kernel instances: field fp, n = 12 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(12, true, fp)
