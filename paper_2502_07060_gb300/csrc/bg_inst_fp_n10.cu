// Kernel instances: field fp, n = 10 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(10, true, fp)
