// Kernel instances: field fp, n = 7 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(7, true, fp)
