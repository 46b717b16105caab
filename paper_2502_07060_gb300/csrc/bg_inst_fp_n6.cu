// Kernel instances: field fp, n = 6 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(6, true, fp)
