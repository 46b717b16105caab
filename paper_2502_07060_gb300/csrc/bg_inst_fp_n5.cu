// Kernel instances: field fp, n = 5 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(5, true, fp)
