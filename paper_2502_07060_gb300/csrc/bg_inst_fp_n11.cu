// Kernel instances: field fp, n = 11 gluons (all compiled dimensions and metrics).
#include "bg_instances.cuh"
BG_DEFINE_REGISTRY(11, true, fp)
