// Kernel instantiations: slab pass, FP32, x length 256, one kernel per launch type.
#include "launch_defs.cuh"

SGSPM_INST_XZ_MODES(256)
