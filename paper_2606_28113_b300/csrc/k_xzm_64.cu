// Kernel instantiations: slab pass, FP32, x length 64, one kernel per launch type.
#include "launch_defs.cuh"

SGSPM_INST_XZ_MODES(64)
