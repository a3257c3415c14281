// Kernel instantiations: slab pass, FP32, runtime and short x lengths.
#include "launch_defs.cuh"

SGSPM_INST_XZ(float, 0, false, false)
SGSPM_INST_XZ(float, 8, false, false)
SGSPM_INST_XZ(float, 16, false, false)
SGSPM_INST_XZ(float, 32, false, false)
