// Kernel instantiations: slab pass, FP32, x length 512; TF32X3 form at x length 128.
#include "launch_defs.cuh"

SGSPM_INST_XZ(float, 512, false, false)
SGSPM_INST_XZ(float, 128, true, false)
