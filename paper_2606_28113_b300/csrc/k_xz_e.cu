// Kernel instantiations: slab pass, TF32X3 form at x lengths 256 and 512.
#include "launch_defs.cuh"

SGSPM_INST_XZ(float, 256, true, false)
SGSPM_INST_XZ(float, 512, true, false)
