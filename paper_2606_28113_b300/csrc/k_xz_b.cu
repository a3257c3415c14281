// Kernel instantiations: slab pass, FP32, x lengths 64 and 128 (one and several rows per CTA).
#include "launch_defs.cuh"

SGSPM_INST_XZ(float, 64, false, false)
SGSPM_INST_XZ(float, 128, false, false)
SGSPM_INST_XZ(float, 64, false, true)
SGSPM_INST_XZ(float, 128, false, true)
