// Kernel instantiations: slab pass, FP32, x length 256 and the runtime length with several rows per CTA.
#include "launch_defs.cuh"

SGSPM_INST_XZ(float, 256, false, false)
SGSPM_INST_XZ(float, 256, false, true)
SGSPM_INST_XZ(float, 0, false, true)
