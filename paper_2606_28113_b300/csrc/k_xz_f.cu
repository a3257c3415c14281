// Kernel instantiations: slab pass, FP64 form (runtime x length).
#include "launch_defs.cuh"

SGSPM_INST_XZ(double, 0, false, false)
