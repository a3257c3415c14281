// Kernel instantiations: line passes, FP64 form.
#include "launch_defs.cuh"

SGSPM_INST_YH(double, 0)
SGSPM_INST_YS(double)
SGSPM_INST_YW(double, 1, 2)
SGSPM_INST_YW(double, 1, 4)
SGSPM_INST_YW(double, 1, 8)
SGSPM_INST_YW(double, 1, 16)
SGSPM_INST_YW(double, 2, 2)
SGSPM_INST_YW(double, 2, 4)
SGSPM_INST_YW(double, 2, 8)
SGSPM_INST_YW(double, 2, 16)
SGSPM_INST_YW(double, 3, 2)
SGSPM_INST_YW(double, 3, 4)
SGSPM_INST_YW(double, 3, 8)
SGSPM_INST_YW(double, 3, 16)
