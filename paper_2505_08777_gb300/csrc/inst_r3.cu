// Transform kernels for D in [13, 16].
#include "inst_template.cuh"
ASH_DEFINE_RANGE(3)
