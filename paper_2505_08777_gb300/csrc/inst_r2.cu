// Transform kernels for D in [9, 12].
#include "inst_template.cuh"
ASH_DEFINE_RANGE(2)
