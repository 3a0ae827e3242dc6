// Transform kernels for D in [1, 4].
#include "inst_template.cuh"
ASH_DEFINE_RANGE(0)
