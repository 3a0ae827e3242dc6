// Transform kernels for D in [5, 8].
#include "inst_template.cuh"
ASH_DEFINE_RANGE(1)
