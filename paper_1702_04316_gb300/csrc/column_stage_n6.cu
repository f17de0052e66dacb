// The fused 1D-IMEX stage at polynomial order N = 6 (column_stage.cuh); one order per
// translation unit, so that the build compiles the orders in parallel.
#include "column_stage.cuh"

NUMA_STAGE_ORDER_DEFINE(6)
