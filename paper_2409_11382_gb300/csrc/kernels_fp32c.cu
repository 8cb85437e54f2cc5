// FP32 level above an FP64 level (the coarsest level of the FP32 path, or every
// coarse level with BIOT_FP32_COARSE64): float -> double level pair.  A unit of
// its own so that the build compiles it in parallel with the others.
#include "instantiate.h"

BIOT_SWEEP_MOM(float, double)
