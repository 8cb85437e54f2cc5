// FP32 instantiation of the kernels: moment storage, FP32 collisions; the
// coarsest multigrid level stays FP64 (float -> double level pair).
#include "instantiate.h"

BIOT_SWEEP_MOM(float, float)
BIOT_SWEEP_MOM(float, double)
BIOT_FIELDS(float)
