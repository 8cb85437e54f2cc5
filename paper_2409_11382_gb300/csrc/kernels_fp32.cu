// FP32 instantiation of the kernels: moment storage, FP32 collisions (levels
// whose next coarser level is also FP32, and the per-cell field kernels).
#include "instantiate.h"

BIOT_SWEEP_MOM(float, float)
BIOT_FIELDS(float)
