// FP32 instantiation of the kernels: FP32 populations and collisions; the
// coarsest multigrid level stays FP64 (float -> double level pair).
#include "biot_kernels.cuh"

BIOT_INSTANTIATE_LEVEL(float, float)
BIOT_INSTANTIATE_LEVEL(float, double)
BIOT_INSTANTIATE_FIELD(float)
