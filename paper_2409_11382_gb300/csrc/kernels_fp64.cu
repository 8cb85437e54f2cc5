// FP64 instantiation of the kernels (parity path).  Compiled with
// --fmad=false so that no fused multiply-add changes the rounding.
#include "biot_kernels.cuh"

BIOT_INSTANTIATE_LEVEL(double, double)
BIOT_INSTANTIATE_FIELD(double)
