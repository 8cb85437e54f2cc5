// FP64 instantiation of the kernels (the FP64 path, and the coarsest level of
// the FP32 path).  Compiled with --fmad=false so that no fused multiply-add
// changes the rounding.
#include "instantiate.h"

BIOT_SWEEP_MOM(double, double)
BIOT_FIELDS(double)
