// Segments of FP32 levels (sweep_segment.cuh): their programs mix float/float
// and float/double levels, so the kernel holds both tile sweeps.  Compiled with
// the flags of the other FP32 units.
#include "instantiate.h"

BIOT_SEGMENT(float)
