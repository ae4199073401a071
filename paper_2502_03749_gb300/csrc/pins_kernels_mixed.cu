// Mixed (FP32-unit, double-float) policy kernels.
#define PINS_POLICY PolMixed
#define PINS_PASSES_FN passes_mixed
#include "pins_kernels_impl.cuh"
