// FP64 policy kernels.
#define PINS_POLICY PolF64
#define PINS_PASSES_FN passes_f64
#include "pins_kernels_impl.cuh"
