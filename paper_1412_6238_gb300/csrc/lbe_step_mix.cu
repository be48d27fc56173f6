// Step and field-export kernels with StMix population storage (FP32 f, FP16
// g and hbar deviations).
#define LBE_ST ::lbe::StMix
#define LBE_SUFFIX mix
#define LBE_ALL_TILES 1
#define LBE_STASH 1  // the stash strip kernel
#include "lbe_step_inst.cuh"
