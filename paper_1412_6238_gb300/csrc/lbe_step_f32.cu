// Step and field-export kernels with StF32 population storage.
#define LBE_ST ::lbe::StF32
#define LBE_SUFFIX f32
#define LBE_ALL_TILES 1
#define LBE_STRIP 1
#define LBE_R128 7  // staged-row ring depth of the 128-column strip kernel
#define LBE_R64 9   // and of the 64-column one
#define LBE_STASH 1  // the stash strip kernel (FP32 only)
#include "lbe_step_inst.cuh"
