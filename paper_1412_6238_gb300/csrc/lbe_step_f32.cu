// Step and field-export kernels with StF32 population storage.
#define LBE_ST ::lbe::StF32
#define LBE_SUFFIX f32
#define LBE_ALL_TILES 1
#define LBE_STASH 1  // the stash strip kernel
#define LBE_PCORR 1  // the pre-pass of the dissipation term (tile kernel)
#include "lbe_step_inst.cuh"
