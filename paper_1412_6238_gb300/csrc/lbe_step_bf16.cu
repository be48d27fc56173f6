// Step and field-export kernels with StBF16 population storage.
#define LBE_ST ::lbe::StBF16
#define LBE_SUFFIX bf16
#define LBE_ALL_TILES 1
#define LBE_STRIP 1
#define LBE_R128 7  // staged-row ring depth of the 128-column strip kernel
#define LBE_R64 11   // and of the 64-column one
#define LBE_STASH 1  // the stash strip kernel
#include "lbe_step_inst.cuh"
