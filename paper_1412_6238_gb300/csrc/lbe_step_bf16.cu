// Step and field-export kernels with StBF16 population storage.
#define LBE_ST ::lbe::StBF16
#define LBE_SUFFIX bf16
#define LBE_ALL_TILES 1
#include "lbe_step_inst.cuh"
