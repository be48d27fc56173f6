// Step and field-export kernels with StF64 population storage.
#define LBE_ST ::lbe::StF64
#define LBE_SUFFIX f64
#define LBE_ALL_TILES 0
#define LBE_STRIP 0
#define LBE_PCORR 1
#include "lbe_step_inst.cuh"
