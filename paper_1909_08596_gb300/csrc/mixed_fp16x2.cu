// The mixed-precision paths of mixed_impl.cuh for the FP16x2 operand precision.
#define DMET_ONE_PREC DMET_PREC_FP16X2
#define DMET_PREC_TYPE tc::PrecFP16x2
#define DMET_PREC_SUFFIX _fp16x2
#define DMET_PRIMARY_TU 0
#include "mixed_impl.cuh"
