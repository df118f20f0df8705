// The mixed-precision paths of mixed_impl.cuh for the TF32x3 operand precision.
#define DMET_ONE_PREC DMET_PREC_TF32X3
#define DMET_PREC_TYPE tc::PrecTF32x3
#define DMET_PREC_SUFFIX _tf32x3
#define DMET_PRIMARY_TU 0
#include "mixed_impl.cuh"
