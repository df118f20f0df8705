// The mixed-precision paths of mixed_impl.cuh for the BF16x3 operand precision.
#define DMET_ONE_PREC DMET_PREC_BF16X3
#define DMET_PREC_TYPE tc::PrecBF16x3
#define DMET_PREC_SUFFIX _bf16x3
#define DMET_PRIMARY_TU 1
#include "mixed_impl.cuh"
