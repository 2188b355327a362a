// Local factorisation kernels for DG order p = 3.
#define VEF_FACTOR_P 3
#define VEF_FACTOR_FN factor_records_p3
#include "factor_impl.cuh"
