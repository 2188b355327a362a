// Local factorisation kernels for DG order p = 1.
#define VEF_FACTOR_P 1
#define VEF_FACTOR_FN factor_records_p1
#include "factor_impl.cuh"
