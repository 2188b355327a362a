// Local factorisation kernels for DG order p = 2.
#define VEF_FACTOR_P 2
#define VEF_FACTOR_FN factor_records_p2
#include "factor_impl.cuh"
