// Local factorisation kernels for DG order p = 4.
#define VEF_FACTOR_P 4
#define VEF_FACTOR_FN factor_records_p4
#include "factor_impl.cuh"
