// Dispatch of the local factorisation to the per-order translation units.
#include "common.h"

namespace vef {

vef_status factor_records_p1(Mesh*, Schedule*, const double*, int, bool, int, const FactorRhs*, cudaStream_t);
vef_status factor_records_p2(Mesh*, Schedule*, const double*, int, bool, int, const FactorRhs*, cudaStream_t);
vef_status factor_records_p3(Mesh*, Schedule*, const double*, int, bool, int, const FactorRhs*, cudaStream_t);
vef_status factor_records_p4(Mesh*, Schedule*, const double*, int, bool, int, const FactorRhs*, cudaStream_t);

vef_status factor_records(Mesh* mesh, Schedule* S, const double* sigma_t, int precision,
                          bool store_systems, int force_pivot, const FactorRhs* rhs,
                          cudaStream_t stream) {
  switch (mesh->p) {
    case 1: return factor_records_p1(mesh, S, sigma_t, precision, store_systems, force_pivot, rhs, stream);
    case 2: return factor_records_p2(mesh, S, sigma_t, precision, store_systems, force_pivot, rhs, stream);
    case 3: return factor_records_p3(mesh, S, sigma_t, precision, store_systems, force_pivot, rhs, stream);
    default: return factor_records_p4(mesh, S, sigma_t, precision, store_systems, force_pivot, rhs, stream);
  }
}

}  // namespace vef
