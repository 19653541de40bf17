// Mixed-precision sigma and refinement solver (bf16 tcgen05 contractions inside fp64 refinement).
#include "internal.h"

namespace esmp2 {

esmp2_status sigma_mixed(esmp2_handle *h, const double *, double *) {
  h->err = "mixed precision path not built yet";
  return ESMP2_ERR_UNSUPPORTED;
}

esmp2_status profile_mixed(esmp2_handle *h, const double *, double *, int, double *) {
  h->err = "mixed precision path not built yet";
  return ESMP2_ERR_UNSUPPORTED;
}

esmp2_status solve_mixed(esmp2_handle *h, double, int, esmp2_solve_info *) {
  h->err = "mixed precision path not built yet";
  return ESMP2_ERR_UNSUPPORTED;
}

}  // namespace esmp2
