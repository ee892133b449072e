// A priori SGS analysis (Sec. III, Eq. 5-8, 15) -- implemented in a later change.
#include "../../include/qg.h"
#include <string>
extern "C" int qg_sgs_apriori(const double*, int32_t, int32_t, double, const double*, const double*,
                              const qg_closure*, const qg_params*, double, double, int32_t, double*, double*,
                              double*, double*) {
  return QG_ERR_UNSUPPORTED;
}
