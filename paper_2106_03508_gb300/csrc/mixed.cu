// Split-precision moment build (BF16x3 on tcgen05): not yet built.
#include "../../include/agf2.h"
#include "agf2_internal.h"

namespace agf2 {
int mixed_build_moments(const double*, int, int, const double*, int, const double*, int,
                        const double*, const double*, int, double*, double*, void*,
                        std::string& err, cudaStream_t) {
  err = "AGF2_BF16X3 moment build not available in this build";
  return AGF2_ERR_UNSUPPORTED;
}
}  // namespace agf2
