// tc.cu -- mixed-precision H_eff products (BF16x3 split, FP32 accumulate).
#include "engine.h"

namespace gbd {

void tc_prepare(Ctx& C) {
    (void)C;
    throw Error(GBD_ERR_ARG, "mixed-precision products are not available in this build");
}

void tc_apply(Ctx& C) {
    (void)C;
    throw Error(GBD_ERR_ARG, "mixed-precision products are not available in this build");
}

}  // namespace gbd
