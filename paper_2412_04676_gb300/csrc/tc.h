// tc.h -- mixed-precision (BF16x3 split, FP32 accumulate) H_eff products on
// the fifth-generation tensor cores (tcgen05 + TMEM, TMA-fed operands).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "core.h"

namespace gbd {

struct Heff;
struct Ctx;

struct TcHeff {
    bool built = false;
};

}  // namespace gbd
