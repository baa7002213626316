// split.h -- operand splitting for the tensor-core product forms: rows of
// FP64 operators (or of psi^T) become BF16 planes on the device.
// Element (r, c) of the source is src[r * rs + c * cs];
// columns from cols to ldd - 1 are zero padding; plane k of the output
// starts at dst + k * plane.  A group of G lanes handles one (row, 64-column
// block) unit (G = 32, or 8 / 16 for short rows, so a warp then covers
// several rows).  GB300's FP64 pipe is narrow, so the per-element work is
// integer and FP32 arithmetic on the FP64 bit patterns.
// Output rows can be regrouped (a layer-stacked block stored with its layers
// side by side along the row) through R, lpitch and rpitch.
//   MODE 0: x = hi + lo, hi = bf16(f), lo = bf16(f - hi) with f = fp32(x)
//     (|x - hi - lo| <= 2^-18 |x|).
//   MODE 1: error-free slicing: with 2^(e-1) <= max |x| < 2^e over the unit,
//     q = round(x 2^(32-e)) (|q| <= 2^32) is cut into balanced base-256
//     digits q = m1 2^24 + m2 2^16 + m3 2^8 + m4 (|m1| <= 256, |mk| <= 128),
//     and slice k = mk 2^(e - 8k) is exact in BF16; x = sum of the slices
//     + O(2^(e-33)).  Units whose maximum is zero or subnormal are zero.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace gbd {
namespace tc {

struct SplitDesc {
    const double* src;
    long long rs, cs;
    long long rows;
    int cols, ldd;
    __nv_bfloat16* dst;  // source row r goes to dst + (r / R) * lpitch + (r % R) * rpitch
    long long plane;
    long long R, lpitch, rpitch;
    long long rbase;     // row index of src row 0 within the whole block (for the regrouping)
};

// One CTA per descriptor; descriptors cover at most kSplitUnits units, so the
// work spreads over the whole GPU however unequal the operator blocks are.
constexpr int kSplitUnits = 2048;

// Launches the split of nblocks descriptors on st: form 0 BF16x3 (hi, lo),
// form 1 sliced (four slices), form 2 both from one read of the source (d1:
// the sliced destinations of the same source units as d0).
void launch_split(int form, const SplitDesc* d0, const SplitDesc* d1, unsigned nblocks, cudaStream_t st);

}  // namespace tc
}  // namespace gbd
