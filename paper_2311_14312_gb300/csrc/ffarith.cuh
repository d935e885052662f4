// Compensated (float-float) arithmetic shared by the FP32 kernels that must
// keep more than FP32 accuracy: values held as hi + lo pairs of floats.
#pragma once

#include <cuda_runtime.h>

namespace dc {

// hi + lo += a * b for float-float a, b: the leading product is split
// exactly by an FMA (TwoProduct) and added by TwoSum; the rounding errors and
// the cross terms go to lo (the compensated dot product of Ogita, Rump and
// Oishi, 2005).
__device__ __forceinline__ void dot2ff(float &hi, float &lo, float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    const float pe = fmaf(a.x, b.x, -p);
    const float sum = __fadd_rn(hi, p);
    const float bb = __fsub_rn(sum, hi);
    const float se = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bb)), __fsub_rn(p, bb));
    hi = sum;
    lo += se + pe + fmaf(a.x, b.y, a.y * b.x);
}

}  // namespace dc
