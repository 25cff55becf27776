// twosum.cuh -- compensated FP32 summation (Knuth's two-sum): after
// two_sum_add(s, c, x), s + c equals the exact sum of the old s + c and x up to
// the rounding of the small term c. Used where a sum of many FP32 terms must
// lose no more than its final rounding and FP64 (1/64 of the FP32 rate on
// this GPU) would be the cost.
#pragma once

namespace rubix {

__device__ __forceinline__ void two_sum_add(float& s, float& c, float x) {
    const float t = s + x;
    const float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
}

}  // namespace rubix
