// seed_util.cuh -- helpers of the k-means++ distance kernels (single problem and batched): rows of
// d floats handled by groups of lanes narrower than a warp when d is small.
#pragma once

#include "internal.cuh"

namespace gbkm {

// double-float sum (error-free TwoSum at every butterfly step, as warp_sum_df) within every aligned
// group of `width` lanes (a power of two <= 32; every lane of the warp calls it): each group gets
// the sum of its own lanes
__device__ __forceinline__ double group_sum_df(DF a, int width) {
    for (int o = width >> 1; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, a.hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, a.lo, o);
        float s, e;
        two_sum(a.hi, h2, s, e);
        a.hi = s;
        a.lo = __fadd_rn(__fadd_rn(a.lo, l2), e);
    }
    return a.value();
}

// lanes per row for a row of d floats read as float4 (vw = 4) or singly: the smallest power of two
// covering the row's vectors, at most 32
__host__ __device__ __forceinline__ int lanes_per_row(int64_t d, int vw) {
    const int64_t nv = vw == 4 ? d / 4 : d;
    int l = 1;
    while (l < 32 && l < nv) l <<= 1;
    return l;
}

// lanes per row of the D^2 update (rows read as float4 when vw == 4): a power of two giving each lane
// about four vectors of its row, at most 32 lanes, so that a warp has several rows' loads in flight
__host__ __device__ __forceinline__ int lanes_per_row_d2(int64_t d, int vw) {
    const int64_t nv = vw == 4 ? d / 4 : d;
    int l = 1;
    while (l < 32 && 4 * l < nv) l <<= 1;
    return l;
}

}  // namespace gbkm
