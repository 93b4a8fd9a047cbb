// Float-pair ("double-float") helpers of the FP32 form: a double split into two floats,
// compensated accumulation of a lane's 4-vector of sum_k s_k x_k, and the compensated
// squared norm of an R row over its row group.  Shared by the per-kernel path and the
// batched persistent solver.
#pragma once

#include "dev_util.cuh"

namespace alm {

__device__ __forceinline__ void split_pair(double d, float &hi, float &lo) {
    hi = float(d);
    lo = float(d - double(hi));
}
__device__ __forceinline__ void split_pair(double d, double &hi, double &lo) {
    hi = d;
    lo = 0.0;
}
// Accumulator of a lane's vector of sum_k s_k x_k: plain FMAs in the FP64 form,
// compensated (products split exactly with FMA, sums with two-sum) in the FP32 form so
// that G = 2 S R keeps its accuracy when its O(|S||R|) terms cancel.
struct AccD {
    double2 v;
    __device__ __forceinline__ void init() { v = make_double2(0.0, 0.0); }
    __device__ __forceinline__ void add(double s, double2 x) { v = fma4(s, x, v); }
    __device__ __forceinline__ void add_lo(double s, double2 x) { v = fma4(s, x, v); }
    __device__ __forceinline__ double2 value() const { return v; }
};
struct AccF {
    float hi[4], lo[4];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int k = 0; k < 4; ++k) hi[k] = lo[k] = 0.f;
    }
    __device__ __forceinline__ void add(float s, float4 x) {
        const float c[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float p = s * c[k];
            lo[k] += fmaf(s, c[k], -p);
            two_sum_acc(hi[k], lo[k], p);
        }
    }
    __device__ __forceinline__ void add_lo(float s, float4 x) {  // small correction terms
        lo[0] = fmaf(s, x.x, lo[0]);
        lo[1] = fmaf(s, x.y, lo[1]);
        lo[2] = fmaf(s, x.z, lo[2]);
        lo[3] = fmaf(s, x.w, lo[3]);
    }
    __device__ __forceinline__ float4 value() const {
        return make_float4(hi[0] + lo[0], hi[1] + lo[1], hi[2] + lo[2], hi[3] + lo[3]);
    }
};
template <typename T>
struct AccOf;
template <>
struct AccOf<float> {
    using type = AccF;
};
template <>
struct AccOf<double> {
    using type = AccD;
};

// float-pair sum of squares of a lane's vector over the row group (FP32 form); the
// FP64 form returns its plain sum in hi
__device__ __forceinline__ void norm2_pair(float4 v, unsigned mask, int lanes, float &hi, float &lo) {
    const float c[4] = {v.x, v.y, v.z, v.w};
    hi = c[0] * c[0];  // the pair starts from the first square (a two-sum into 0 is exact)
    lo = fmaf(c[0], c[0], -hi);
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        const float p = c[k] * c[k];
        lo += fmaf(c[k], c[k], -p);
        two_sum_acc(hi, lo, p);
    }
    for (int o = lanes / 2; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(mask, hi, o);
        const float l2 = __shfl_xor_sync(mask, lo, o);
        two_sum_acc(hi, lo, h2);
        lo += l2;
    }
}
__device__ __forceinline__ void norm2_pair(double2 v, unsigned mask, int lanes, double &hi, double &lo) {
    double x = v.x * v.x + v.y * v.y;
    for (int o = lanes / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
    hi = x;
    lo = 0.0;
}

}  // namespace alm
