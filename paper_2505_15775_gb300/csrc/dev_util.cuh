// Device helpers shared by the kernels: 16-byte vectors of R rows, row-group
// (sub-warp) reductions, block reductions and the last-block pattern.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "alm_internal.h"

namespace alm {

template <typename T>
struct VecT;
template <>
struct VecT<float> {
    using type = float4;
    static constexpr int W = 4;
};
template <>
struct VecT<double> {
    using type = double2;
    static constexpr int W = 2;
};

__device__ __forceinline__ float4 vzero(float) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ double2 vzero(double) { return make_double2(0.0, 0.0); }

// read-only 16-byte load (the data is not written by the running kernel)
__device__ __forceinline__ float4 ldro(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ double2 ldro(const double *p) { return __ldg(reinterpret_cast<const double2 *>(p)); }
// plain 16-byte load/store
__device__ __forceinline__ float4 ld(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ double2 ld(const double *p) { return *reinterpret_cast<const double2 *>(p); }
__device__ __forceinline__ void stv(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ void stv(double *p, double2 v) { *reinterpret_cast<double2 *>(p) = v; }

__device__ __forceinline__ float dot(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
__device__ __forceinline__ double dot(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }

__device__ __forceinline__ float4 fma4(float s, float4 a, float4 c) {
    return make_float4(fmaf(s, a.x, c.x), fmaf(s, a.y, c.y), fmaf(s, a.z, c.z), fmaf(s, a.w, c.w));
}
__device__ __forceinline__ double2 fma4(double s, double2 a, double2 c) {
    return make_double2(fma(s, a.x, c.x), fma(s, a.y, c.y));
}
__device__ __forceinline__ float4 scale4(float s, float4 a) { return make_float4(s * a.x, s * a.y, s * a.z, s * a.w); }
__device__ __forceinline__ double2 scale4(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

__device__ __forceinline__ float comp(float4 v, int k) { return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w; }
__device__ __forceinline__ double comp(double2 v, int k) { return k == 0 ? v.x : v.y; }

// zero the components of a lane's vector that lie at columns >= r
__device__ __forceinline__ float4 mask_tail(float4 v, int c0, int r) {
    if (c0 + 4 <= r) return v;
    if (c0 >= r) return make_float4(0.f, 0.f, 0.f, 0.f);
    return make_float4(v.x, c0 + 1 < r ? v.y : 0.f, c0 + 2 < r ? v.z : 0.f, 0.f);
}
__device__ __forceinline__ double2 mask_tail(double2 v, int c0, int r) {
    if (c0 + 2 <= r) return v;
    if (c0 >= r) return make_double2(0.0, 0.0);
    return make_double2(v.x, 0.0);
}

// Compensated ("float-float") sum of squares of a lane's vector, reduced over the row
// group: returns hi + lo in double with the rounding errors of every product (exact,
// via FMA) and every addition (Knuth's two-sum) kept in lo.  Used for the diagonal
// constraint values X_ii = |r_i|^2, whose residual X_ii - b_i must be resolved far below
// the FP32 rounding of |r_i|^2 ~ 1 for the ALM dual update.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}
template <int LANES>
__device__ __forceinline__ double ff_norm2(float4 v, unsigned mask) {
    float hi = 0.f, lo = 0.f;
    const float c[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float p = c[k] * c[k];
        lo += fmaf(c[k], c[k], -p);
        two_sum_acc(hi, lo, p);
    }
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(mask, hi, o);
        const float l2 = __shfl_xor_sync(mask, lo, o);
        two_sum_acc(hi, lo, h2);
        lo += l2;
    }
    return double(hi) + double(lo);
}
template <int LANES>
__device__ __forceinline__ double ff_norm2(double2 v, unsigned mask) {
    double x = v.x * v.x + v.y * v.y;
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
    return x;
}

// lane mask of the LANES-wide row group that contains `lane`
template <int LANES>
__device__ __forceinline__ unsigned group_mask(int lane) {
    if (LANES == 32) return 0xffffffffu;
    return ((1u << LANES) - 1u) << (lane & ~(LANES - 1));
}

template <int LANES, typename T>
__device__ __forceinline__ T group_sum(T x, unsigned mask) {
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
    return x;
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Sum of `v` over the block; the result is valid in thread 0.  `sh` holds 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = (l < int(blockDim.x >> 5)) ? sh[l] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

// After every block has written its partials: returns true in exactly one block
// (the last to arrive), which may then read all partials.  The counter is reset
// by that block.
__device__ __forceinline__ bool last_block(unsigned int *counter) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x - 1);
        if (is_last) *counter = 0u;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// In the last block: deterministic sum over blocks of partial slot `k`.
__device__ __forceinline__ double sum_partials(const double *partials, int k, double *sh) {
    double t = 0.0;
    for (int b = threadIdx.x; b < int(gridDim.x); b += blockDim.x) t += __ldcg(partials + size_t(b) * kPartStride + k);
    return block_sum(t, sh);
}

}  // namespace alm
