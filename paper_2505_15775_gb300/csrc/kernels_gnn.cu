// Warm-start network: forward, loss and backward kernels (inference and training).
//
// The network predicts (R0, y0) for a unit-diagonal SDP from C alone (motivation: the
// local convergence of ALM-BM in Sec. 4.2 needs a starting factor near a solution and a
// multiplier near y*).  Three message-passing layers of width 64 on the pattern of C,
//     agg_i = (sum_j a_ij h_j) / max(deg_i, 1),   h'_i = relu(Ws h_i + Wn agg_i + b),
// a_ij = C_ij / mean|C_ij|, then the heads rhat_i = W_R h_i (32 columns) and
// yhat_i = w_y . h_i + b_y.  Activations are stored in BF16 (or FP32) and every product
// accumulates in FP32; gradients are FP32.  The 64-wide layers move ~0.5 KB per row and
// do ~16 KFLOP per row: they stay on the CUDA cores (below the tensor-core ridge once
// the neighbour gathers are counted), one warp per row with the weights in shared memory.
//
// Rows are the global rows of a batch (alm_batch); row g belongs to instance
// row_inst[g], whose first row is row_off[row_inst[g]] and whose pattern uses local
// column indices.
#include <cuda_bf16.h>

#include <cmath>

#include "dev_util.cuh"
#include "gnn_internal.h"

namespace alm {
namespace {

__device__ __forceinline__ float tof(float x) { return x; }
__device__ __forceinline__ float tof(__nv_bfloat16 x) { return __bfloat162float(x); }
template <typename T>
__device__ __forceinline__ T fromf(float x);
template <>
__device__ __forceinline__ float fromf<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 fromf<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

__device__ __forceinline__ float warp_sumf(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// SplitMix64 counter generator mapped to [-1, 1) (the same definition as the Lanczos
// start vector)
__device__ __forceinline__ float smx_pm1(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return float(2.0 * (double(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0);
}

// x_i = [1, deg_i/dbar, s_i/sbar, log(n)/8, u_1..u_4]
template <typename T>
__global__ void k_gnn_features(GnnGraph g, uint64_t feat_seed, T *__restrict__ H0) {
    for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < g.rows; r += int64_t(gridDim.x) * blockDim.x) {
        const int b = g.row_inst[r];
        const float4 sc = g.scal[b];
        const int e0 = g.rowptr[r], e1 = g.rowptr[r + 1];
        float s = 0.f;
        for (int e = e0; e < e1; ++e) s += g.val[e];
        const uint64_t li = uint64_t(r - g.row_off[b]);
        T *h = H0 + r * kGnnFeat;
        h[0] = fromf<T>(1.f);
        h[1] = fromf<T>(float(e1 - e0) * sc.x);
        h[2] = fromf<T>(s * sc.z);
        h[3] = fromf<T>(sc.w);
        for (int k = 0; k < 4; ++k) h[4 + k] = fromf<T>(smx_pm1(feat_seed + uint64_t(k), li));
    }
}

// One layer, one warp per row: agg (stored for the backward), h' = relu(Ws h + Wn agg + b).
// Lane l owns inputs l and l + 32 (DIN = 64) or input l (DIN = 8, l < 8), outputs l, l + 32.
template <typename T, int DIN>
__global__ void __launch_bounds__(256) k_gnn_layer_fwd(GnnGraph g, const float *__restrict__ Ws,
                                                       const float *__restrict__ Wn, const float *__restrict__ bias,
                                                       const T *__restrict__ H, T *__restrict__ AGG,
                                                       T *__restrict__ Hout) {
    __shared__ float ws[kGnnHid * (DIN + 1)], wn[kGnnHid * (DIN + 1)], bs[kGnnHid];
    __shared__ float hv[8][DIN], av[8][DIN];
    for (int t = threadIdx.x; t < kGnnHid * DIN; t += blockDim.x) {
        const int o = t / DIN, k = t % DIN;
        ws[o * (DIN + 1) + k] = Ws[t];
        wn[o * (DIN + 1) + k] = Wn[t];
    }
    for (int t = threadIdx.x; t < kGnnHid; t += blockDim.x) bs[t] = bias[t];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t r = int64_t(blockIdx.x) * (blockDim.x >> 5) + wid; r < g.rows; r += nwarps) {
        const int b = g.row_inst[r];
        const int64_t base = g.row_off[b];
        const float icb = g.scal[b].y;
        const int e0 = g.rowptr[r], e1 = g.rowptr[r + 1];
        float a0 = 0.f, a1 = 0.f;
        for (int e = e0; e < e1; ++e) {
            const float a = g.val[e] * icb;
            const T *hj = H + (base + g.col[e]) * DIN;
            if (DIN == 64) {
                a0 = fmaf(a, tof(hj[lane]), a0);
                a1 = fmaf(a, tof(hj[lane + 32]), a1);
            } else if (lane < DIN) {
                a0 = fmaf(a, tof(hj[lane]), a0);
            }
        }
        const float inv = 1.f / float(max(e1 - e0, 1));
        const T *hi = H + r * DIN;
        __syncwarp();
        if (DIN == 64) {
            const T q0 = fromf<T>(a0 * inv), q1 = fromf<T>(a1 * inv);
            AGG[r * DIN + lane] = q0;
            AGG[r * DIN + lane + 32] = q1;
            hv[wid][lane] = tof(hi[lane]);
            hv[wid][lane + 32] = tof(hi[lane + 32]);
            av[wid][lane] = tof(q0);  // the backward sees the stored (rounded) value
            av[wid][lane + 32] = tof(q1);
        } else if (lane < DIN) {
            const T q0 = fromf<T>(a0 * inv);
            AGG[r * DIN + lane] = q0;
            hv[wid][lane] = tof(hi[lane]);
            av[wid][lane] = tof(q0);
        }
        __syncwarp();
        float z0 = bs[lane], z1 = bs[lane + 32];
#pragma unroll 8
        for (int k = 0; k < DIN; ++k) {
            const float h = hv[wid][k], a = av[wid][k];
            z0 = fmaf(ws[lane * (DIN + 1) + k], h, fmaf(wn[lane * (DIN + 1) + k], a, z0));
            z1 = fmaf(ws[(lane + 32) * (DIN + 1) + k], h, fmaf(wn[(lane + 32) * (DIN + 1) + k], a, z1));
        }
        Hout[r * kGnnHid + lane] = fromf<T>(fmaxf(z0, 0.f));
        Hout[r * kGnnHid + lane + 32] = fromf<T>(fmaxf(z1, 0.f));
        __syncwarp();
    }
}

// heads: rhat = W_R h (lane c -> column c), yhat = w_y . h + b_y
template <typename T>
__global__ void __launch_bounds__(256) k_gnn_heads(GnnGraph g, const float *__restrict__ WR,
                                                   const float *__restrict__ wy, const float *__restrict__ by,
                                                   const T *__restrict__ H, float *__restrict__ rhat,
                                                   float *__restrict__ yhat) {
    __shared__ float wr[kGnnRank * (kGnnHid + 1)], wys[kGnnHid];
    __shared__ float hv[8][kGnnHid];
    for (int t = threadIdx.x; t < kGnnRank * kGnnHid; t += blockDim.x) wr[(t / kGnnHid) * (kGnnHid + 1) + t % kGnnHid] = WR[t];
    for (int t = threadIdx.x; t < kGnnHid; t += blockDim.x) wys[t] = wy[t];
    __syncthreads();
    const float b0 = by[0];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t r = int64_t(blockIdx.x) * (blockDim.x >> 5) + wid; r < g.rows; r += nwarps) {
        const float h0 = tof(H[r * kGnnHid + lane]), h1 = tof(H[r * kGnnHid + lane + 32]);
        hv[wid][lane] = h0;
        hv[wid][lane + 32] = h1;
        __syncwarp();
        float acc = 0.f;
#pragma unroll 8
        for (int k = 0; k < kGnnHid; ++k) acc = fmaf(wr[lane * (kGnnHid + 1) + k], hv[wid][k], acc);
        rhat[r * kGnnRank + lane] = acc;
        const float yv = warp_sumf(fmaf(wys[lane], h0, wys[lane + 32] * h1));
        if (lane == 0) yhat[r] = yv + b0;
        __syncwarp();
    }
}

// R0 = normalise(rhat/|rhat| + mix u/|u|), u_i a seeded uniform row (SplitMix64 stream
// mix_seed, element 32 i + c): mixing keeps R0 of full rank when the network's rows span
// few directions.  A zero row becomes u/|u| (e_1 if mix = 0).  y0 = cbar * yhat.
// 8 lanes per row (float4).
__global__ void k_gnn_warm(GnnGraph g, const float *__restrict__ rhat, const float *__restrict__ yhat,
                           const double *__restrict__ cbar, float mix, uint64_t mix_seed, float *__restrict__ R0,
                           double *__restrict__ y0) {
    const int lane = threadIdx.x & 31, gl = lane & 7;
    const unsigned gm = 0xffu << (lane & ~7);
    const int64_t ng = (int64_t(gridDim.x) * blockDim.x) >> 3;
    for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 3; r < g.rows; r += ng) {
        const float4 v = *reinterpret_cast<const float4 *>(rhat + r * kGnnRank + gl * 4);
        const uint64_t li = uint64_t(r - g.row_off[g.row_inst[r]]) * kGnnRank + gl * 4;
        const float4 u = make_float4(smx_pm1(mix_seed, li), smx_pm1(mix_seed, li + 1), smx_pm1(mix_seed, li + 2),
                                     smx_pm1(mix_seed, li + 3));
        float s = v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
        float su = u.x * u.x + u.y * u.y + u.z * u.z + u.w * u.w;
        for (int o = 4; o > 0; o >>= 1) {
            s += __shfl_xor_sync(gm, s, o);
            su += __shfl_xor_sync(gm, su, o);
        }
        const float a = s > 0.f ? rsqrtf(s) : 0.f;
        const float bmix = su > 0.f ? mix * rsqrtf(su) : 0.f;
        float4 w = make_float4(a * v.x + bmix * u.x, a * v.y + bmix * u.y, a * v.z + bmix * u.z, a * v.w + bmix * u.w);
        float sw = w.x * w.x + w.y * w.y + w.z * w.z + w.w * w.w;
        for (int o = 4; o > 0; o >>= 1) sw += __shfl_xor_sync(gm, sw, o);
        float4 out;
        if (sw > 0.f) {
            const float inv = rsqrtf(sw);
            out = make_float4(w.x * inv, w.y * inv, w.z * inv, w.w * inv);
        } else {
            out = make_float4(gl == 0 ? 1.f : 0.f, 0.f, 0.f, 0.f);
        }
        *reinterpret_cast<float4 *>(R0 + r * kGnnRank + gl * 4) = out;
        if (gl == 0) y0[r] = cbar[g.row_inst[r]] * double(yhat[r]);
    }
}

// Loss and its gradient w.r.t. the heads' outputs, one warp per row i (lane c = column c):
//   e_ii = |rhat_i|^2 - |r*_i|^2,  e_ij = rhat_i.rhat_j - r*_i.r*_j (j a pattern neighbour)
//   dL/drhat_i = (4/np) e_ii rhat_i + (2/np) sum_j e_ij rhat_j   (both (i,j) and (j,i) in the
//   full pattern, so each unordered pair reaches both rows);  loss terms e_ii^2 and, for j > i,
//   e_ij^2;  ey = yhat_i - y*_i/cbar,  dL/dyhat_i = 2 lam ey / nrow.
// Also dH3_i = W_R^T dr_i + w_y dy_i.  Per-block loss partials in part[block].
__global__ void __launch_bounds__(256) k_gnn_loss(GnnGraph g, const float *__restrict__ rhat,
                                                  const float *__restrict__ yhat, const float *__restrict__ Rs,
                                                  const double *__restrict__ ys, const double *__restrict__ cbar,
                                                  const float *__restrict__ WR, const float *__restrict__ wy,
                                                  float inv_np, float lam_nrow, float *__restrict__ dR,
                                                  float *__restrict__ dY, float *__restrict__ dH,
                                                  double *__restrict__ part) {
    __shared__ float wr[kGnnRank * (kGnnHid + 1)], wys[kGnnHid];
    __shared__ float dv[8][kGnnRank];
    __shared__ double red[8];
    for (int t = threadIdx.x; t < kGnnRank * kGnnHid; t += blockDim.x) wr[(t / kGnnHid) * (kGnnHid + 1) + t % kGnnHid] = WR[t];
    for (int t = threadIdx.x; t < kGnnHid; t += blockDim.x) wys[t] = wy[t];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
    float lsum = 0.f, lcomp = 0.f;
    for (int64_t r = int64_t(blockIdx.x) * (blockDim.x >> 5) + wid; r < g.rows; r += nwarps) {
        const int b = g.row_inst[r];
        const int64_t base = g.row_off[b];
        const int64_t li = r - base;
        const float ri = rhat[r * kGnnRank + lane], si = Rs[r * kGnnRank + lane];
        const float eii = warp_sumf(ri * ri) - warp_sumf(si * si);
        float d = 4.f * inv_np * eii * ri;
        float le = eii * eii;
        const int e1 = g.rowptr[r + 1];
        for (int e = g.rowptr[r]; e < e1; ++e) {
            const int j = g.col[e];
            const float rj = rhat[(base + j) * kGnnRank + lane], sj = Rs[(base + j) * kGnnRank + lane];
            const float eij = warp_sumf(ri * rj) - warp_sumf(si * sj);
            d = fmaf(2.f * inv_np * eij, rj, d);
            if (j > li) le += eij * eij;
        }
        dR[r * kGnnRank + lane] = d;
        const float ey = float(double(yhat[r]) - ys[r] / cbar[b]);
        const float dy = 2.f * lam_nrow * ey;
        if (lane == 0) {
            dY[r] = dy;
            const float t = le * inv_np + lam_nrow * ey * ey;
            const float s2 = lsum + t;  // two-sum
            const float bb = s2 - lsum;
            lcomp += (lsum - (s2 - bb)) + (t - bb);
            lsum = s2;
        }
        dv[wid][lane] = d;
        __syncwarp();
        float h0 = wys[lane] * dy, h1 = wys[lane + 32] * dy;
#pragma unroll 8
        for (int c = 0; c < kGnnRank; ++c) {
            const float dc = dv[wid][c];
            h0 = fmaf(wr[c * (kGnnHid + 1) + lane], dc, h0);
            h1 = fmaf(wr[c * (kGnnHid + 1) + lane + 32], dc, h1);
        }
        dH[r * kGnnHid + lane] = h0;
        dH[r * kGnnHid + lane + 32] = h1;
        __syncwarp();
    }
    if (lane == 0) red[wid] = double(lsum) + double(lcomp);
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// Layer backward, one warp per row: dz = dH (.) [h' > 0] (stored), dHprev_i = Ws^T dz,
// U_i = (Wn^T dz) / max(deg_i, 1) (the aggregation's adjoint is applied by k_gnn_agg_t).
template <typename T, int DIN>
__global__ void __launch_bounds__(256) k_gnn_layer_bwd(GnnGraph g, const float *__restrict__ Ws,
                                                       const float *__restrict__ Wn, const T *__restrict__ Hout,
                                                       const float *__restrict__ dH, float *__restrict__ dZ,
                                                       float *__restrict__ dHprev, float *__restrict__ U,
                                                       int want_prev) {
    __shared__ float ws[kGnnHid * DIN], wn[kGnnHid * DIN];
    __shared__ float zv[8][kGnnHid];
    for (int t = threadIdx.x; t < kGnnHid * DIN; t += blockDim.x) {
        ws[t] = Ws[t];
        wn[t] = Wn[t];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t r = int64_t(blockIdx.x) * (blockDim.x >> 5) + wid; r < g.rows; r += nwarps) {
        const float z0 = tof(Hout[r * kGnnHid + lane]) > 0.f ? dH[r * kGnnHid + lane] : 0.f;
        const float z1 = tof(Hout[r * kGnnHid + lane + 32]) > 0.f ? dH[r * kGnnHid + lane + 32] : 0.f;
        dZ[r * kGnnHid + lane] = z0;
        dZ[r * kGnnHid + lane + 32] = z1;
        if (!want_prev) continue;
        zv[wid][lane] = z0;
        zv[wid][lane + 32] = z1;
        __syncwarp();
        const float inv = 1.f / float(max(g.rowptr[r + 1] - g.rowptr[r], 1));
        for (int k = lane; k < DIN; k += 32) {
            float s = 0.f, u = 0.f;
#pragma unroll 8
            for (int o = 0; o < kGnnHid; ++o) {
                const float zo = zv[wid][o];
                s = fmaf(ws[o * DIN + k], zo, s);
                u = fmaf(wn[o * DIN + k], zo, u);
            }
            dHprev[r * DIN + k] = s;
            U[r * DIN + k] = u * inv;
        }
        __syncwarp();
    }
}

// dHprev_j += sum_{i in N(j)} a_ij U_i (the pattern is symmetric), one warp per row
template <int DIN>
__global__ void __launch_bounds__(256) k_gnn_agg_t(GnnGraph g, const float *__restrict__ U,
                                                   float *__restrict__ dHprev) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t nwarps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t r = int64_t(blockIdx.x) * (blockDim.x >> 5) + wid; r < g.rows; r += nwarps) {
        const int b = g.row_inst[r];
        const int64_t base = g.row_off[b];
        const float icb = g.scal[b].y;
        float s0 = 0.f, s1 = 0.f;
        const int e1 = g.rowptr[r + 1];
        for (int e = g.rowptr[r]; e < e1; ++e) {
            const float a = g.val[e] * icb;
            const float *uj = U + (base + g.col[e]) * DIN;
            if (lane < DIN) s0 = fmaf(a, uj[lane], s0);
            if (DIN == 64) s1 = fmaf(a, uj[lane + 32], s1);
        }
        if (lane < DIN) dHprev[r * DIN + lane] += s0;
        if (DIN == 64) dHprev[r * DIN + lane + 32] += s1;
    }
}

// Per-block partial of sum_rows A_r^T B_r (M x K, A FP32 rows x M, B rows x K in T) and,
// when `colsum`, of sum_rows A_r (M): tiles of 32 rows staged in shared memory; thread t
// owns outputs t, t + blockDim, ...  part[block * ldp + ...].
template <typename T, int M, int K>
__global__ void __launch_bounds__(256) k_gnn_outer(const float *__restrict__ A, const T *__restrict__ B, int64_t rows,
                                                   int colsum, float *__restrict__ part, int64_t ldp) {
    constexpr int TR = 32;
    constexpr int NOUT = M * K;
    constexpr int PER = (NOUT + 255) / 256;
    __shared__ float at[TR][M], bt[TR][K];
    float acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) acc[q] = 0.f;
    float cs = 0.f;
    for (int64_t r0 = int64_t(blockIdx.x) * TR; r0 < rows; r0 += int64_t(gridDim.x) * TR) {
        for (int t = threadIdx.x; t < TR * M; t += blockDim.x) {
            const int64_t r = r0 + t / M;
            at[t / M][t % M] = r < rows ? A[r * M + t % M] : 0.f;
        }
        for (int t = threadIdx.x; t < TR * K; t += blockDim.x) {
            const int64_t r = r0 + t / K;
            bt[t / K][t % K] = r < rows ? tof(B[r * K + t % K]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int o = threadIdx.x + q * 256;
            if (o < NOUT) {
                const int m = o / K, k = o % K;
                float s = acc[q];
#pragma unroll 8
                for (int rr = 0; rr < TR; ++rr) s = fmaf(at[rr][m], bt[rr][k], s);
                acc[q] = s;
            }
        }
        if (colsum && threadIdx.x < M)
            for (int rr = 0; rr < TR; ++rr) cs += at[rr][threadIdx.x];
        __syncthreads();
    }
    float *p = part + int64_t(blockIdx.x) * ldp;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int o = threadIdx.x + q * 256;
        if (o < NOUT) p[o] = acc[q];
    }
    if (colsum && threadIdx.x < M) p[NOUT + threadIdx.x] = cs;
}

// grad[dst + k] = sum over blocks of part[b * ldp + k], k < cnt (fixed order)
__global__ void k_gnn_reduce(const float *__restrict__ part, int nblk, int64_t ldp, int cnt, float *__restrict__ grad) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += double(part[int64_t(b) * ldp + k]);
        grad[k] = float(s);
    }
}

__global__ void k_gnn_sum_loss(const double *__restrict__ part, int nblk, double *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[b];
        *out = s;
    }
}

// Adam (Kingma and Ba, ICLR 2015) with bias correction
__global__ void k_gnn_adam(float *__restrict__ theta, const float *__restrict__ grad, float *__restrict__ m,
                           float *__restrict__ v, int cnt, float lr, float b1, float b2, float eps, float c1,
                           float c2) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
        const float g = grad[k];
        const float mk = b1 * m[k] + (1.f - b1) * g;
        const float vk = b2 * v[k] + (1.f - b2) * g * g;
        m[k] = mk;
        v[k] = vk;
        theta[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
static int warp_grid(int64_t rows, int sms) {
    const int64_t need = (rows + 7) / 8;
    const int64_t cap = int64_t(sms) * 8;
    return int(std::max<int64_t>(1, std::min(need, cap)));
}

template <typename T>
cudaError_t gnn_forward(const GnnGraph &g, const GnnParams &p, uint64_t feat_seed, GnnActs<T> &a, float *rhat,
                        float *yhat, int sms, cudaStream_t s) {
    const int grid = warp_grid(g.rows, sms);
    k_gnn_features<T><<<std::max<int64_t>(1, std::min<int64_t>((g.rows + 255) / 256, int64_t(sms) * 8)), 256, 0, s>>>(
        g, feat_seed, a.H[0]);
    k_gnn_layer_fwd<T, kGnnFeat><<<grid, 256, 0, s>>>(g, p.Ws[0], p.Wn[0], p.b[0], a.H[0], a.AGG[0], a.H[1]);
    for (int l = 1; l < kGnnLayers; ++l)
        k_gnn_layer_fwd<T, kGnnHid><<<grid, 256, 0, s>>>(g, p.Ws[l], p.Wn[l], p.b[l], a.H[l], a.AGG[l], a.H[l + 1]);
    k_gnn_heads<T><<<grid, 256, 0, s>>>(g, p.WR, p.wy, p.by, a.H[kGnnLayers], rhat, yhat);
    return cudaGetLastError();
}

cudaError_t gnn_warm(const GnnGraph &g, const float *rhat, const float *yhat, const double *cbar, float mix,
                     uint64_t mix_seed, float *R0, double *y0, int sms, cudaStream_t s) {
    const int64_t need = (g.rows * 8 + 255) / 256;
    k_gnn_warm<<<int(std::max<int64_t>(1, std::min<int64_t>(need, int64_t(sms) * 8))), 256, 0, s>>>(
        g, rhat, yhat, cbar, mix, mix_seed, R0, y0);
    return cudaGetLastError();
}

template <typename T>
static void outer_launch(const float *A, const T *B, int64_t rows, int M, int K, int colsum, float *part, int64_t ldp,
                         int nblk, cudaStream_t s) {
    if (M == 64 && K == 64) k_gnn_outer<T, 64, 64><<<nblk, 256, 0, s>>>(A, B, rows, colsum, part, ldp);
    else if (M == 64 && K == 8) k_gnn_outer<T, 64, 8><<<nblk, 256, 0, s>>>(A, B, rows, colsum, part, ldp);
    else if (M == 32 && K == 64) k_gnn_outer<T, 32, 64><<<nblk, 256, 0, s>>>(A, B, rows, colsum, part, ldp);
    else if (M == 1 && K == 64) k_gnn_outer<T, 1, 64><<<nblk, 256, 0, s>>>(A, B, rows, colsum, part, ldp);
}

template <typename T>
cudaError_t gnn_loss_grad(const GnnGraph &g, const GnnParams &p, const GnnParams &grad, GnnActs<T> &a,
                          const float *rhat, const float *yhat, const float *Rs, const double *ys, const double *cbar,
                          double lam, double n_pattern, double n_rows, double *loss_dev, int sms, cudaStream_t s) {
    const int grid = warp_grid(g.rows, sms);
    k_gnn_loss<<<grid, 256, 0, s>>>(g, rhat, yhat, Rs, ys, cbar, p.WR, p.wy, float(1.0 / n_pattern),
                                    float(lam / n_rows), a.dR, a.dY, a.dH, a.lpart);
    k_gnn_sum_loss<<<1, 32, 0, s>>>(a.lpart, grid, loss_dev);
    const int nblk = a.nblk;
    const int64_t ldp = a.ldp;
    auto reduce = [&](float *dst, int cnt) {
        k_gnn_reduce<<<(cnt + 255) / 256, 256, 0, s>>>(a.part, nblk, ldp, cnt, dst);
    };
    const T *H3 = a.H[kGnnLayers];
    // heads: dWR = dR^T H3, dwy = dY^T H3, dby = sum dY
    outer_launch<T>(a.dR, H3, g.rows, kGnnRank, kGnnHid, 0, a.part, ldp, nblk, s);
    reduce(grad.WR, kGnnRank * kGnnHid);
    outer_launch<T>(a.dY, H3, g.rows, 1, kGnnHid, 1, a.part, ldp, nblk, s);
    reduce(grad.wy, kGnnHid);
    k_gnn_reduce<<<1, 32, 0, s>>>(a.part + kGnnHid, nblk, ldp, 1, grad.by);
    float *dH = a.dH;
    for (int l = kGnnLayers - 1; l >= 0; --l) {
        const int din = l == 0 ? kGnnFeat : kGnnHid;
        const bool prev = l > 0;
        if (din == kGnnHid)
            k_gnn_layer_bwd<T, kGnnHid><<<grid, 256, 0, s>>>(g, p.Ws[l], p.Wn[l], a.H[l + 1], dH, a.dZ, a.dHp, a.U, prev);
        else
            k_gnn_layer_bwd<T, kGnnFeat><<<grid, 256, 0, s>>>(g, p.Ws[l], p.Wn[l], a.H[l + 1], dH, a.dZ, a.dHp, a.U, prev);
        outer_launch<T>(a.dZ, a.H[l], g.rows, kGnnHid, din, 1, a.part, ldp, nblk, s);
        reduce(grad.Ws[l], kGnnHid * din);
        k_gnn_reduce<<<1, 64, 0, s>>>(a.part + kGnnHid * din, nblk, ldp, kGnnHid, grad.b[l]);
        outer_launch<T>(a.dZ, a.AGG[l], g.rows, kGnnHid, din, 0, a.part, ldp, nblk, s);
        reduce(grad.Wn[l], kGnnHid * din);
        if (prev) {
            k_gnn_agg_t<kGnnHid><<<grid, 256, 0, s>>>(g, a.U, a.dHp);
            std::swap(a.dH, a.dHp);
            dH = a.dH;
        }
    }
    return cudaGetLastError();
}

cudaError_t gnn_adam(float *theta, const float *grad, float *m, float *v, int cnt, double lr, int step,
                     cudaStream_t s) {
    const double b1 = 0.9, b2 = 0.999;
    const double c1 = 1.0 - std::pow(b1, step), c2 = 1.0 - std::pow(b2, step);
    k_gnn_adam<<<(cnt + 255) / 256, 256, 0, s>>>(theta, grad, m, v, cnt, float(lr), float(b1), float(b2), 1e-8f,
                                                 float(c1), float(c2));
    return cudaGetLastError();
}

#define ALM_GNN_INST(T)                                                                                             \
    template cudaError_t gnn_forward<T>(const GnnGraph &, const GnnParams &, uint64_t, GnnActs<T> &, float *,      \
                                        float *, int, cudaStream_t);                                                \
    template cudaError_t gnn_loss_grad<T>(const GnnGraph &, const GnnParams &, const GnnParams &, GnnActs<T> &,    \
                                          const float *, const float *, const float *, const double *,             \
                                          const double *, double, double, double, double *, int, cudaStream_t);
ALM_GNN_INST(float)
ALM_GNN_INST(__nv_bfloat16)

}  // namespace alm
