// Device and host helpers shared by the sparse kernels of the inner loop (kernels_sparse.cu,
// kernels_inner.cu): row loads, deterministic block / grid reductions, the float-pair slack
// diagonal, ELL fetches, and the last-block bookkeeping of the SpMM and the line search.
#pragma once

#include <cmath>
#include <mutex>
#include <unordered_map>

#include "dev_util.cuh"
#include "fpair.cuh"
#include "quartic.cuh"

namespace alm {

template <typename T>
__device__ __forceinline__ typename VecT<T>::type load_row(const T *__restrict__ R, int64_t i, int ldr, int gl,
                                                           bool active) {
    constexpr int W = VecT<T>::W;
    return active ? ldro(R + i * ldr + gl * W) : vzero(T());
}

// In the last block: deterministic sums over blocks of the partial slots 0..NV-1, all
// slots loaded in one pass (results valid in thread 0).
template <int NV>
__device__ __forceinline__ void sum_partials_n(const double *partials, double (&out)[NV], double *shm) {
    double t[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) t[k] = 0.0;
    for (int b = threadIdx.x; b < int(gridDim.x); b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) t[k] += __ldcg(partials + size_t(b) * kPartStride + k);
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = block_sum(t[k], shm);
}

// write the block sums of vals[0..NV) to part[0..NV)
template <int NV>
__device__ __forceinline__ void block_partials(const double (&vals)[NV], double *part, double *shm) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const double t = block_sum(vals[k], shm);
        if (threadIdx.x == 0) part[k] = t;
    }
}

// a double as a float pair hi + lo (FP32 form) or as itself (FP64 form)
template <typename T>
__device__ __forceinline__ void store_slack_diag(const SparseView<T> &v, int64_t i, double d) {
    T hi, lo;
    split_pair(d, hi, lo);
    v.d_s[i] = hi;
    if (v.d_s_lo) v.d_s_lo[i] = lo;
}

// ---------------------------------------------------------------------------------------
// inner-loop slack update for diagonal-selector problems (MaxCut): with y fixed during an
// inner solve, S_ii = (C_ii - a_i y_k) + sigma a_i (a_i |r_i|^2 - b_k) = base_i + sigma a_i res_i.
// base_i is a float pair computed once per outer iteration; res_i is formed from the
// compensated |r_i|^2 in float-pair arithmetic (the subtraction of b_k ~ 1 is where FP32
// would lose the residual), so the whole update runs in FP32 on one streaming pass over R.
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void slack_pair(const SparseView<T> &v, int64_t i, T xh, T xl, T sigma, T &dh_out,
                                           T &dl_out) {
    const int k = v.d_sel_k[i];
    T dh = v.base_hi[i], dl = v.base_lo ? v.base_lo[i] : T(0);
    if (k >= 0) {
        const T a = sizeof(T) == 8 ? T(v.d_sel_a[i]) : T(v.d_sel_af[i]);
        const T ph = a * xh;
        const T pe = fma(a, xh, -ph) + a * xl;
        const T s0 = ph - v.b_hi[i];
        const T bb = s0 - ph;
        const T e0 = (ph - (s0 - bb)) + (-v.b_hi[i] - bb);
        const T res = s0 + (e0 + pe - (v.b_lo ? v.b_lo[i] : T(0)));
        const T corr = sigma * a * res;
        const T s1 = dh + corr;
        const T b1 = s1 - dh;
        dl += (dh - (s1 - b1)) + (corr - b1);
        dh = s1;
    }
    dh_out = dh;
    dl_out = dl;
}

// ---------------------------------------------------------------------------------------
// ELL forms of the SpMM and of the line-search SDDMM (static S_off, rows of at most KF
// entries).  One row per group and iteration; the column indices and values of the
// group's next row are fetched before the current row's gathers are issued, so that a
// row costs one memory latency instead of a chain of three.
// ---------------------------------------------------------------------------------------
template <typename T, int KF>
__device__ __forceinline__ void ell_fetch(const int *__restrict__ cols, const T *__restrict__ vals, int64_t row,
                                          int (&jj)[KF], T (&ss)[KF]) {
    const int4 *cp = reinterpret_cast<const int4 *>(cols + row * KF);
#pragma unroll
    for (int q = 0; q < KF / 4; ++q) {
        const int4 c = __ldg(cp + q);
        jj[4 * q] = c.x;
        jj[4 * q + 1] = c.y;
        jj[4 * q + 2] = c.z;
        jj[4 * q + 3] = c.w;
    }
#pragma unroll
    for (int k = 0; k < KF; ++k) ss[k] = __ldg(vals + row * KF + k);
}
template <typename T, int K>
__device__ __forceinline__ void ell_fetch2(const int *__restrict__ cols, const T *__restrict__ vals, int64_t row,
                                           int (&jj)[K], T (&ss)[K]) {  // K = 2 (8-byte rows)
    const int2 c = __ldg(reinterpret_cast<const int2 *>(cols + row * K));
    jj[0] = c.x;
    jj[1] = c.y;
    ss[0] = __ldg(vals + row * K);
    ss[1] = __ldg(vals + row * K + 1);
}

// last-block bookkeeping of the inner CG step (shared by the CSR and ELL SpMMs)
__device__ __forceinline__ void spmm_finish(DevState *st, double gg, double go, double gd, double zg) {
    st->gg = gg;
    if (!isfinite(gg)) {
        st->status = ALM_ERR_NUMERIC;
        st->done = 1;
    } else if (sqrt(gg) <= st->tau_abs) {
        st->done = 1;
    }
    double beta = 0.0;
    if (!st->restart && st->method == ALM_INNER_CG && st->zg_prev > 0.0) {
        beta = fmax(0.0, (zg - go) / st->zg_prev);
        if (-zg + beta * gd >= 0.0) beta = 0.0;  // not a descent direction: restart
    }
    st->beta = beta;
    st->g_gprev = go;
    st->g_dprev = gd;
    st->gg_prev = gg;
    st->zg = zg;
    st->zg_prev = zg;
    st->restart = 0;
}

// thread 0 of the last block of a line-search SDDMM: FP64 quartic coefficients, the
// exact step and (MODE 1) the inner-loop bookkeeping
template <typename T, int MODE, bool LR>
__device__ __forceinline__ void ls_finish(const SparseView<T> &v, DevState *st, int r, const double (&tot)[5]) {
        double s1 = tot[0], s2 = tot[1], a11 = tot[2], a12 = tot[3], a22 = tot[4];
        if (LR)  // <s u u^T, RD^T + DR^T> = 2 s (R^T u).(D^T u),  <s u u^T, DD^T> = s |D^T u|^2
            for (int l = 0; l < v.lr_k; ++l) {
                double zr = 0.0, dd = 0.0;
                for (int col = 0; col < r; ++col) {
                    zr += st->z[l][col] * st->zd[l][col];
                    dd += st->zd[l][col] * st->zd[l][col];
                }
                s1 += v.lr_s[l] * 2.0 * zr;
                s2 += v.lr_s[l] * dd;
            }
        for (int g = 0; g < v.m_gen; ++g) {
            const double A1 = v.g_a1[g], A2 = v.g_a2[g];
            a11 += A1 * A1;
            a12 += A1 * A2;
            a22 += A2 * A2;
        }
        const double sigma = st->sigma;
        double q[5];
        q[0] = st->L;
        q[1] = (MODE == 1) ? (-st->zg + st->beta * st->g_dprev) : s1;  // <G, D>, D = -Z + beta D_old
        q[2] = s2 + 0.5 * sigma * a11;
        q[3] = sigma * a12;
        q[4] = 0.5 * sigma * a22;
        st->c1 = s1;
        st->c2 = s2;
        st->a11 = a11;
        st->a12 = a12;
        st->a22 = a22;
        for (int k = 0; k < 5; ++k) st->q[k] = q[k];
        int unb = 0;
        const double alpha = quartic_argmin(q, &unb);
        st->alpha = unb ? 0.0 : alpha;
        if (MODE == 1) {
            bool finite = true;
            for (int k = 0; k < 5; ++k) finite = finite && isfinite(q[k]);
            if (!finite) {
                st->status = ALM_ERR_NUMERIC;
                st->done = 1;
            } else if (unb) {
                st->status = ALM_ERR_UNBOUNDED;
                st->done = 1;
            } else if (!(alpha > 0.0)) {
                st->done = 1;
            } else {
                st->iters += 1;
                if (st->iters >= st->max_inner) st->done = 2;
            }
        } else if (unb) {
            st->status = ALM_ERR_UNBOUNDED;
            st->alpha = INFINITY;
        }
    }

// blocks of kBlock threads per SM that the kernel can keep resident (cached per kernel)
static int resident_blocks(const void *fn) {
    static std::mutex mu;
    static std::unordered_map<const void *, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(fn);
    if (it != cache.end()) return it->second;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kBlock, 0) != cudaSuccess || b < 1) {
        (void)cudaGetLastError();
        b = 1;
    }
    cache[fn] = b;
    return b;
}

template <typename K>
static int grid_for(const LaunchCtx &c, K *fn, int64_t items, int64_t items_per_block) {
    int64_t need = (items + items_per_block - 1) / items_per_block;
    if (need < 1) need = 1;
    int64_t cap = int64_t(c.sms) * resident_blocks(reinterpret_cast<const void *>(fn));
    if (cap > c.grid) cap = c.grid;
    return int(need < cap ? need : cap);
}

static inline int lanes_for(int r, int W) {
    const int nvec = (r + W - 1) / W;
    int L = 1;
    while (L < nvec) L <<= 1;
    return L;
}

#define ALM_DISPATCH_LANES(L, ...)                                \
    switch (L) {                                                  \
        case 1: { constexpr int LN = 1; __VA_ARGS__; } break;    \
        case 2: { constexpr int LN = 2; __VA_ARGS__; } break;    \
        case 4: { constexpr int LN = 4; __VA_ARGS__; } break;    \
        case 8: { constexpr int LN = 8; __VA_ARGS__; } break;    \
        default: { constexpr int LN = 16; __VA_ARGS__; } break;  \
    }

}  // namespace alm
