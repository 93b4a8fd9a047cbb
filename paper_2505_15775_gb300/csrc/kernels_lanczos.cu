// Lanczos kernels for the smallest eigenpair of S = C - A^*(w) = grad_X L_sigma
// (arXiv 2505.15775, Alg. 1: eigenvectors of grad_X L drive the rank growth;
// Sec. 6: lambda_min(C - A^* y) is the dual term of the KKT error)  [hot path (d)].
//
// One restart cycle builds an orthonormal basis Q = [q_0 .. q_m] (column-major,
// each q_l contiguous) of the Krylov space of S.  Step j (four launches):
//   k_lz_reorth<SPMV>  w = S q_j (sparse part, diagonal, low-rank part of C), formed in
//                      registers and stored, then h1 = Q^T w
//   k_lz_reorth x2     the rest of classical Gram-Schmidt against q_0..q_j, applied twice:
//                      w -= Q h1; h2 = Q^T w; w -= Q h2; beta_j = ||w||
//                      (alpha_j = h1_j + h2_j)
//   k_lz_normalize     q_{j+1} = w / beta_j
// (k_lz_spmv alone serves the residual check of the final Ritz pair)
// and at the end of a cycle
//   k_lz_tridiag    smallest eigenpair (theta, s) of the m x m tridiagonal T in FP64
//                   (Sturm-sequence bisection, then inverse iteration with a pivoted
//                   tridiagonal solve), residual estimate |beta_{m-1} s_{m-1}|
//   k_lz_ritz       v = Q s, the next start vector / the result.
// Dot products accumulate in FP64; the vectors are stored in the working precision.
#include <cfloat>
#include <cmath>

#include "dev_util.cuh"
#include "tridiag.cuh"

namespace alm {

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) as a counter-based generator:
// element i of the stream `seed` is mix(seed + (i + 1) * golden_gamma).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_lz_start(T *__restrict__ q, int64_t n, uint64_t seed, DevState *st,
                                                     double *partials) {
    __shared__ double shm[32];
    double acc = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const uint64_t z = splitmix64_at(seed, uint64_t(i));
        const double u = double(z >> 11) * (1.0 / 9007199254740992.0);  // [0, 1)
        const T x = T(2.0 * u - 1.0);
        q[i] = x;
        acc += double(x) * double(x);
    }
    const double t = block_sum(acc, shm);
    if (threadIdx.x == 0) partials[size_t(blockIdx.x) * kPartStride] = t;
    if (!last_block(&st->counter[CNT_LZ])) return;
    const double s = sum_partials(partials, 0, shm);
    if (threadIdx.x == 0) {
        st->nrm2 = s;
        st->lz_stop = 0;
        st->lz_m = 0;
        st->anorm = 0.0;
    }
}

// warm start: q += (0.05 / |u|) u (|u|^2 in st->nrm2 from k_lz_start), then |q|^2 -> st->nrm2
template <typename T>
__global__ void __launch_bounds__(kBlock) k_lz_mix(T *__restrict__ q, const T *__restrict__ u, int64_t n, DevState *st,
                                                   double *partials) {
    __shared__ double shm[32];
    const T sc = T(0.05 / sqrt(st->nrm2));
    double acc = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const T x = q[i] + sc * u[i];
        q[i] = x;
        acc += double(x) * double(x);
    }
    const double t = block_sum(acc, shm);
    __syncthreads();  // every thread has read st->nrm2
    if (threadIdx.x == 0) partials[size_t(blockIdx.x) * kPartStride] = t;
    if (!last_block(&st->counter[CNT_LZ])) return;
    const double s = sum_partials(partials, 0, shm);
    if (threadIdx.x == 0) st->nrm2 = s;
}

// w = S q (one thread per row)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_lz_spmv(SparseView<T> v, const T *__restrict__ q, T *__restrict__ w,
                                                    const DevState *st) {
    if (st->lz_stop) return;
    T qu[kMaxLR];
    for (int l = 0; l < v.lr_k; ++l) qu[l] = T(v.lr_s[l] * st->qu[l]);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < v.n; i += int64_t(gridDim.x) * blockDim.x) {
        T acc = v.d_s[i] * q[i];
        const int e1 = v.f_ptr[i + 1];
        for (int e = v.f_ptr[i]; e < e1; ++e) acc += v.f_val[e] * q[v.f_col[e]];
        for (int l = 0; l < v.lr_k; ++l) acc += T(v.lr_u[int64_t(l) * v.n + i]) * qu[l];
        w[i] = acc;
    }
}

// stage 0: h = Q^T w, ||w||^2                      (j-th step, nvec = j + 1 basis vectors)
// stage 1: w -= Q h_in; h = Q^T w, ||w||^2
// stage 2: w -= Q h_in; ||w||^2 -> beta_j
// Rows are processed in tiles of kBlock * RPT (each thread keeps RPT entries of w in
// registers); products and per-warp sums are in the working precision, the per-warp
// sums are accumulated over tiles in FP64 in shared memory.
// SPMV (stage 0 only): the SpMV of the step is fused in -- each thread forms its rows of
// w = S q (as k_lz_spmv, same order of operations), stores them and keeps them in
// registers for the dot products, so w is not read back and the step has one launch less.
template <typename T, int RPT, bool SPMV>
__global__ void __launch_bounds__(kBlock) k_lz_reorth(SparseView<T> v, const T *__restrict__ q,
                                                      const T *__restrict__ Q, int64_t ldq, int nvec, T *__restrict__ w,
                                                      int64_t n, const double *__restrict__ h_in, double *h_out, int j,
                                                      int stage, DevState *st, double *partials) {
    if (st->lz_stop) return;
    T qu[kMaxLR];
    if constexpr (SPMV)
        for (int l = 0; l < v.lr_k; ++l) qu[l] = T(v.lr_s[l] * st->qu[l]);
    constexpr int NW = kBlock / 32;
    __shared__ T hs[kLzMax + 1];
    __shared__ double wsum[NW][kLzMax + 2];
    __shared__ double shm[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int l = threadIdx.x; l < nvec; l += blockDim.x) hs[l] = stage > 0 ? T(h_in[l]) : T(0);
    for (int t = threadIdx.x; t < NW * (kLzMax + 2); t += blockDim.x) (&wsum[0][0])[t] = 0.0;
    __syncthreads();
    const int64_t tile = int64_t(kBlock) * RPT;
    T nrm = T(0);
    for (int64_t base = int64_t(blockIdx.x) * tile; base < n; base += int64_t(gridDim.x) * tile) {
        T x[RPT];
        int64_t idx[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            idx[k] = base + threadIdx.x + int64_t(k) * kBlock;
            if constexpr (SPMV) {
                T acc = T(0);
                if (idx[k] < n) {
                    const int64_t i = idx[k];
                    acc = v.d_s[i] * q[i];
                    const int e1 = v.f_ptr[i + 1];
                    for (int e = v.f_ptr[i]; e < e1; ++e) acc += v.f_val[e] * q[v.f_col[e]];
                    for (int l = 0; l < v.lr_k; ++l) acc += T(v.lr_u[int64_t(l) * v.n + i]) * qu[l];
                    w[i] = acc;
                }
                x[k] = acc;
            } else {
                x[k] = idx[k] < n ? w[idx[k]] : T(0);
            }
        }
        if (stage > 0) {
            for (int l = 0; l < nvec; ++l) {
                const T hl = hs[l];
                const T *ql = Q + int64_t(l) * ldq;
#pragma unroll
                for (int k = 0; k < RPT; ++k)
                    if (idx[k] < n) x[k] -= ql[idx[k]] * hl;
            }
#pragma unroll
            for (int k = 0; k < RPT; ++k)
                if (idx[k] < n) w[idx[k]] = x[k];
        }
        if (stage < 2) {
            for (int l = 0; l < nvec; ++l) {
                const T *ql = Q + int64_t(l) * ldq;
                T a = T(0);
#pragma unroll
                for (int k = 0; k < RPT; ++k)
                    if (idx[k] < n) a += ql[idx[k]] * x[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
                if (lane == 0) wsum[warp][l] += double(a);
            }
        }
#pragma unroll
        for (int k = 0; k < RPT; ++k) nrm += x[k] * x[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if (lane == 0) wsum[warp][kLzMax + 1] = double(nrm);
    __syncthreads();
    double *part = partials + size_t(blockIdx.x) * kPartStride;
    const int nslots = stage < 2 ? nvec : 0;
    for (int t = threadIdx.x; t <= nslots; t += blockDim.x) {
        const int src = t == 0 ? kLzMax + 1 : t - 1;
        double sacc = 0.0;
        for (int ww = 0; ww < NW; ++ww) sacc += wsum[ww][src];
        part[t] = sacc;  // slot 0: ||w||^2, slot 1 + l: (Q^T w)_l
    }
    if (!last_block(&st->counter[CNT_LZ])) return;
    // the slots' sums over blocks: one warp per slot, lanes over the blocks in a fixed order
    // (deterministic), all slots at once instead of one block reduction after another
    __shared__ double tot[kLzMax + 2];
    for (int t = warp; t <= nslots; t += NW) {
        double a = 0.0;
        for (int b = lane; b < int(gridDim.x); b += 32) a += __ldcg(partials + size_t(b) * kPartStride + t);
        a = warp_sum(a);
        if (lane == 0) tot[t] = a;
    }
    __syncthreads();
    if (stage < 2)
        for (int l = threadIdx.x; l < nvec; l += blockDim.x) h_out[l] = tot[1 + l];
    const double nrm2 = tot[0];
    (void)shm;
    if (threadIdx.x == 0) {
        st->nrm2 = nrm2;
        if (stage == 0) st->lz_alpha[j] = tot[1 + j];
        if (stage == 1) st->lz_alpha[j] += tot[1 + j];
        if (stage == 2) {
            const double beta = sqrt(nrm2);
            st->lz_beta[j] = beta;
            const double bprev = j > 0 ? st->lz_beta[j - 1] : 0.0;
            st->anorm = fmax(st->anorm, fabs(st->lz_alpha[j]) + beta + bprev);
            st->lz_m = j + 1;
            if (!(beta > 1e-13 * st->anorm)) st->lz_stop = 1;  // invariant subspace (or non-finite)
        }
    }
}

// mode 0: dst = src / sqrt(nrm2);   mode 1: dst = src / beta_j (skipped after a breakdown)
// both: qu_l = u_l^T dst
template <typename T>
__global__ void __launch_bounds__(kBlock) k_lz_normalize(SparseView<T> v, const T *__restrict__ src, T *__restrict__ dst,
                                                         int64_t n, int mode, int j, DevState *st, double *partials) {
    if (mode == 1 && st->lz_stop) return;
    __shared__ double shm[32];
    const double nrm = mode == 0 ? sqrt(st->nrm2) : st->lz_beta[j];
    const T sc = T(nrm > 0.0 ? 1.0 / nrm : 0.0);
    double acc[kMaxLR] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const T x = src[i] * sc;
        dst[i] = x;
        for (int l = 0; l < v.lr_k; ++l) acc[l] += v.lr_u[int64_t(l) * n + i] * double(x);
    }
    if (v.lr_k == 0) return;
    double *part = partials + size_t(blockIdx.x) * kPartStride;
    for (int l = 0; l < v.lr_k; ++l) {
        const double t = block_sum(acc[l], shm);
        if (threadIdx.x == 0) part[l] = t;
    }
    if (!last_block(&st->counter[CNT_LZ])) return;
    for (int l = 0; l < v.lr_k; ++l) {
        const double s = sum_partials(partials, l, shm);
        if (threadIdx.x == 0) st->qu[l] = s;
    }
}

// smallest eigenpair of the m x m tridiagonal T of the cycle (one warp)
__global__ void k_lz_tridiag(DevState *st, int mmax) {
    if (blockIdx.x != 0) return;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) return;
    __shared__ double a[kLzMax], b[kLzMax];
    __shared__ int msh;
    if (lane == 0) msh = st->lz_m < mmax ? st->lz_m : mmax;
    __syncwarp();
    const int m = msh;
    if (m <= 0) return;
    for (int i = lane; i < m; i += 32) {
        a[i] = st->lz_alpha[i];
        b[i] = st->lz_beta[i];
    }
    __syncwarp();
    double resid = 0.0;
    const double theta = warp_tridiag_min(a, b, m, st->lz_s, &resid);
    if (lane != 0) return;
    st->theta = theta;
    st->resid_est = resid;
    st->lz_m = m;
}

// dst = Q[:, 0..m-1] s (and ||dst||^2)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_lz_ritz(const T *__restrict__ Q, int64_t ldq, int mmax, T *__restrict__ dst,
                                                    int64_t n, DevState *st, double *partials) {
    __shared__ double shm[32];
    __shared__ double s[kLzMax];
    const int m = st->lz_m < mmax ? st->lz_m : mmax;
    for (int l = threadIdx.x; l < m; l += blockDim.x) s[l] = st->lz_s[l];
    __syncthreads();
    __shared__ T sT[kLzMax];
    for (int l = threadIdx.x; l < m; l += blockDim.x) sT[l] = T(s[l]);
    __syncthreads();
    T acc = T(0);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        T x = T(0);
        for (int l = 0; l < m; ++l) x += Q[l * ldq + i] * sT[l];
        dst[i] = x;
        acc += x * x;
    }
    const double t = block_sum(double(acc), shm);
    if (threadIdx.x == 0) partials[size_t(blockIdx.x) * kPartStride] = t;
    if (!last_block(&st->counter[CNT_LZ])) return;
    const double nrm2 = sum_partials(partials, 0, shm);
    if (threadIdx.x == 0) st->nrm2 = nrm2;
}

// ||w - theta v||^2 -> st->red[1]   (true residual of the final Ritz pair)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_lz_resid(const T *__restrict__ w, const T *__restrict__ v, int64_t n,
                                                     DevState *st, double *partials) {
    __shared__ double shm[32];
    const T th = T(st->theta);
    T acc = T(0);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const T d = w[i] - th * v[i];
        acc += d * d;
    }
    const double t = block_sum(double(acc), shm);
    if (threadIdx.x == 0) partials[size_t(blockIdx.x) * kPartStride] = t;
    if (!last_block(&st->counter[CNT_LZ])) return;
    const double s = sum_partials(partials, 0, shm);
    if (threadIdx.x == 0) st->red[1] = s;
}

__global__ void k_lz_reset(DevState *st) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st->lz_stop = 0;
        st->lz_m = 0;
    }
}

// ---------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------
static inline int lz_grid(const LaunchCtx &c, int64_t n) {
    int64_t need = (n + kBlock - 1) / kBlock;
    if (need < 1) need = 1;
    return int(need < c.grid ? need : c.grid);
}

template <typename T>
void launch_lz_start(const LaunchCtx &c, T *q, int64_t n, uint64_t seed) {
    k_lz_start<T><<<lz_grid(c, n), kBlock, 0, c.stream>>>(q, n, seed, c.st, c.partials);
    ++*c.launches;
}

template <typename T>
void launch_lz_mix(const LaunchCtx &c, T *q, const T *u, int64_t n) {
    k_lz_mix<T><<<lz_grid(c, n), kBlock, 0, c.stream>>>(q, u, n, c.st, c.partials);
    ++*c.launches;
}

template <typename T>
void launch_lz_spmv(const LaunchCtx &c, const SparseView<T> &v, const T *q, T *w) {
    k_lz_spmv<T><<<lz_grid(c, v.n), kBlock, 0, c.stream>>>(v, q, w, c.st);
    ++*c.launches;
}

static inline int lz_tiles_grid(const LaunchCtx &c, int64_t n, int rpt) {
    const int64_t tiles = (n + int64_t(kBlock) * rpt - 1) / (int64_t(kBlock) * rpt);
    return int(tiles < c.grid ? tiles : c.grid);
}

// Four rows per thread amortise the per-tile warp sums; a vector too short to give every
// multiprocessor a tile that way takes one row per thread (more CTAs, shorter chains: the
// small eigensolves are latency-bound).
static inline bool lz_one_row(const LaunchCtx &c, int64_t n) {
    return (n + int64_t(kBlock) * 4 - 1) / (int64_t(kBlock) * 4) < int64_t(c.sms);
}

template <typename T>
void launch_lz_reorth(const LaunchCtx &c, const T *Q, int64_t ldq, int nvec, T *w, int64_t n, const double *h_in,
                      double *h_out, int j, int stage) {
    if (lz_one_row(c, n))
        k_lz_reorth<T, 1, false><<<lz_tiles_grid(c, n, 1), kBlock, 0, c.stream>>>(
            SparseView<T>{}, nullptr, Q, ldq, nvec, w, n, h_in, h_out, j, stage, c.st, c.partials);
    else
        k_lz_reorth<T, 4, false><<<lz_tiles_grid(c, n, 4), kBlock, 0, c.stream>>>(
            SparseView<T>{}, nullptr, Q, ldq, nvec, w, n, h_in, h_out, j, stage, c.st, c.partials);
    ++*c.launches;
}

template <typename T>
void launch_lz_spmv_reorth(const LaunchCtx &c, const SparseView<T> &v, const T *q, const T *Q, int64_t ldq, int nvec,
                           T *w, double *h_out, int j) {
    if (lz_one_row(c, v.n))
        k_lz_reorth<T, 1, true><<<lz_tiles_grid(c, v.n, 1), kBlock, 0, c.stream>>>(
            v, q, Q, ldq, nvec, w, v.n, nullptr, h_out, j, 0, c.st, c.partials);
    else
        k_lz_reorth<T, 4, true><<<lz_tiles_grid(c, v.n, 4), kBlock, 0, c.stream>>>(
            v, q, Q, ldq, nvec, w, v.n, nullptr, h_out, j, 0, c.st, c.partials);
    ++*c.launches;
}

template <typename T>
void launch_lz_normalize(const LaunchCtx &c, const SparseView<T> &v, const T *src, T *dst, int64_t n, int mode,
                         int j) {
    k_lz_normalize<T><<<lz_grid(c, n), kBlock, 0, c.stream>>>(v, src, dst, n, mode, j, c.st, c.partials);
    ++*c.launches;
}

void launch_lz_tridiag(const LaunchCtx &c, int m) {
    k_lz_tridiag<<<1, 32, 0, c.stream>>>(c.st, m);
    ++*c.launches;
}

void launch_lz_reset(const LaunchCtx &c) {
    k_lz_reset<<<1, 32, 0, c.stream>>>(c.st);
    ++*c.launches;
}

template <typename T>
void launch_lz_ritz(const LaunchCtx &c, const T *Q, int64_t ldq, int m, T *dst, int64_t n) {
    k_lz_ritz<T><<<lz_grid(c, n), kBlock, 0, c.stream>>>(Q, ldq, m, dst, n, c.st, c.partials);
    ++*c.launches;
}

template <typename T>
void launch_lz_resid(const LaunchCtx &c, const T *w, const T *v, int64_t n) {
    k_lz_resid<T><<<lz_grid(c, n), kBlock, 0, c.stream>>>(w, v, n, c.st, c.partials);
    ++*c.launches;
}

#define ALM_LZ_INST(T)                                                                                          \
    template void launch_lz_start<T>(const LaunchCtx &, T *, int64_t, uint64_t);                                \
    template void launch_lz_mix<T>(const LaunchCtx &, T *, const T *, int64_t);                                 \
    template void launch_lz_spmv<T>(const LaunchCtx &, const SparseView<T> &, const T *, T *);                  \
    template void launch_lz_reorth<T>(const LaunchCtx &, const T *, int64_t, int, T *, int64_t, const double *, \
                                      double *, int, int);                                                      \
    template void launch_lz_spmv_reorth<T>(const LaunchCtx &, const SparseView<T> &, const T *, const T *, int64_t, \
                                           int, T *, double *, int);                                            \
    template void launch_lz_normalize<T>(const LaunchCtx &, const SparseView<T> &, const T *, T *, int64_t, int, \
                                         int);                                                                  \
    template void launch_lz_ritz<T>(const LaunchCtx &, const T *, int64_t, int, T *, int64_t);                  \
    template void launch_lz_resid<T>(const LaunchCtx &, const T *, const T *, int64_t);

ALM_LZ_INST(float)
ALM_LZ_INST(double)

}  // namespace alm
