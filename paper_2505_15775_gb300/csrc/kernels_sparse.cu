// Hot-path kernels of the ALM-BM inner loop (arXiv 2505.15775, Eq. AL-BM, Alg. 1):
//
//   k_eval       A(RR^T) and <C, RR^T> (SDDMM v_p = r_i . r_j over the aggregated
//                pattern) with the direct scatter of selector constraints into A(X);
//                for problems whose constraints are all diagonal selectors (MaxCut)
//                also the dual update w = y - sigma(A(X) - b), diag(S) and the L / KKT
//                reductions                                            [hot path (a)]
//   k_gen_eval   A(RR^T)_k of the general (multi-entry) constraints
//   k_dual_slack w, the L / KKT reductions and S = C - A^*(w) (general problems)
//   k_spmm       G = 2 S R (+ the low-rank part of C), ||G||^2 and the CG inner
//                products                                              [hot path (b)]
//   k_dir        D = -G + beta D
//   k_ls         the quartic phi(alpha) = L(R + alpha D): a1 = A(RD^T + DR^T),
//                a2 = A(DD^T), <S, RD^T + DR^T>, <S, DD^T> in one pass over R and D,
//                FP64 coefficients and the exact minimiser            [hot path (c)]
//   k_gen_ls     a1, a2 of the general constraints
//   k_axpy       R += alpha D
//
// Work decomposition.  A group of LANES lanes owns one row of R (lane l holds the
// 16-byte vector of columns [l W, l W + W), W = 4 floats or 2 doubles), so a gathered
// row is one coalesced 16*LANES-byte read and a dot product is a shuffle reduction
// inside the group.  The SDDMMs run a streaming pass over the diagonal (rows) and an
// entry-parallel pass over the strict upper pattern (COO), two entries per group and
// iteration, so that every lane keeps four independent row gathers in flight.  The
// SpMM walks two rows per group and iteration with predicated, independent gathers.
//
// Precision.  FP64 arithmetic is scarce on GB300, so in the FP32 form every per-entry
// product and every per-thread partial sum is FP32; partials are promoted to FP64 once
// per thread, summed per block in FP64 and over blocks in FP64 by the last block to
// finish (a fixed order: results are deterministic).  The dual w and the constraint
// residuals are FP64 throughout.
#include <cfloat>
#include <cmath>
#include <mutex>
#include <unordered_map>

#include "sparse_common.cuh"

namespace alm {

// ---------------------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------------------

// Block-reduce the per-lane column vectors acc[l][k] (column gl*W + k of term l) over the
// row groups of the block into part[l*kMaxRank + col] (columns no lane covers are 0).
template <typename T, int LANES>
__device__ __forceinline__ void block_reduce_cols(double (*acc)[VecT<T>::W], int nl, double *part, double *shm) {
    constexpr int W = VecT<T>::W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = threadIdx.x; t < nl * kMaxRank; t += blockDim.x) part[t] = 0.0;
    for (int l = 0; l < nl; ++l) {
        for (int k = 0; k < W; ++k) {
            double x = acc[l][k];
#pragma unroll
            for (int o = 16; o >= LANES; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            __syncthreads();
            if (lane < LANES) shm[warp * 32 + lane] = x;
            __syncthreads();
            if (threadIdx.x < LANES) {
                double t = 0.0;
                for (int w = 0; w < nw; ++w) t += shm[w * 32 + threadIdx.x];
                const int col = threadIdx.x * W + k;
                if (col < kMaxRank) part[l * kMaxRank + col] = t;
            }
        }
    }
}




template <typename T, int LANES>
__device__ __forceinline__ void slack_row(const SparseView<T> &v, int64_t i, T xh, T xl, T sigma) {
    const int k = v.d_sel_k[i];
    T dh = v.base_hi[i], dl = v.base_lo ? v.base_lo[i] : T(0);
    if (k >= 0) {
        const T a = sizeof(T) == 8 ? T(v.d_sel_a[i]) : T(v.d_sel_af[i]);
        // a x = (ph + pe) + a xl exactly up to the last term's rounding
        const T ph = a * xh;
        const T pe = fma(a, xh, -ph) + a * xl;
        // res = (ph - b_hi) + (pe - b_lo), the first difference with two-sum
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
    v.d_s[i] = dh;
    if (v.d_s_lo) v.d_s_lo[i] = dl;
    if (v.ls_rec) v.ls_rec[i].ds = dh;
}

// STEP: first apply the pending step R += alpha D of the previous line search (alpha = 0
// at the start of an inner solve), so that no separate update pass is needed.
// Four rows per group and iteration are loaded before any of them is used.
template <typename T, int LANES, bool STEP>
__global__ void __launch_bounds__(kBlock, 4) k_inner_slack(SparseView<T> v, T *__restrict__ R, const T *__restrict__ D,
                                                        int r, int ldr, const DevState *st, const int *done) {
    if (*done) return;
    using V = typename VecT<T>::type;
    constexpr int W = VecT<T>::W;
    constexpr int B = 4;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (LANES - 1);
    const unsigned gmask = group_mask<LANES>(lane);
    const int gpb = kBlock / LANES;
    const int64_t ng = int64_t(gridDim.x) * gpb;
    const bool active = gl * W < r;
    const bool writer = gl * W < ldr;
    const T sigma = T(st->sigma);
    const T alpha = STEP ? T(st->alpha) : T(0);
    const bool step = STEP && alpha != T(0);
    for (int64_t i0 = int64_t(blockIdx.x) * gpb + threadIdx.x / LANES; i0 < v.n; i0 += B * ng) {
        V rv[B];
        int64_t row[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            row[b] = i0 + b * ng;
            const bool ok = row[b] < v.n;
            rv[b] = ok && writer ? ld(R + row[b] * ldr + gl * W) : vzero(T());
        }
        if (step) {
            V dv[B];
#pragma unroll
            for (int b = 0; b < B; ++b) dv[b] = row[b] < v.n && writer ? ld(D + row[b] * ldr + gl * W) : vzero(T());
#pragma unroll
            for (int b = 0; b < B; ++b) {
                rv[b] = fma4(alpha, dv[b], rv[b]);
                if (row[b] < v.n && writer) stv(R + row[b] * ldr + gl * W, rv[b]);
            }
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            if (row[b] >= v.n) break;  // group-uniform
            T xh, xl;
            norm2_pair(mask_tail(rv[b], gl * W, r), gmask, LANES, xh, xl);
            if (gl == 0) slack_row<T, LANES>(v, row[b], xh, xl, sigma);
        }
    }
}

// base_i = C_ii - a_i y_k(i) (rows without a diagonal selector: C_ii), as a float pair
template <typename T>
__global__ void __launch_bounds__(kBlock) k_prep_base(SparseView<T> v, const double *__restrict__ y,
                                                      T *__restrict__ base_hi, T *__restrict__ base_lo) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < v.n; i += int64_t(gridDim.x) * blockDim.x) {
        double d = double(v.d_c[i]);
        const int k = v.d_sel_k[i];
        if (k >= 0) d -= v.d_sel_a[i] * y[k];
        T hi, lo;
        split_pair(d, hi, lo);
        base_hi[i] = hi;
        if (base_lo) base_lo[i] = lo;
        if (v.step_rec) {
            v.step_rec[i].base_hi = float(hi);
            v.step_rec[i].base_lo = float(lo);
        }
    }
}

// ---------------------------------------------------------------------------------------
// (a) constraint map + <C, RR^T> (+ fused dual update for diagonal-selector problems)
// ---------------------------------------------------------------------------------------
template <typename T, int LANES, bool OFFSEL, bool LR, bool FUSED>
__global__ void __launch_bounds__(kBlock) k_eval(SparseView<T> v, const T *__restrict__ R, int r, int ldr,
                                                 double *__restrict__ AX, const double *__restrict__ y,
                                                 double *__restrict__ w, DevState *st, double *partials,
                                                 const int *done) {
    if (*done) return;
    using V = typename VecT<T>::type;
    constexpr int W = VecT<T>::W;
    __shared__ double shm[32 * 32];
    const int lane = threadIdx.x & 31;
    const int gl = lane & (LANES - 1);
    const unsigned gmask = group_mask<LANES>(lane);
    const int gpb = kBlock / LANES;
    const int64_t g0 = int64_t(blockIdx.x) * gpb + threadIdx.x / LANES;
    const int64_t ng = int64_t(gridDim.x) * gpb;
    const bool active = gl * W < r;
    const double sigma = FUSED ? st->sigma : 0.0;
    T pc = T(0);
    double pyres = 0.0, pres2 = 0.0, pbw = 0.0;
    double lacc[LR ? kMaxLR : 1][W];
    if (LR)
        for (int l = 0; l < kMaxLR; ++l)
            for (int k = 0; k < W; ++k) lacc[l][k] = 0.0;

    // diagonal entries: one streaming pass over the rows of R
    for (int64_t i = g0; i < v.n; i += ng) {
        const V ri = mask_tail(load_row(R, i, ldr, gl, active), gl * W, r);
        const double viid = ff_norm2<LANES>(ri, gmask);  // compensated in FP32
        const T vii = T(viid);
        if (gl == 0) {
            const T cii = v.d_c[i];
            pc += cii * vii;
            const int k = v.d_sel_k[i];
            if (k >= 0) {
                const double a = v.d_sel_a[i];
                const double ax = a * viid;
                AX[k] = ax;
                if (FUSED) {
                    const double res = ax - v.b[k];
                    const double wk = y[k] - sigma * res;
                    w[k] = wk;
                    store_slack_diag(v, i, double(cii) - wk * a);
                    pyres += y[k] * res;
                    pres2 += res * res;
                    pbw += v.b[k] * wk;
                }
            } else if (FUSED) {
                store_slack_diag(v, i, double(cii));
            }
        }
        if (LR)
            for (int l = 0; l < v.lr_k; ++l) {
                const double u = v.lr_u[int64_t(l) * v.n + i];
                for (int k = 0; k < W; ++k) lacc[l][k] += u * double(comp(ri, k));
            }
    }
    // strict upper entries: two per group and iteration
    for (int64_t e = g0; e < v.nnz_u; e += 2 * ng) {
        const int64_t e2 = e + ng;
        const bool has2 = e2 < v.nnz_u;
        const int i0 = v.up_row[e], j0 = v.up_col[e];
        const int i1 = has2 ? v.up_row[e2] : i0, j1 = has2 ? v.up_col[e2] : j0;
        const V a0 = load_row(R, i0, ldr, gl, active);
        const V b0 = load_row(R, j0, ldr, gl, active);
        const V a1 = load_row(R, i1, ldr, gl, active);
        const V b1 = load_row(R, j1, ldr, gl, active);
        const T x0 = group_sum<LANES>(dot(mask_tail(a0, gl * W, r), b0), gmask);
        const T x1 = group_sum<LANES>(dot(mask_tail(a1, gl * W, r), b1), gmask);
        if (gl == 0) {
            pc += T(2) * v.up_c[e] * x0;
            if (has2) pc += T(2) * v.up_c[e2] * x1;
            if (OFFSEL) {
                const int k0 = v.up_sel_k[e];
                if (k0 >= 0) AX[k0] = 2.0 * v.up_sel_a[e] * double(x0);
                if (has2) {
                    const int k1 = v.up_sel_k[e2];
                    if (k1 >= 0) AX[k1] = 2.0 * v.up_sel_a[e2] * double(x1);
                }
            }
        }
    }
    double *part = partials + size_t(blockIdx.x) * kPartStride;
    if (FUSED) {
        const double vals[4] = {double(pc), pyres, pres2, pbw};
        block_partials<4>(vals, part, shm);
    } else {
        const double vals[1] = {double(pc)};
        block_partials<1>(vals, part, shm);
    }
    if (LR) block_reduce_cols<T, LANES>(lacc, v.lr_k, part + 4, shm);
    if (!last_block(&st->counter[CNT_EVAL])) return;
    const double c0 = sum_partials(partials, 0, shm);
    double yres = 0.0, res2 = 0.0, bw = 0.0;
    if (FUSED) {
        yres = sum_partials(partials, 1, shm);
        res2 = sum_partials(partials, 2, shm);
        bw = sum_partials(partials, 3, shm);
    }
    if (LR)
        for (int l = 0; l < v.lr_k; ++l)
            for (int col = 0; col < kMaxRank; ++col) {
                const double t = sum_partials(partials, 4 + l * kMaxRank + col, shm);
                if (threadIdx.x == 0) st->z[l][col] = t;
            }
    if (threadIdx.x == 0) {
        double c = c0;
        for (int l = 0; LR && l < v.lr_k; ++l) {
            double zz = 0.0;
            for (int col = 0; col < r; ++col) zz += st->z[l][col] * st->z[l][col];
            c += v.lr_s[l] * zz;
        }
        st->c0 = c;
        if (FUSED) {
            st->yres = yres;
            st->res2 = res2;
            st->bw = bw;
            st->L = c - yres + 0.5 * sigma * res2;
            if (!isfinite(st->L)) {
                st->status = ALM_ERR_NUMERIC;
                st->done = 1;
            }
        }
    }
}

// general constraints: A(X)_k = sum over its entries of kappa a (r_i . r_j); one block each
template <typename T>
__global__ void __launch_bounds__(kBlock) k_gen_eval(SparseView<T> v, const T *__restrict__ R, int r, int ldr,
                                                     double *__restrict__ AX, const int *done) {
    if (*done) return;
    __shared__ double shm[32];
    for (int g = blockIdx.x; g < v.m_gen; g += gridDim.x) {
        double acc = 0.0;
        for (int t = v.g_ptr[g] + threadIdx.x; t < v.g_ptr[g + 1]; t += blockDim.x) {
            const int i = v.g_i[t], j = v.g_j[t];
            T x = T(0);
            for (int c = 0; c < r; ++c) x += R[int64_t(i) * ldr + c] * R[int64_t(j) * ldr + c];
            acc += (i == j ? 1.0 : 2.0) * v.g_a[t] * double(x);
        }
        const double s = block_sum(acc, shm);
        if (threadIdx.x == 0) AX[v.g_con[g]] = s;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// dual update, L and KKT reductions, slack values S = C - A^*(w) (general problems)
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBlock) k_dual_slack(SparseView<T> v, const double *__restrict__ y,
                                                       const double *__restrict__ AX, double *__restrict__ w,
                                                       const int2 *__restrict__ up_slot, DevState *st,
                                                       double *partials, const int *done) {
    if (*done) return;
    __shared__ double shm[32];
    const double sigma = st->sigma;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nt = int64_t(gridDim.x) * blockDim.x;
    double pyres = 0.0, pres2 = 0.0, pbw = 0.0;
    for (int64_t k = tid; k < v.m; k += nt) {
        const double res = AX[k] - v.b[k];
        const double wk = y[k] - sigma * res;
        w[k] = wk;
        pyres += y[k] * res;
        pres2 += res * res;
        pbw += v.b[k] * wk;
    }
    // w_k is recomputed where another block owns k
#define WOF(k) (y[(k)] - sigma * (AX[(k)] - v.b[(k)]))
    for (int64_t i = tid; i < v.n; i += nt) {
        double s = double(v.d_c[i]);
        const int k = v.d_sel_k[i];
        if (k >= 0) s -= WOF(k) * v.d_sel_a[i];
        if (v.gd_ptr)
            for (int t = v.gd_ptr[i]; t < v.gd_ptr[i + 1]; ++t) s -= WOF(v.gd_k[t]) * v.gd_a[t];
        store_slack_diag(v, i, s);
    }
    if (v.off_dynamic) {
        for (int64_t e = tid; e < v.nnz_u; e += nt) {
            double s = double(v.up_c[e]);
            if (v.has_off_sel) {
                const int k = v.up_sel_k[e];
                if (k >= 0) s -= WOF(k) * v.up_sel_a[e];
            }
            if (v.gu_ptr)
                for (int t = v.gu_ptr[e]; t < v.gu_ptr[e + 1]; ++t) s -= WOF(v.gu_k[t]) * v.gu_a[t];
            const T sv = T(s);
            v.up_s[e] = sv;
            const int2 sl = up_slot[e];
            v.f_val[sl.x] = sv;
            v.f_val[sl.y] = sv;
        }
    }
#undef WOF
    const double vals[3] = {pyres, pres2, pbw};
    block_partials<3>(vals, partials + size_t(blockIdx.x) * kPartStride, shm);
    if (!last_block(&st->counter[CNT_DUAL])) return;
    const double yres = sum_partials(partials, 0, shm);
    const double res2 = sum_partials(partials, 1, shm);
    const double bw = sum_partials(partials, 2, shm);
    if (threadIdx.x == 0) {
        st->yres = yres;
        st->res2 = res2;
        st->bw = bw;
        st->L = st->c0 - yres + 0.5 * sigma * res2;
        if (!isfinite(st->L)) {
            st->status = ALM_ERR_NUMERIC;
            st->done = 1;
        }
    }
}

// ---------------------------------------------------------------------------------------
// (b) G = 2 S R
//   MODE 0: gradient only (and ||G||^2)
//   MODE 1: inner CG step: also <G, G_old> (G is updated in place) and <G, D_old>, the
//           stop test ||G|| <= tau and the Polak-Ribiere+ coefficient
// ---------------------------------------------------------------------------------------
template <typename T, int LANES, bool LR, int MODE>
__global__ void __launch_bounds__(kBlock, 3) k_spmm(SparseView<T> v, const T *__restrict__ R, int r, int ldr,
                                                 T *G, const T *D, DevState *st, double *partials,
                                                 const int *done) {
    if (*done) return;
    using V = typename VecT<T>::type;
    constexpr int W = VecT<T>::W;
    constexpr int U = 4;  // neighbours per row and round
    __shared__ double shm[32];
    const int lane = threadIdx.x & 31;
    const int gl = lane & (LANES - 1);
    const int gpb = kBlock / LANES;
    const int64_t g0 = int64_t(blockIdx.x) * gpb + threadIdx.x / LANES;
    const int64_t ng = int64_t(gridDim.x) * gpb;
    const bool active = gl * W < r;
    const bool writer = gl * W < ldr;
    V zl[LR ? kMaxLR : 1];
    if (LR)
        for (int l = 0; l < v.lr_k; ++l) {
            T zz[W];
            for (int k = 0; k < W; ++k) {
                const int col = gl * W + k;
                zz[k] = (col < r) ? T(v.lr_s[l] * st->z[l][col]) : T(0);
            }
            if constexpr (W == 4) zl[l] = make_float4(zz[0], zz[1], zz[2], zz[3]);
            else zl[l] = make_double2(zz[0], zz[1]);
        }
    T pgg = T(0), pgo = T(0), pgd = T(0), pzg = T(0);
    const unsigned gmask = group_mask<LANES>(lane);
    const bool pc = MODE == 1 && st->precond;
    const T sig = T(st->sigma);
    const T pc_floor = T(st->pc_floor);
    for (int64_t i = g0; i < v.n; i += 2 * ng) {
        const int64_t i2 = i + ng;
        const bool has2 = i2 < v.n;
        const int64_t ib = has2 ? i2 : i;  // a valid row for predicated accesses
        const V ri = mask_tail(load_row(R, i, ldr, gl, active), gl * W, r);
        const V rb = mask_tail(load_row(R, ib, ldr, gl, active), gl * W, r);
        using Acc = typename AccOf<T>::type;
        Acc acc, acb;
        acc.init();
        acb.init();
        acc.add(v.d_s[i], ri);
        acb.add(has2 ? v.d_s[ib] : T(0), rb);
        if (v.d_s_lo) {
            acc.add_lo(v.d_s_lo[i], ri);
            acb.add_lo(has2 ? v.d_s_lo[ib] : T(0), rb);
        }
        int e = v.f_ptr[i];
        const int e1 = v.f_ptr[i + 1];
        int f = has2 ? v.f_ptr[ib] : 0;
        const int f1 = has2 ? v.f_ptr[ib + 1] : 0;
        while (e < e1 || f < f1) {
            int ja[U], jb[U];
            T sa[U], sb[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const bool oa = e + k < e1, ob = f + k < f1;
                ja[k] = oa ? v.f_col[e + k] : int(i);
                sa[k] = oa ? v.f_val[e + k] : T(0);
                jb[k] = ob ? v.f_col[f + k] : int(ib);
                sb[k] = ob ? v.f_val[f + k] : T(0);
            }
            V ga[U], gb[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                ga[k] = load_row(R, ja[k], ldr, gl, active);
                gb[k] = load_row(R, jb[k], ldr, gl, active);
            }
#pragma unroll
            for (int k = 0; k < U; ++k) {
                acc.add(sa[k], ga[k]);
                acb.add(sb[k], gb[k]);
            }
            e += U;
            f += U;
        }
        if (LR)
            for (int l = 0; l < v.lr_k; ++l) {
                acc.add(T(v.lr_u[int64_t(l) * v.n + i]), zl[l]);
                acb.add(T(v.lr_u[int64_t(l) * v.n + ib]), zl[l]);
            }
        const V ga = mask_tail(scale4(T(2), acc.value()), gl * W, r);
        const V gb = mask_tail(scale4(T(2), acb.value()), gl * W, r);
        pgg += dot(ga, ga);
        if (has2) pgg += dot(gb, gb);
        if (MODE == 1) {
            // Row-block Jacobi preconditioner Z = P^{-1} G with P_i = 2 s_i I + 4 sigma a_i^2 r_i r_i^T
            // (the block of the Hessian of L in row i: the S_ii part and the penalty of the
            // diagonal selector a_i e_i e_i^T), inverted by Sherman-Morrison; s_i = S_ii floored.
            V za = ga, zb = gb;
            if (pc) {
                const T rga = group_sum<LANES>(dot(ri, ga), gmask), rra = group_sum<LANES>(dot(ri, ri), gmask);
                const T rgb = group_sum<LANES>(dot(rb, gb), gmask), rrb = group_sum<LANES>(dot(rb, rb), gmask);
                auto precond_row = [&](int64_t row, T rg, T rr, V g, V rv) -> V {
                    T sdi = v.d_s[row] + (v.d_s_lo ? v.d_s_lo[row] : T(0));
                    sdi = sdi > pc_floor ? sdi : pc_floor;
                    const int k = v.d_sel_k[row];
                    const T a = k >= 0 ? T(v.d_sel_a[row]) : T(0);
                    const T ka = T(4) * sig * a * a;
                    const T coef = ka * rg / (T(2) * sdi + ka * rr);
                    const T inv = T(1) / (T(2) * sdi);
                    V z = fma4(-coef, rv, g);
                    return scale4(inv, z);
                };
                za = precond_row(i, rga, rra, ga, ri);
                zb = precond_row(ib, rgb, rrb, gb, rb);
            }
            if (active) {
                pzg += dot(za, ga);
                pgo += dot(ga, ld(G + i * ldr + gl * W));
                pgd += dot(ga, ld(D + i * ldr + gl * W));
                if (has2) {
                    pzg += dot(zb, gb);
                    pgo += dot(gb, ld(G + ib * ldr + gl * W));
                    pgd += dot(gb, ld(D + ib * ldr + gl * W));
                }
            }
            if (writer) {
                stv(G + i * ldr + gl * W, za);
                if (has2) stv(G + ib * ldr + gl * W, zb);
            }
        } else if (writer) {
            stv(G + i * ldr + gl * W, ga);
            if (has2) stv(G + ib * ldr + gl * W, gb);
        }
    }
    double *part = partials + size_t(blockIdx.x) * kPartStride;
    if (MODE == 1) {
        const double vals[4] = {double(pgg), double(pgo), double(pgd), double(pzg)};
        block_partials<4>(vals, part, shm);
    } else {
        const double vals[1] = {double(pgg)};
        block_partials<1>(vals, part, shm);
    }
    if (!last_block(&st->counter[CNT_SPMM])) return;
    const double gg = sum_partials(partials, 0, shm);
    double go = 0.0, gd = 0.0, zg = 0.0;
    if (MODE == 1) {
        go = sum_partials(partials, 1, shm);
        gd = sum_partials(partials, 2, shm);
        zg = sum_partials(partials, 3, shm);
    }
    if (threadIdx.x == 0) {
        st->gg = gg;
        if (MODE == 1) {
            if (!isfinite(gg)) {
                st->status = ALM_ERR_NUMERIC;
                st->done = 1;
            } else if (sqrt(gg) <= st->tau_abs) {
                st->done = 1;
            }
            // Polak-Ribiere+ on the preconditioned gradient Z (Z = G without preconditioning):
            // beta = max(0, <Z, G - G_old> / <Z_old, G_old>), with <Z, G_old> taken as
            // <G, Z_old> (P symmetric and slowly varying), so that only Z is stored
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
    }
}


template <typename T, int LANES, int KF, int MODE>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 8 ? 3 : 4) k_spmm_ell(SparseView<T> v, const T *__restrict__ R, int r, int ldr,
                                                     T *G, const T *D, DevState *st, double *partials,
                                                     const int *done) {
    if (*done) return;
    using V = typename VecT<T>::type;
    constexpr int W = VecT<T>::W;
    __shared__ double shm[32];
    const int lane = threadIdx.x & 31;
    const int gl = lane & (LANES - 1);
    const unsigned gmask = group_mask<LANES>(lane);
    const int gpb = kBlock / LANES;
    const int64_t ng = int64_t(gridDim.x) * gpb;
    const bool active = gl * W < r;
    const bool writer = gl * W < ldr;
    const bool pc = MODE == 1 && st->precond;
    const T sig = T(st->sigma);
    const T pc_floor = T(st->pc_floor);
    T pgg = T(0), pgo = T(0), pgd = T(0), pzg = T(0);
    int jc[KF];
    T sc[KF];
    int64_t i = int64_t(blockIdx.x) * gpb + threadIdx.x / LANES;
    if (i < v.n) ell_fetch<T, KF>(v.f_ell_col, v.f_ell_val, i, jc, sc);
    for (; i < v.n; i += ng) {
        const int64_t inext = i + ng;
        int jn[KF];
        T sn[KF];
        if (inext < v.n) ell_fetch<T, KF>(v.f_ell_col, v.f_ell_val, inext, jn, sn);
        const V ri = mask_tail(load_row(R, i, ldr, gl, active), gl * W, r);
        const T dsi = v.d_s[i];
        const T dlo = v.d_s_lo ? v.d_s_lo[i] : T(0);
        V gold = vzero(T()), dold = vzero(T());
        if (MODE == 1 && active) {
            gold = ld(G + i * ldr + gl * W);
            dold = ld(D + i * ldr + gl * W);
        }
        V gth[KF];
#pragma unroll
        for (int k = 0; k < KF; ++k) gth[k] = load_row(R, jc[k], ldr, gl, active);
        using Acc = typename AccOf<T>::type;
        Acc acc;
        acc.init();
        acc.add(dsi, ri);
        acc.add_lo(dlo, ri);
#pragma unroll
        for (int k = 0; k < KF; ++k) acc.add(sc[k], gth[k]);
        const V g = mask_tail(scale4(T(2), acc.value()), gl * W, r);
        pgg += dot(g, g);
        if (MODE == 1) {
            V z = g;
            if (pc) {
                const T rg = group_sum<LANES>(dot(ri, g), gmask), rr = group_sum<LANES>(dot(ri, ri), gmask);
                T sdi = dsi + dlo;
                sdi = sdi > pc_floor ? sdi : pc_floor;
                const int k = v.d_sel_k[i];
                const T a = k >= 0 ? T(v.d_sel_a[i]) : T(0);
                const T ka = T(4) * sig * a * a;
                const T coef = ka * rg / (T(2) * sdi + ka * rr);
                z = scale4(T(1) / (T(2) * sdi), fma4(-coef, ri, g));
            }
            pzg += dot(z, g);
            pgo += dot(g, gold);
            pgd += dot(g, dold);
            if (writer) stv(G + i * ldr + gl * W, z);
        } else if (writer) {
            stv(G + i * ldr + gl * W, g);
        }
#pragma unroll
        for (int k = 0; k < KF; ++k) {
            jc[k] = jn[k];
            sc[k] = sn[k];
        }
    }
    double *part = partials + size_t(blockIdx.x) * kPartStride;
    const double vals[4] = {double(pgg), double(pgo), double(pgd), double(pzg)};
    block_partials<4>(vals, part, shm);
    if (!last_block(&st->counter[CNT_SPMM])) return;
    double tot[4];
    sum_partials_n<4>(partials, tot, shm);
    if (threadIdx.x == 0) {
        if (MODE == 1) spmm_finish(st, tot[0], tot[1], tot[2], tot[3]);
        else st->gg = tot[0];
    }
}


// D = -G + beta D
template <typename T>
__global__ void __launch_bounds__(kBlock) k_dir(const T *__restrict__ G, T *__restrict__ D, int64_t nvec,
                                                const DevState *st, const int *done) {
    if (*done) return;
    using V = typename VecT<T>::type;
    const T beta = T(st->beta);
    const V *g = reinterpret_cast<const V *>(G);
    V *d = reinterpret_cast<V *>(D);
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nvec; t += int64_t(gridDim.x) * blockDim.x) {
        const V gv = g[t];
        V dv = (beta != T(0)) ? d[t] : vzero(T());  // D may hold stale values when beta = 0
        d[t] = fma4(beta, dv, scale4(T(-1), gv));
    }
}


// ---------------------------------------------------------------------------------------
// (c) exact line search along D.  With a1 = A(RD^T + DR^T), a2 = A(DD^T) and S = C - A^*(w)
// at the current R, phi(alpha) = L(R + alpha D) has
//   q1 = <S, RD^T + DR^T> (= <grad_R L, D>),  q2 = <S, DD^T> + sigma/2 |a1|^2,
//   q3 = sigma a1.a2,  q4 = sigma/2 |a2|^2,  q0 = L
// (the expansion of Eq. AL with c_k - w.a_k folded into <S, .>).
//   MODE 0: coefficients and step only.
//   MODE 1: inner loop: q1 from the SpMM's inner products (<G, D> = -|G|^2 + beta <G, D_old>,
//           free of cancellation), plus the done / iteration bookkeeping.
// ---------------------------------------------------------------------------------------
template <typename T, int LANES, bool OFFSEL, bool LR, int MODE>
__global__ void __launch_bounds__(kBlock, 3) k_ls(SparseView<T> v, const T *__restrict__ R, const T *__restrict__ D,
                                               int r, int ldr, DevState *st, double *partials, const int *done) {
    if (*done) return;
    using V = typename VecT<T>::type;
    constexpr int W = VecT<T>::W;
    __shared__ double shm[32 * 32];
    const int lane = threadIdx.x & 31;
    const int gl = lane & (LANES - 1);
    const unsigned gmask = group_mask<LANES>(lane);
    const int gpb = kBlock / LANES;
    const int64_t g0 = int64_t(blockIdx.x) * gpb + threadIdx.x / LANES;
    const int64_t ng = int64_t(gridDim.x) * gpb;
    const bool active = gl * W < r;
    T p1 = T(0), p2 = T(0), p11 = T(0), p12 = T(0), p22 = T(0);
    double lacc[LR ? kMaxLR : 1][W];
    if (LR)
        for (int l = 0; l < kMaxLR; ++l)
            for (int k = 0; k < W; ++k) lacc[l][k] = 0.0;

    // one row-based pass: rows i and i + ng per group and iteration, each with its strict
    // upper neighbours (two per round, predicated), so that R and D stream from HBM once
    constexpr int U = 2;
    auto sel_terms = [&](int k, double a_k, T x1, T x2) {
        if (k >= 0) {
            const T a = T(a_k);
            const T A1 = a * x1, A2 = a * x2;
            p11 += A1 * A1;
            p12 += A1 * A2;
            p22 += A2 * A2;
        }
    };
    for (int64_t i = g0; i < v.n; i += 2 * ng) {
        const int64_t i2 = i + ng;
        const bool has2 = i2 < v.n;
        const int64_t ib = has2 ? i2 : i;
        const V ri = mask_tail(load_row(R, i, ldr, gl, active), gl * W, r);
        const V di = mask_tail(load_row(D, i, ldr, gl, active), gl * W, r);
        const V rb = mask_tail(load_row(R, ib, ldr, gl, active), gl * W, r);
        const V db = mask_tail(load_row(D, ib, ldr, gl, active), gl * W, r);
        const T a1i = T(2) * group_sum<LANES>(dot(ri, di), gmask);
        const T a2i = group_sum<LANES>(dot(di, di), gmask);
        const T a1b = T(2) * group_sum<LANES>(dot(rb, db), gmask);
        const T a2b = group_sum<LANES>(dot(db, db), gmask);
        if (gl == 0) {
            const T si = v.d_s[i];
            p1 += si * a1i;
            p2 += si * a2i;
            sel_terms(v.d_sel_k[i], v.d_sel_a[i], a1i, a2i);
            if (has2) {
                const T sb = v.d_s[ib];
                p1 += sb * a1b;
                p2 += sb * a2b;
                sel_terms(v.d_sel_k[ib], v.d_sel_a[ib], a1b, a2b);
            }
        }
        if (LR)
            for (int l = 0; l < v.lr_k; ++l) {
                const double u = v.lr_u[int64_t(l) * v.n + i];
                const double ub = has2 ? v.lr_u[int64_t(l) * v.n + ib] : 0.0;
                for (int k = 0; k < W; ++k) lacc[l][k] += u * double(comp(di, k)) + ub * double(comp(db, k));
            }
        int e = v.up_ptr[i];
        const int e1 = v.up_ptr[i + 1];
        int f = has2 ? v.up_ptr[ib] : 0;
        const int f1 = has2 ? v.up_ptr[ib + 1] : 0;
        while (e < e1 || f < f1) {
            int ja[U], jb[U];
            T sa[U], sbv[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const bool oa = e + k < e1, ob = f + k < f1;
                ja[k] = oa ? v.up_col[e + k] : int(i);
                sa[k] = oa ? T(2) * v.up_s[e + k] : T(0);
                jb[k] = ob ? v.up_col[f + k] : int(ib);
                sbv[k] = ob ? T(2) * v.up_s[f + k] : T(0);
            }
            V rja[U], dja[U], rjb[U], djb[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                rja[k] = load_row(R, ja[k], ldr, gl, active);
                dja[k] = load_row(D, ja[k], ldr, gl, active);
                rjb[k] = load_row(R, jb[k], ldr, gl, active);
                djb[k] = load_row(D, jb[k], ldr, gl, active);
            }
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const T x1a = group_sum<LANES>(dot(ri, dja[k]) + dot(di, rja[k]), gmask);
                const T x2a = group_sum<LANES>(dot(di, dja[k]), gmask);
                const T x1b = group_sum<LANES>(dot(rb, djb[k]) + dot(db, rjb[k]), gmask);
                const T x2b = group_sum<LANES>(dot(db, djb[k]), gmask);
                if (gl == 0) {
                    p1 += sa[k] * x1a + sbv[k] * x1b;
                    p2 += sa[k] * x2a + sbv[k] * x2b;
                    if (OFFSEL) {
                        if (e + k < e1) sel_terms(v.up_sel_k[e + k], 2.0 * v.up_sel_a[e + k], x1a, x2a);
                        if (f + k < f1) sel_terms(v.up_sel_k[f + k], 2.0 * v.up_sel_a[f + k], x1b, x2b);
                    }
                }
            }
            e += U;
            f += U;
        }
    }
    double *part = partials + size_t(blockIdx.x) * kPartStride;
    const double vals[5] = {double(p1), double(p2), double(p11), double(p12), double(p22)};
    block_partials<5>(vals, part, shm);
    if (LR) block_reduce_cols<T, LANES>(lacc, v.lr_k, part + 8, shm);
    if (!last_block(&st->counter[CNT_LS])) return;
    double tot[5];
    for (int k = 0; k < 5; ++k) tot[k] = sum_partials(partials, k, shm);
    if (LR)
        for (int l = 0; l < v.lr_k; ++l)
            for (int col = 0; col < kMaxRank; ++col) {
                const double t = sum_partials(partials, 8 + l * kMaxRank + col, shm);
                if (threadIdx.x == 0) st->zd[l][col] = t;
            }
    if (threadIdx.x == 0) ls_finish<T, MODE, LR>(v, st, r, tot);
}

// ELL form of the line-search SDDMM (static S_off: no off-diagonal selector constraints,
// no low-rank C): one row per group and iteration, the next row's upper neighbours fetched
// ahead of the current row's gathers of R and D
template <typename T, int LANES, int KU, int MODE>
__global__ void __launch_bounds__(kBlock, 4) k_ls_ell(SparseView<T> v, const T *__restrict__ R,
                                                   const T *__restrict__ D, int r, int ldr, DevState *st,
                                                   double *partials, const int *done) {
    if (*done) return;
    using V = typename VecT<T>::type;
    constexpr int W = VecT<T>::W;
    __shared__ double shm[32];
    const int lane = threadIdx.x & 31;
    const int gl = lane & (LANES - 1);
    const unsigned gmask = group_mask<LANES>(lane);
    const int gpb = kBlock / LANES;
    const int64_t ng = int64_t(gridDim.x) * gpb;
    const bool active = gl * W < r;
    T p1 = T(0), p2 = T(0), p11 = T(0), p12 = T(0), p22 = T(0);
    int jc[KU];
    T sc[KU];
    auto fetch = [&](int64_t row, int (&jj)[KU], T (&ss)[KU]) {
        if constexpr (KU == 2) ell_fetch2<T, KU>(v.u_ell_col, v.u_ell_val, row, jj, ss);
        else ell_fetch<T, KU>(v.u_ell_col, v.u_ell_val, row, jj, ss);
    };
    int64_t i = int64_t(blockIdx.x) * gpb + threadIdx.x / LANES;
    if (i < v.n) fetch(i, jc, sc);
    for (; i < v.n; i += ng) {
        const V ri = mask_tail(load_row(R, i, ldr, gl, active), gl * W, r);
        const V di = mask_tail(load_row(D, i, ldr, gl, active), gl * W, r);
        V rj[KU], dj[KU];
#pragma unroll
        for (int k = 0; k < KU; ++k) {
            rj[k] = load_row(R, jc[k], ldr, gl, active);
            dj[k] = load_row(D, jc[k], ldr, gl, active);
        }
        T sq[KU];
#pragma unroll
        for (int k = 0; k < KU; ++k) sq[k] = T(2) * sc[k];
        // the next row's neighbours, fetched while this row's gathers are in flight
        if (i + ng < v.n) fetch(i + ng, jc, sc);
        // <S, RD^T + DR^T> and <S, DD^T> need no per-row reduction: every lane accumulates its
        // columns' share (the S values are the same for all lanes of the row) and the block
        // reduction at the end sums lanes and rows together.  Only the diagonal selector's
        // a1, a2 are reduced per row (their squares enter q2..q4).
        const T rdi = dot(ri, di), ddi = dot(di, di);
        const T sii = v.d_s[i];
        T l1 = T(2) * sii * rdi, l2 = sii * ddi;
#pragma unroll
        for (int k = 0; k < KU; ++k) {
            l1 += sq[k] * (dot(ri, dj[k]) + dot(di, rj[k]));
            l2 += sq[k] * dot(di, dj[k]);
        }
        p1 += l1;
        p2 += l2;
        const int ksel = v.d_sel_k[i];
        if (ksel >= 0) {  // group-uniform
            const T a1 = T(2) * group_sum<LANES>(rdi, gmask);
            const T a2 = group_sum<LANES>(ddi, gmask);
            if (gl == 0) {
                const T a = T(v.d_sel_a[i]);
                const T A1 = a * a1, A2 = a * a2;
                p11 += A1 * A1;
                p12 += A1 * A2;
                p22 += A2 * A2;
            }
        }
    }
    const double vals[5] = {double(p1), double(p2), double(p11), double(p12), double(p22)};
    block_partials<5>(vals, partials + size_t(blockIdx.x) * kPartStride, shm);
    if (!last_block(&st->counter[CNT_LS])) return;
    double tot[5];
    sum_partials_n<5>(partials, tot, shm);
    if (threadIdx.x == 0) ls_finish<T, MODE, false>(v, st, r, tot);
}


// general constraints of the line search: A1_g, A2_g; one block each
template <typename T>
__global__ void __launch_bounds__(kBlock) k_gen_ls(SparseView<T> v, const T *__restrict__ R,
                                                   const T *__restrict__ D, int r, int ldr, const int *done) {
    if (*done) return;
    __shared__ double shm[32];
    for (int g = blockIdx.x; g < v.m_gen; g += gridDim.x) {
        double a1 = 0.0, a2 = 0.0;
        for (int t = v.g_ptr[g] + threadIdx.x; t < v.g_ptr[g + 1]; t += blockDim.x) {
            const int i = v.g_i[t], j = v.g_j[t];
            T x1 = T(0), x2 = T(0);
            for (int c = 0; c < r; ++c) {
                const T ric = R[int64_t(i) * ldr + c], rjc = R[int64_t(j) * ldr + c];
                const T dic = D[int64_t(i) * ldr + c], djc = D[int64_t(j) * ldr + c];
                x1 += ric * djc + dic * rjc;
                x2 += dic * djc;
            }
            const double ka = (i == j ? 1.0 : 2.0) * v.g_a[t];
            a1 += ka * double(x1);
            a2 += ka * double(x2);
        }
        const double s1 = block_sum(a1, shm);
        const double s2 = block_sum(a2, shm);
        if (threadIdx.x == 0) {
            v.g_a1[g] = s1;
            v.g_a2[g] = s2;
        }
        __syncthreads();
    }
}

// R += alpha D  (skipped when done == 1; done == 2, the step that reached the iteration cap,
// still takes this update and then becomes done == 1, so that the remaining launches of the
// chunk apply nothing)
template <typename T>
__global__ void __launch_bounds__(kBlock) k_axpy(T *__restrict__ R, const T *__restrict__ D, int64_t nvec,
                                                 DevState *st, const int *done, int final_only) {
    const int d = *done;
    if (d == 1 || (final_only && d != 2)) return;
    using V = typename VecT<T>::type;
    const T alpha = T(st->alpha);
    V *x = reinterpret_cast<V *>(R);
    const V *dv = reinterpret_cast<const V *>(D);
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < nvec; t += int64_t(gridDim.x) * blockDim.x)
        x[t] = fma4(alpha, dv[t], x[t]);
    if (d == 2 && last_block(&st->counter[CNT_AXPY]) && threadIdx.x == 0) st->done = 1;
}

// dst (n x ld_dst) <- src (n x ld_src) columns 0..r-1, zero columns r..ld_dst-1,
// optionally column r <- scale * col
template <typename T>
__global__ void __launch_bounds__(kBlock) k_relayout(const T *__restrict__ src, int ld_src, T *__restrict__ dst,
                                                     int ld_dst, int r, int64_t n, const T *__restrict__ col,
                                                     double scale) {
    const int64_t total = n * ld_dst;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += int64_t(gridDim.x) * blockDim.x) {
        const int64_t i = t / ld_dst;
        const int c = int(t - i * ld_dst);
        T x = T(0);
        if (c < r) x = src[i * ld_src + c];
        else if (c == r && col) x = T(scale * double(col[i]));
        dst[t] = x;
    }
}

// st->red[0] = sum_k x_k^2
static __global__ void __launch_bounds__(kBlock) k_sumsq(const double *__restrict__ x, int64_t m, DevState *st,
                                                  double *partials) {
    __shared__ double shm[32];
    double acc = 0.0;
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < m; k += int64_t(gridDim.x) * blockDim.x)
        acc += x[k] * x[k];
    const double t = block_sum(acc, shm);
    if (threadIdx.x == 0) partials[size_t(blockIdx.x) * kPartStride] = t;
    if (!last_block(&st->counter[CNT_RED])) return;
    const double s = sum_partials(partials, 0, shm);
    if (threadIdx.x == 0) st->red[0] = s;
}

// ---------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------

template <typename T, int LN, bool OFF, bool LRB, bool FUS>
static void eval_one(const LaunchCtx &c, const SparseView<T> &v, const T *R, int r, int ldr, double *AX,
                     const double *y, double *w, const int *done) {
    auto *fn = k_eval<T, LN, OFF, LRB, FUS>;
    const int grid = grid_for(c, fn, v.n + v.nnz_u, kBlock / LN);
    fn<<<grid, kBlock, 0, c.stream>>>(v, R, r, ldr, AX, y, w, c.st, c.partials, done);
}

template <typename T>
void launch_eval(const LaunchCtx &c, const SparseView<T> &v, const T *R, int r, int ldr, double *AX, const int *done,
                 const double *y, double *w) {
    constexpr int W = VecT<T>::W;
    const int L = lanes_for(r, W);
    if (v.m_gen > 0) {
        k_gen_eval<T><<<v.m_gen < c.grid ? v.m_gen : c.grid, kBlock, 0, c.stream>>>(v, R, r, ldr, AX, done);
        ++*c.launches;
    }
    const bool fused = v.fused_dual && y && w;
    const bool off = v.has_off_sel, lr = v.lr_k > 0;
    ALM_DISPATCH_LANES(L, {
        if (fused) {
            if (lr) eval_one<T, LN, false, true, true>(c, v, R, r, ldr, AX, y, w, done);
            else eval_one<T, LN, false, false, true>(c, v, R, r, ldr, AX, y, w, done);
        } else if (off && lr) eval_one<T, LN, true, true, false>(c, v, R, r, ldr, AX, y, w, done);
        else if (off) eval_one<T, LN, true, false, false>(c, v, R, r, ldr, AX, y, w, done);
        else if (lr) eval_one<T, LN, false, true, false>(c, v, R, r, ldr, AX, y, w, done);
        else eval_one<T, LN, false, false, false>(c, v, R, r, ldr, AX, y, w, done);
    });
    ++*c.launches;
}

template <typename T>
void launch_inner_slack(const LaunchCtx &c, const SparseView<T> &v, T *R, const T *D, int r, int ldr,
                        const int *done) {
    constexpr int W = VecT<T>::W;
    const int L = lanes_for(r, W);
    ALM_DISPATCH_LANES(L, {
        if (D) {
            auto *fn = k_inner_slack<T, LN, true>;
            const int grid = grid_for(c, fn, v.n, 4 * (kBlock / LN));
            fn<<<grid, kBlock, 0, c.stream>>>(v, R, D, r, ldr, c.st, done);
        } else {
            auto *fn = k_inner_slack<T, LN, false>;
            const int grid = grid_for(c, fn, v.n, 4 * (kBlock / LN));
            fn<<<grid, kBlock, 0, c.stream>>>(v, R, D, r, ldr, c.st, done);
        }
    });
    ++*c.launches;
}

template <typename T>
void launch_prep_base(const LaunchCtx &c, const SparseView<T> &v, const double *y, T *base_hi, T *base_lo) {
    auto *fn = k_prep_base<T>;
    const int grid = grid_for(c, fn, v.n, kBlock * 4);
    fn<<<grid, kBlock, 0, c.stream>>>(v, y, base_hi, base_lo);
    ++*c.launches;
}

template <typename T>
void launch_dual_slack(const LaunchCtx &c, const SparseView<T> &v, const double *y, const double *AX, double *w,
                       const int *done, const int2 *up_slot) {
    int64_t items = v.n > v.m ? v.n : v.m;
    if (v.off_dynamic && v.nnz_u > items) items = v.nnz_u;
    auto *fn = k_dual_slack<T>;
    const int grid = grid_for(c, fn, items, kBlock * 2);
    fn<<<grid, kBlock, 0, c.stream>>>(v, y, AX, w, up_slot, c.st, c.partials, done);
    ++*c.launches;
}

template <typename T, int LN, bool LRB, int MODE>
static void spmm_one(const LaunchCtx &c, const SparseView<T> &v, const T *R, int r, int ldr, T *G, const T *D,
                     const int *done) {
    auto *fn = k_spmm<T, LN, LRB, MODE>;
    const int grid = grid_for(c, fn, v.n, 2 * (kBlock / LN));
    fn<<<grid, kBlock, 0, c.stream>>>(v, R, r, ldr, G, D, c.st, c.partials, done);
}

template <typename T, int LN, int KF>
static void spmm_ell_one(const LaunchCtx &c, const SparseView<T> &v, const T *R, int r, int ldr, T *G, const T *D,
                         int mode, const int *done) {
    if (mode == 1) {
        auto *fn = k_spmm_ell<T, LN, KF, 1>;
        fn<<<grid_for(c, fn, v.n, kBlock / LN), kBlock, 0, c.stream>>>(v, R, r, ldr, G, D, c.st, c.partials, done);
    } else {
        auto *fn = k_spmm_ell<T, LN, KF, 0>;
        fn<<<grid_for(c, fn, v.n, kBlock / LN), kBlock, 0, c.stream>>>(v, R, r, ldr, G, D, c.st, c.partials, done);
    }
}

template <typename T>
void launch_spmm(const LaunchCtx &c, const SparseView<T> &v, const T *R, int r, int ldr, T *G, const T *D, int mode,
                 const int *done) {
    constexpr int W = VecT<T>::W;
    const int L = lanes_for(r, W);
    const bool lr = v.lr_k > 0;
    if (v.ell_kf > 0 && !lr) {
        ALM_DISPATCH_LANES(L, {
            if (v.ell_kf == 4) spmm_ell_one<T, LN, 4>(c, v, R, r, ldr, G, D, mode, done);
            else if (v.ell_kf == 8) spmm_ell_one<T, LN, 8>(c, v, R, r, ldr, G, D, mode, done);
            else spmm_ell_one<T, LN, 16>(c, v, R, r, ldr, G, D, mode, done);
        });
        ++*c.launches;
        return;
    }
    ALM_DISPATCH_LANES(L, {
        if (mode == 1) {
            if (lr) spmm_one<T, LN, true, 1>(c, v, R, r, ldr, G, D, done);
            else spmm_one<T, LN, false, 1>(c, v, R, r, ldr, G, D, done);
        } else {
            if (lr) spmm_one<T, LN, true, 0>(c, v, R, r, ldr, G, D, done);
            else spmm_one<T, LN, false, 0>(c, v, R, r, ldr, G, D, done);
        }
    });
    ++*c.launches;
}

template <typename T>
void launch_dir(const LaunchCtx &c, const T *G, T *D, int64_t count, const int *done) {
    constexpr int W = VecT<T>::W;
    const int64_t nvec = count / W;
    auto *fn = k_dir<T>;
    const int grid = grid_for(c, fn, nvec, kBlock * 2);
    fn<<<grid, kBlock, 0, c.stream>>>(G, D, nvec, c.st, done);
    ++*c.launches;
}

template <typename T, int LN, bool OFF, bool LRB, int MODE>
static void ls_one(const LaunchCtx &c, const SparseView<T> &v, const T *R, const T *D, int r, int ldr,
                   const int *done) {
    auto *fn = k_ls<T, LN, OFF, LRB, MODE>;
    const int grid = grid_for(c, fn, v.n, 2 * (kBlock / LN));
    fn<<<grid, kBlock, 0, c.stream>>>(v, R, D, r, ldr, c.st, c.partials, done);
}

template <typename T, int LN, int KU>
static void ls_ell_one(const LaunchCtx &c, const SparseView<T> &v, const T *R, const T *D, int r, int ldr, int mode,
                       const int *done) {
    if (mode == 1) {
        auto *fn = k_ls_ell<T, LN, KU, 1>;
        fn<<<grid_for(c, fn, v.n, kBlock / LN), kBlock, 0, c.stream>>>(v, R, D, r, ldr, c.st, c.partials, done);
    } else {
        auto *fn = k_ls_ell<T, LN, KU, 0>;
        fn<<<grid_for(c, fn, v.n, kBlock / LN), kBlock, 0, c.stream>>>(v, R, D, r, ldr, c.st, c.partials, done);
    }
}

template <typename T>
void launch_ls(const LaunchCtx &c, const SparseView<T> &v, const T *R, const T *D, int r, int ldr, const double *w,
               int mode, const int *done) {
    (void)w;
    constexpr int W = VecT<T>::W;
    const int L = lanes_for(r, W);
    if (v.ell_ku > 0 && v.lr_k == 0 && !v.has_off_sel && v.m_gen == 0) {
        ALM_DISPATCH_LANES(L, {
            if (v.ell_ku == 2) ls_ell_one<T, LN, 2>(c, v, R, D, r, ldr, mode, done);
            else if (v.ell_ku == 4) ls_ell_one<T, LN, 4>(c, v, R, D, r, ldr, mode, done);
            else if (v.ell_ku == 8) ls_ell_one<T, LN, 8>(c, v, R, D, r, ldr, mode, done);
            else ls_ell_one<T, LN, 16>(c, v, R, D, r, ldr, mode, done);
        });
        ++*c.launches;
        return;
    }
    if (v.m_gen > 0) {
        k_gen_ls<T><<<v.m_gen < c.grid ? v.m_gen : c.grid, kBlock, 0, c.stream>>>(v, R, D, r, ldr, done);
        ++*c.launches;
    }
    const bool off = v.has_off_sel, lr = v.lr_k > 0;
#define ALM_LS(OFF, LRB)                                                     \
    if (mode == 1) ls_one<T, LN, OFF, LRB, 1>(c, v, R, D, r, ldr, done);    \
    else ls_one<T, LN, OFF, LRB, 0>(c, v, R, D, r, ldr, done);
    ALM_DISPATCH_LANES(L, {
        if (off && lr) { ALM_LS(true, true) }
        else if (off) { ALM_LS(true, false) }
        else if (lr) { ALM_LS(false, true) }
        else { ALM_LS(false, false) }
    });
#undef ALM_LS
    ++*c.launches;
}

template <typename T>
void launch_axpy(const LaunchCtx &c, T *R, const T *D, int64_t count, const int *done, int final_only) {
    constexpr int W = VecT<T>::W;
    const int64_t nvec = count / W;
    auto *fn = k_axpy<T>;
    const int grid = grid_for(c, fn, nvec, kBlock * 2);
    fn<<<grid, kBlock, 0, c.stream>>>(R, D, nvec, c.st, done, final_only);
    ++*c.launches;
}

template <typename T>
void launch_relayout(const LaunchCtx &c, const T *src, int ld_src, T *dst, int ld_dst, int r, int64_t n, const T *col,
                     double scale) {
    auto *fn = k_relayout<T>;
    const int grid = grid_for(c, fn, n * ld_dst, kBlock * 4);
    fn<<<grid, kBlock, 0, c.stream>>>(src, ld_src, dst, ld_dst, r, n, col, scale);
    ++*c.launches;
}

template <typename T>
void launch_sumsq(const LaunchCtx &c, const double *x, int64_t m) {
    const int grid = grid_for(c, k_sumsq, m, kBlock * 4);
    k_sumsq<<<grid, kBlock, 0, c.stream>>>(x, m, c.st, c.partials);
    ++*c.launches;
}

#define ALM_INST(T)                                                                                              \
    template void launch_eval<T>(const LaunchCtx &, const SparseView<T> &, const T *, int, int, double *,        \
                                 const int *, const double *, double *);                                         \
    template void launch_dual_slack<T>(const LaunchCtx &, const SparseView<T> &, const double *, const double *, \
                                       double *, const int *, const int2 *);                                     \
    template void launch_inner_slack<T>(const LaunchCtx &, const SparseView<T> &, T *, const T *, int, int,      \
                                        const int *);                                                             \
    template void launch_prep_base<T>(const LaunchCtx &, const SparseView<T> &, const double *, T *, T *);      \
    template void launch_spmm<T>(const LaunchCtx &, const SparseView<T> &, const T *, int, int, T *, const T *,  \
                                 int, const int *);                                                              \
    template void launch_dir<T>(const LaunchCtx &, const T *, T *, int64_t, const int *);                         \
    template void launch_ls<T>(const LaunchCtx &, const SparseView<T> &, const T *, const T *, int, int,         \
                               const double *, int, const int *);                                                \
    template void launch_axpy<T>(const LaunchCtx &, T *, const T *, int64_t, const int *, int);                   \
    template void launch_relayout<T>(const LaunchCtx &, const T *, int, T *, int, int, int64_t, const T *,       \
                                     double);                                                                    \
    template void launch_sumsq<T>(const LaunchCtx &, const double *, int64_t);

// ALM_INST_ONLY (1: float, 2: double) lets the build compile the two precisions as separate
// objects in parallel
#if !defined(ALM_INST_ONLY) || ALM_INST_ONLY == 1
ALM_INST(float)
#endif
#if !defined(ALM_INST_ONLY) || ALM_INST_ONLY == 2
ALM_INST(double)
#endif

}  // namespace alm
