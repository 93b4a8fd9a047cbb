// Batched persistent ALORA solver: thousands of small unit-diagonal SDPs
//     min <C_b, X_b>  s.t.  diag(X_b) = 1,  X_b >= 0      (the MaxCut SDP of Sec. 6.1)
// in ONE kernel launch.  Each CTA takes instances from a global work counter (largest
// first: the host orders the queue by decreasing work) and runs the whole of Alg. 1 for
// one instance before it takes the next:
//   inner solve of (AL-BM) at fixed y  -- preconditioned PR+ CG with the exact quartic
//                                          line search, four row passes per step
//   smallest eigenpair of S = C - Diag(w)  -- Lanczos with twice-applied classical
//                                          Gram-Schmidt, restarted from the Ritz vector
//   rank-one growth along the eigenvector, y <- w (Eq. ALM), relative KKT (Sec. 6)
// with the same arithmetic as the per-kernel path of alm_solve in its FP32 form: FP32
// rows, float-pair (compensated) diagonal terms, FP64 scalars.  Nothing waits on another
// CTA: the only inter-CTA traffic is the atomic work counter, so no wait can hang.
//
// Layout.  One row group of 8 lanes owns a row of R (8 float4 = the 32 columns of the
// fixed row stride); a CTA walks its instance's rows group by group, so a row pass is a
// sequence of coalesced 128-byte row loads and gathers.  Row data (R, the CTA's Z, D and
// Lanczos basis) is addressed through the generic path, where it stays in L1/L2 for the
// small instances this kernel is for.  Block reductions accumulate float pairs (two-sum)
// per thread and per warp and finish in FP64 across warps: FP64 units are scarce on this
// part, so no per-row work uses them in the inner loop.
#include <cfloat>
#include <cmath>

#include "batch_internal.h"
#include "dev_util.cuh"
#include "fpair.cuh"
#include "quartic.cuh"
#include "tridiag.cuh"

namespace alm {
namespace {

struct BShared {
    double red[4];
    double wpart[32 * 4];
    double sigma, tau_abs, alpha, beta, zg, zg_prev, gd, gg;
    int done, iters, status, restart, inst;
    double lz_a[kLzMax + 1], lz_b[kLzMax + 1], lz_s[kLzMax + 1], h1[kLzMax + 1], h2[kLzMax + 1];
    float h1f[kLzMax + 1], h2f[kLzMax + 1], lz_sf[kLzMax + 1];  // FP32 copies for the row loops
    double theta, resid;
};

__device__ __forceinline__ void pacc(float &h, float &l, float x) { two_sum_acc(h, l, x); }

// Sum over the CTA of NV float pairs (hi + lo); the FP64 results are in sh.red[0..NV-1]
// for every thread on return.  Contains two __syncthreads.
template <int NV>
__device__ __forceinline__ void cta_reduce(const float (&hi)[NV], const float (&lo)[NV], BShared &sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        float h = hi[k], l = lo[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, h, o);
            const float l2 = __shfl_xor_sync(0xffffffffu, l, o);
            two_sum_acc(h, l, h2);
            l += l2;
        }
        if (lane == 0) sh.wpart[warp * 4 + k] = double(h) + double(l);
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double t = lane < nw ? sh.wpart[lane * 4 + k] : 0.0;
            t = warp_sum(t);
            if (lane == 0) sh.red[k] = t;
        }
    }
    __syncthreads();
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) as a counter-based generator: element i
// of the stream `seed` (the per-kernel Lanczos start vector uses the same definition)
__device__ __forceinline__ float splitmix_uniform_pm1(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    const double u = double(z >> 11) * (1.0 / 9007199254740992.0);
    return float(2.0 * u - 1.0);
}

// sum_e val[e] X[col[e], lane's 4 columns] over the entries e0..e1 of a row (four gathers
// in flight per step)
__device__ __forceinline__ float4 gather_rows(const int32_t *__restrict__ col, const float *__restrict__ val, int e0,
                                              int e1, const float *X, int c0) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int e = e0;
    for (; e + 4 <= e1; e += 4) {
        const int j0 = col[e], j1 = col[e + 1], j2 = col[e + 2], j3 = col[e + 3];
        const float s0 = val[e], s1 = val[e + 1], s2 = val[e + 2], s3 = val[e + 3];
        const float4 x0 = ld(X + int64_t(j0) * kMaxRank + c0), x1 = ld(X + int64_t(j1) * kMaxRank + c0);
        const float4 x2 = ld(X + int64_t(j2) * kMaxRank + c0), x3 = ld(X + int64_t(j3) * kMaxRank + c0);
        acc = fma4(s0, x0, acc);
        acc = fma4(s1, x1, acc);
        acc = fma4(s2, x2, acc);
        acc = fma4(s3, x3, acc);
    }
    for (; e < e1; ++e) acc = fma4(val[e], ld(X + int64_t(col[e]) * kMaxRank + c0), acc);
    return acc;
}

// the compensated form of the same sum for the gradient (its terms cancel near a solution)
__device__ __forceinline__ void gather_rows_acc(const int32_t *__restrict__ col, const float *__restrict__ val,
                                                int e0, int e1, const float *X, int c0, AccF &acc) {
    int e = e0;
    for (; e + 4 <= e1; e += 4) {
        const int j0 = col[e], j1 = col[e + 1], j2 = col[e + 2], j3 = col[e + 3];
        const float s0 = val[e], s1 = val[e + 1], s2 = val[e + 2], s3 = val[e + 3];
        const float4 x0 = ld(X + int64_t(j0) * kMaxRank + c0), x1 = ld(X + int64_t(j1) * kMaxRank + c0);
        const float4 x2 = ld(X + int64_t(j2) * kMaxRank + c0), x3 = ld(X + int64_t(j3) * kMaxRank + c0);
        acc.add(s0, x0);
        acc.add(s1, x1);
        acc.add(s2, x2);
        acc.add(s3, x3);
    }
    for (; e < e1; ++e) acc.add(val[e], ld(X + int64_t(col[e]) * kMaxRank + c0));
}

// the GPU's global nanosecond timer (PTX special register %globaltimer)
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int BS>
__device__ void solve_instance(const BatchArgs &a, const int b, float *scr, double *scrd, BShared &sh) {
    const uint64_t t_start = global_ns();
    constexpr int L = kBatchLanes;
    constexpr int NG = BS / L;  // row groups per CTA
    constexpr int NW = BS / 32;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int gl = lane & (L - 1);
    const int grp = tid / L;
    const int c0 = gl * 4;
    const unsigned gmask = group_mask<L>(lane);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);

    const int64_t row0 = a.row_off[b];
    const int n = int(a.row_off[b + 1] - row0);
    const int32_t *rp = a.rowptr + row0;
    const int32_t *col = a.col;
    const float *val = a.val;
    float *R = a.R + row0 * kMaxRank;
    double *y = a.y + row0;
    const double *cd = a.cdiag + row0;
    const int64_t nm = a.nmax;
    float *Z = scr;
    float *D = scr + nm * kMaxRank;
    float *Q = scr + 2 * nm * kMaxRank;
    float *lzw = Q + int64_t(a.lanczos_k + 1) * nm;
    float *shi = lzw + nm, *slo = shi + nm, *bhi = slo + nm, *blo = bhi + nm;
    double *w = scrd;
    const double norm_c = a.norm_c[b];
    const float pcf = float(a.pc_floor[b]);
    const int kk = a.lanczos_k < n ? a.lanczos_k : n;
    int r = a.rank[b];
    r = r < 1 ? 1 : (r > a.r_max ? a.r_max : r);

    // columns r..31 of R and the CG buffers start at zero
    for (int t = tid; t < n * L; t += BS) {
        const int i = t / L, g = (t % L) * 4;
        stv(R + int64_t(i) * kMaxRank + g, mask_tail(ld(R + int64_t(i) * kMaxRank + g), g, r));
        stv(Z + int64_t(i) * kMaxRank + g, z4);
        stv(D + int64_t(i) * kMaxRank + g, z4);
    }
    __syncthreads();

    // ---- eval at the current R: w = y - sigma (diag(RR^T) - 1) into w, S_ii = C_ii - w_i into
    //      (shi, slo); sh.red = {|A(X) - b|^2, <C, X>, b.w}
    auto eval_dual = [&](double sigma) {
        float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
        for (int i = grp; i < n; i += NG) {
            const float4 ri = ld(R + int64_t(i) * kMaxRank + c0);
            float xh, xl;
            norm2_pair(ri, gmask, L, xh, xl);
            const float4 cr = gather_rows(col, val, rp[i], rp[i + 1], R, c0);
            pacc(h[1], l[1], dot(ri, cr));  // off-diagonal part of <C, RR^T>, lane partial
            if (gl == 0) {
                const double x = double(xh) + double(xl);
                const double res = x - 1.0;
                const double wi = y[i] - sigma * res;
                w[i] = wi;
                float ph, pl;
                split_pair(cd[i] - wi, ph, pl);
                shi[i] = ph;
                slo[i] = pl;
                pacc(h[0], l[0], float(res * res));
                split_pair(cd[i] * x, ph, pl);
                pacc(h[1], l[1], ph);
                l[1] += pl;
                split_pair(wi, ph, pl);
                pacc(h[2], l[2], ph);
                l[2] += pl;
            }
        }
        cta_reduce<3>(h, l, sh);
    };

    // ---- Lanczos on S = C - Diag(w) (diag(S) in shi + slo); result in sh.theta, the unit
    //      Ritz vector in Q[:, 0]; returns the number of S-products
    //      (warm: start from the Ritz vector left in Q[:, 0] plus a seeded perturbation of norm 0.05)
    auto lanczos = [&](uint64_t seed, double tol_abs, bool warm) -> int {
        {
            float h[1] = {0.f}, l[1] = {0.f};
            float *u = warm ? lzw : Q;
            for (int i = tid; i < n; i += BS) {
                const float x = splitmix_uniform_pm1(seed, uint64_t(i));
                u[i] = x;
                pacc(h[0], l[0], x * x);
            }
            cta_reduce<1>(h, l, sh);
            if (warm) {
                const float su = float(0.05 / sqrt(sh.red[0]));
                float h2[1] = {0.f}, l2[1] = {0.f};
                for (int i = tid; i < n; i += BS) {
                    const float x = fmaf(su, lzw[i], Q[i]);
                    Q[i] = x;
                    pacc(h2[0], l2[0], x * x);
                }
                cta_reduce<1>(h2, l2, sh);
            }
            const float sc = float(1.0 / sqrt(sh.red[0]));
            for (int i = tid; i < n; i += BS) Q[i] *= sc;
            __syncthreads();
        }
        const double tol_rel = a.lanczos_tol > 1e-5 ? a.lanczos_tol : 1e-5;  // FP32 vectors
        int matvecs = 0;
        auto proj = [&](int j, double *hout, float *hf) {  // hout[l] = q_l . w, one warp per basis vector
            for (int l = warp; l <= j; l += NW) {
                const float *ql = Q + int64_t(l) * nm;
                float h = 0.f, lo = 0.f;
                for (int i = lane; i < n; i += 32) pacc(h, lo, ql[i] * lzw[i]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float h2 = __shfl_xor_sync(0xffffffffu, h, o);
                    const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
                    two_sum_acc(h, lo, h2);
                    lo += l2;
                }
                if (lane == 0) {
                    hout[l] = double(h) + double(lo);
                    hf[l] = float(hout[l]);
                }
            }
        };
        for (int cycle = 0; cycle < a.lanczos_max_restarts; ++cycle) {
            double anorm = 0.0;
            int m = 0;
            bool stop = false;
            for (int j = 0; j < kk; ++j) {
                const float *qj = Q + int64_t(j) * nm;
                for (int i = tid; i < n; i += BS) {
                    float acc = (shi[i] + slo[i]) * qj[i];
                    const int e1 = rp[i + 1];
                    for (int e = rp[i]; e < e1; ++e) acc = fmaf(val[e], qj[col[e]], acc);
                    lzw[i] = acc;
                }
                __syncthreads();
                proj(j, sh.h1, sh.h1f);
                __syncthreads();
                for (int i = tid; i < n; i += BS) {
                    float x = lzw[i];
                    for (int l = 0; l <= j; ++l) x = fmaf(-sh.h1f[l], Q[int64_t(l) * nm + i], x);
                    lzw[i] = x;
                }
                __syncthreads();
                proj(j, sh.h2, sh.h2f);
                __syncthreads();
                float h[1] = {0.f}, lo[1] = {0.f};
                for (int i = tid; i < n; i += BS) {
                    float x = lzw[i];
                    for (int l = 0; l <= j; ++l) x = fmaf(-sh.h2f[l], Q[int64_t(l) * nm + i], x);
                    lzw[i] = x;
                    pacc(h[0], lo[0], x * x);
                }
                cta_reduce<1>(h, lo, sh);
                const double beta = sqrt(fmax(sh.red[0], 0.0));
                const double alpha = sh.h1[j] + sh.h2[j];
                const double bprev = j > 0 ? sh.lz_b[j - 1] : 0.0;
                anorm = fmax(anorm, fabs(alpha) + beta + bprev);
                __syncthreads();  // every thread has read lz_b[j - 1] and h1/h2
                if (tid == 0) {
                    sh.lz_a[j] = alpha;
                    sh.lz_b[j] = beta;
                }
                m = j + 1;
                if (!(beta > 1e-13 * anorm)) {  // invariant subspace (or non-finite)
                    stop = true;
                    __syncthreads();
                    break;
                }
                const float sc = float(1.0 / beta);
                float *qn = Q + int64_t(j + 1) * nm;
                for (int i = tid; i < n; i += BS) qn[i] = lzw[i] * sc;
                __syncthreads();
            }
            matvecs += m;
            if (warp == 0) {
                double res = 0.0;
                const double th = warp_tridiag_min(sh.lz_a, sh.lz_b, m, sh.lz_s, &res);
                __syncwarp();
                for (int l = lane; l < m; l += 32) sh.lz_sf[l] = float(sh.lz_s[l]);
                if (lane == 0) {
                    sh.theta = th;
                    sh.resid = res;
                }
            }
            __syncthreads();
            float h[1] = {0.f}, lo[1] = {0.f};
            for (int i = tid; i < n; i += BS) {
                float x = 0.f;
                for (int l = 0; l < m; ++l) x = fmaf(sh.lz_sf[l], Q[int64_t(l) * nm + i], x);
                lzw[i] = x;
                pacc(h[0], lo[0], x * x);
            }
            cta_reduce<1>(h, lo, sh);
            const float sc = float(1.0 / sqrt(sh.red[0]));
            for (int i = tid; i < n; i += BS) Q[i] = lzw[i] * sc;
            __syncthreads();
            if (!isfinite(sh.theta)) break;
            if (sh.resid <= fmax(tol_rel * anorm, tol_abs) || stop) break;
        }
        return matvecs;
    };

    double sigma = a.sigma0, tau_in = a.inner_start, kkt_prev = -1.0, p_prev = INFINITY;
    const double tau_lam = a.eps * (1.0 + norm_c);
    int status = ALM_ERR_NOT_CONVERGED, inner_total = 0, growth = 0, matvecs = 0, outer = 0;
    int fell_back = 0, restart_outer = 0;
    bool lz_before = false;  // a Lanczos ran earlier for this instance (its Ritz vector is in Q[:, 0])
    double kkt[3] = {0.0, 0.0, 0.0}, lam = 0.0, objective = 0.0;
    for (outer = 1; outer <= a.max_outer; ++outer) {
        if (!fell_back && a.fallback_inner > 0 && inner_total > a.fallback_inner) {
            // the start has cost more than the budget: restart once from a seeded cold start
            // (rows uniform on [-1, 1)^r, normalised; y = 0) with the initial sigma and tolerance
            const uint64_t cs = a.seed ^ (0xc01d57a27ULL + uint64_t(b) * 0x9e3779b97f4a7c15ULL);
            for (int i = grp; i < n; i += NG) {
                float4 u = make_float4(splitmix_uniform_pm1(cs, uint64_t(i) * kMaxRank + c0),
                                       splitmix_uniform_pm1(cs, uint64_t(i) * kMaxRank + c0 + 1),
                                       splitmix_uniform_pm1(cs, uint64_t(i) * kMaxRank + c0 + 2),
                                       splitmix_uniform_pm1(cs, uint64_t(i) * kMaxRank + c0 + 3));
                u = mask_tail(u, c0, r);
                const float nn = group_sum<L>(dot(u, u), gmask);
                stv(R + int64_t(i) * kMaxRank + c0, scale4(nn > 0.f ? rsqrtf(nn) : 0.f, u));
                if (gl == 0) y[i] = 0.0;
            }
            for (int t = tid; t < n * L; t += BS) {
                const int64_t o = int64_t(t / L) * kMaxRank + (t % L) * 4;
                stv(Z + o, z4);
                stv(D + o, z4);
            }
            __syncthreads();
            fell_back = 1;
            restart_outer = outer - 1;
            sigma = a.sigma0;
            tau_in = a.inner_start;
            kkt_prev = -1.0;
            p_prev = INFINITY;
        }
        if (outer > restart_outer + 1) {
            double cap = a.inner_decay * tau_in;
            if (kkt_prev >= 0.0) cap = fmin(cap, a.inner_rel * kkt_prev);
            tau_in = fmax(a.inner_floor * a.eps, cap);
        }
        const double tau_abs = tau_in * (1.0 + norm_c);
        const float sg = float(sigma);
        // base_i = C_ii - y_i as a float pair (y is fixed during the inner solve)
        for (int i = tid; i < n; i += BS) {
            float ph, pl;
            split_pair(cd[i] - y[i], ph, pl);
            bhi[i] = ph;
            blo[i] = pl;
        }
        if (tid == 0) {
            sh.alpha = 0.0;
            sh.done = 0;
            sh.iters = 0;
            sh.restart = 1;
            sh.zg_prev = 0.0;
            sh.status = 0;
        }
        __syncthreads();
        // ---- inner solve of (AL-BM) at fixed y ----------------------------------------
        for (;;) {
            // (1) pending step R += alpha D, then S_ii = base_i + sigma (|r_i|^2 - 1) (float pair)
            const float alpha = float(sh.alpha);
            for (int i = grp; i < n; i += NG) {
                float4 rv = ld(R + int64_t(i) * kMaxRank + c0);
                if (alpha != 0.f) {
                    rv = fma4(alpha, ld(D + int64_t(i) * kMaxRank + c0), rv);
                    stv(R + int64_t(i) * kMaxRank + c0, rv);
                }
                float xh, xl;
                norm2_pair(rv, gmask, L, xh, xl);
                if (gl == 0) {
                    // res = (xh - 1) + xl with the first difference by two-sum
                    const float s0 = xh - 1.f;
                    const float bb = s0 - xh;
                    const float e0 = (xh - (s0 - bb)) + (-1.f - bb);
                    const float res = s0 + (e0 + xl);
                    const float corr = sg * res;
                    const float dh = bhi[i];
                    const float s1 = dh + corr;
                    const float b1 = s1 - dh;
                    shi[i] = s1;
                    slo[i] = blo[i] + ((dh - (s1 - b1)) + (corr - b1));
                }
            }
            __syncthreads();
            // (2) G = 2 S R, Z = P^{-1} G (row-block Jacobi), CG inner products
            {
                float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
                for (int i = grp; i < n; i += NG) {
                    const float4 ri = ld(R + int64_t(i) * kMaxRank + c0);
                    const float dh = shi[i], dl = slo[i];
                    AccF acc;
                    acc.init();
                    acc.add(dh, ri);
                    acc.add_lo(dl, ri);
                    gather_rows_acc(col, val, rp[i], rp[i + 1], R, c0, acc);
                    const float4 g = mask_tail(scale4(2.f, acc.value()), c0, r);
                    float4 zz = g;
                    if (a.precond) {
                        const float rg = group_sum<L>(dot(ri, g), gmask), rr = group_sum<L>(dot(ri, ri), gmask);
                        float sdi = dh + dl;
                        sdi = sdi > pcf ? sdi : pcf;
                        const float ka = 4.f * sg;
                        const float coef = ka * rg / (2.f * sdi + ka * rr);
                        zz = scale4(1.f / (2.f * sdi), fma4(-coef, ri, g));
                    }
                    const float4 zo = ld(Z + int64_t(i) * kMaxRank + c0);
                    const float4 dold = ld(D + int64_t(i) * kMaxRank + c0);
                    pacc(h[0], l[0], dot(g, g));
                    pacc(h[1], l[1], dot(g, zo));
                    pacc(h[2], l[2], dot(g, dold));
                    pacc(h[3], l[3], dot(zz, g));
                    stv(Z + int64_t(i) * kMaxRank + c0, zz);
                }
                cta_reduce<4>(h, l, sh);
                if (tid == 0) {
                    const double gg = sh.red[0], go = sh.red[1], gd = sh.red[2], zg = sh.red[3];
                    sh.gg = gg;
                    if (!isfinite(gg) || !isfinite(zg)) {
                        sh.status = ALM_ERR_NUMERIC;
                        sh.done = 1;
                    } else if (sqrt(gg) <= tau_abs) {
                        sh.done = 1;
                    }
                    double beta = 0.0;
                    if (!sh.restart && a.inner_method == ALM_INNER_CG && sh.zg_prev > 0.0) {
                        beta = fmax(0.0, (zg - go) / sh.zg_prev);
                        if (-zg + beta * gd >= 0.0) beta = 0.0;  // not a descent direction: restart
                    }
                    sh.beta = beta;
                    sh.gd = gd;
                    sh.zg = zg;
                    sh.zg_prev = zg;
                    sh.restart = 0;
                }
                __syncthreads();
            }
            if (sh.done) break;
            // (3) D = -Z + beta D
            {
                const float beta = float(sh.beta);
                for (int t = tid; t < n * L; t += BS) {
                    const int64_t o = int64_t(t / L) * kMaxRank + (t % L) * 4;
                    const float4 zv = ld(Z + o);
                    const float4 dv = beta != 0.f ? ld(D + o) : z4;
                    stv(D + o, fma4(beta, dv, scale4(-1.f, zv)));
                }
                __syncthreads();
            }
            // (4) exact line search: s2 = <S, DD^T>, a1_i = 2 r_i.d_i, a2_i = |d_i|^2
            {
                float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
                for (int i = grp; i < n; i += NG) {
                    const float4 ri = ld(R + int64_t(i) * kMaxRank + c0);
                    const float4 di = ld(D + int64_t(i) * kMaxRank + c0);
                    const float4 sd = gather_rows(col, val, rp[i], rp[i + 1], D, c0);
                    const float sii = shi[i] + slo[i];
                    pacc(h[0], l[0], dot(di, fma4(sii, di, sd)));
                    const float a1 = 2.f * group_sum<L>(dot(ri, di), gmask);
                    const float a2 = group_sum<L>(dot(di, di), gmask);
                    if (gl == 0) {
                        pacc(h[1], l[1], a1 * a1);
                        pacc(h[2], l[2], a1 * a2);
                        pacc(h[3], l[3], a2 * a2);
                    }
                }
                cta_reduce<4>(h, l, sh);
                if (tid == 0) {
                    double q[5];
                    q[0] = 0.0;
                    q[1] = -sh.zg + sh.beta * sh.gd;  // <G, D> with D = -Z + beta D_old
                    q[2] = sh.red[0] + 0.5 * sigma * sh.red[1];
                    q[3] = sigma * sh.red[2];
                    q[4] = 0.5 * sigma * sh.red[3];
                    int unb = 0;
                    const double al = quartic_argmin(q, &unb);
                    bool finite = true;
                    for (int k = 1; k < 5; ++k) finite = finite && isfinite(q[k]);
                    sh.alpha = 0.0;
                    if (!finite) {
                        sh.status = ALM_ERR_NUMERIC;
                        sh.done = 1;
                    } else if (unb) {
                        sh.status = ALM_ERR_UNBOUNDED;
                        sh.done = 1;
                    } else if (!(al > 0.0)) {
                        sh.done = 1;
                    } else {
                        sh.alpha = al;
                        sh.iters += 1;
                        if (sh.iters >= a.max_inner) sh.done = 2;
                    }
                }
                __syncthreads();
            }
            if (sh.done == 1) break;
            if (sh.done == 2) {  // iteration cap: apply the last step and stop
                const float al = float(sh.alpha);
                for (int t = tid; t < n * L; t += BS) {
                    const int64_t o = int64_t(t / L) * kMaxRank + (t % L) * 4;
                    stv(R + o, fma4(al, ld(D + o), ld(R + o)));
                }
                __syncthreads();
                break;
            }
        }
        inner_total += sh.iters;
        if (sh.status != 0) {
            status = sh.status;
            break;
        }
        // ---- spectral information of grad_X L at X = RR^T --------------------------------
        eval_dual(sigma);
        double res2 = sh.red[0], c0v = sh.red[1], bw = sh.red[2];
        // lambda_min serves the rank growth (only while r < r_max) and the dual KKT term
        // (which decides only once the primal and gap terms are <= eps): skip it otherwise
        bool have_lam = r < a.r_max;
        if (!have_lam) {
            const double p0 = sqrt(fmax(res2, 0.0)) / (1.0 + sqrt(double(n)));
            const double g0 = fabs(c0v - bw) / (1.0 + fabs(c0v) + fabs(bw));
            have_lam = p0 <= a.eps && g0 <= a.eps;
        }
        if (have_lam) {
            matvecs += lanczos(a.seed + uint64_t(outer) * 0x100000001ULL + uint64_t(b) * 0x9e3779b97f4a7c15ULL,
                               0.1 * a.eps * (1.0 + norm_c), a.lanczos_warm != 0 && lz_before);
            lz_before = true;
            lam = sh.theta;
            if (!isfinite(lam)) {
                status = ALM_ERR_NUMERIC;
                break;
            }
        }
        bool grew = false;
        if (have_lam && lam < -tau_lam && r < a.r_max) {
            // ||A(v v^T)||^2 = sum_i v_i^4 for diagonal constraints
            float h[1] = {0.f}, l[1] = {0.f};
            for (int i = tid; i < n; i += BS) {
                const float v2 = Q[i] * Q[i];
                pacc(h[0], l[0], v2 * v2);
            }
            cta_reduce<1>(h, l, sh);
            const double av2 = sh.red[0];
            if (!(av2 > 0.0)) {
                status = ALM_ERR_UNBOUNDED;
                break;
            }
            const float sq = float(sqrt(-lam / (sigma * av2)));
            for (int i = tid; i < n; i += BS) R[int64_t(i) * kMaxRank + r] = sq * Q[i];
            r += 1;
            growth += 1;
            __syncthreads();
            eval_dual(sigma);
            res2 = sh.red[0];
            c0v = sh.red[1];
            bw = sh.red[2];
            grew = true;
        }
        // ---- dual update (Eq. ALM): y <- w -------------------------------------------------
        for (int i = tid; i < n; i += BS) y[i] = w[i];
        __syncthreads();
        objective = c0v;
        if (grew) continue;
        const double p = sqrt(fmax(res2, 0.0)) / (1.0 + sqrt(double(n)));
        const double d = have_lam ? fabs(fmin(0.0, lam)) / (1.0 + norm_c) : 0.0;
        const double g = fabs(c0v - bw) / (1.0 + fabs(c0v) + fabs(bw));
        kkt[0] = p;
        kkt[1] = d;
        kkt[2] = g;
        if (a.sigma_rule == ALM_SIGMA_ADAPTIVE && kkt_prev >= 0.0 && p > 0.25 * p_prev)
            sigma = fmin(2.0 * sigma, a.sigma_max);
        p_prev = p;
        kkt_prev = fmax(p, fmax(d, g));
        if (have_lam && kkt_prev <= a.eps) {
            status = ALM_OK;
            break;
        }
    }
    if (tid == 0) {
        alm_instance_stats s;
        s.status = status;
        s.outer = outer < a.max_outer ? outer : a.max_outer;
        s.inner_total = inner_total;
        s.rank = r;
        s.lanczos_matvecs = matvecs;
        s.growth_steps = growth;
        s.kkt[0] = kkt[0];
        s.kkt[1] = kkt[1];
        s.kkt[2] = kkt[2];
        s.objective = objective;
        s.lambda_min = lam;
        s.sigma = sigma;
        s.device_ms = double(global_ns() - t_start) * 1e-6;
        s.fell_back = fell_back;
        s.reserved = 0;
        a.out[b] = s;
        a.rank[b] = r;
    }
    __syncthreads();
}

template <int BS>
__global__ void __launch_bounds__(BS, 1024 / BS) k_batch_solve(const BatchArgs a) {
    __shared__ BShared sh;
    float *scr = a.scr_f + int64_t(blockIdx.x) * a.scr_f_stride;
    double *scrd = a.scr_d + int64_t(blockIdx.x) * a.scr_d_stride;
    for (;;) {
        if (threadIdx.x == 0) sh.inst = atomicAdd(a.queue, 1);
        __syncthreads();
        const int q = sh.inst;
        __syncthreads();
        if (q >= a.count) return;
        solve_instance<BS>(a, a.order[q], scr, scrd, sh);
    }
}

}  // namespace

cudaError_t launch_batch_solve(const BatchArgs &a, int threads, int grid, cudaStream_t s) {
    switch (threads) {
        case 256: k_batch_solve<256><<<grid, 256, 0, s>>>(a); break;
        case 512: k_batch_solve<512><<<grid, 512, 0, s>>>(a); break;
        case 1024: k_batch_solve<1024><<<grid, 1024, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int batch_ctas_per_sm(int threads) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (threads) {
        case 256: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_solve<256>, 256, 0); break;
        case 512: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_solve<512>, 512, 0); break;
        case 1024: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_solve<1024>, 1024, 0); break;
        default: break;
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return nb;
}

}  // namespace alm
