// Rank growth along several eigenvectors (Alg. 1 of arXiv 2505.15775: the eigenvectors of
// grad_X L with negative eigenvalues, an r x r SDP over the PSD cone, R <- [R, V S^{1/2}])
// for problems whose constraints are all diagonal selectors a_i X_ii = b_k (the MaxCut form).
//
// With V (n x k, orthonormal eigenvectors of Z(w) = grad_X L for the eigenvalues lambda_a)
// and X' = X + V S V^T, L is quadratic in X, so
//   L(X') - L(X) = <diag(lambda), S> + sigma/2 ||A(V S V^T)||^2,
// and for diagonal selectors A(V S V^T)_i = a_i v_i^T S v_i (v_i the i-th row of V), so
//   ||A(V S V^T)||^2 = sum_{abcd} M_abcd S_ab S_cd,  M_abcd = sum_i a_i^2 v_ia v_ib v_ic v_id.
// The kernels here: the fourth moments M (one pass over the rows, symmetric tuples only),
// the k x k problem min_{S >= 0} <diag(lambda), S> + sigma/2 <S, M(S)> by projected gradient
// (step 1 / (sigma lambda_max(M))) in one thread, with Jacobi eigendecompositions of the
// k x k iterates for the projection and for S^{1/2}, and the append of V S^{1/2}.
#include "sparse_common.cuh"

namespace alm {

constexpr int kGrowMax = 4;    // directions per growth step
constexpr int kGrowMom = 35;   // fourth moments of 4 directions: C(4 + 3, 4)

// index of the sorted tuple a <= b <= c <= d in the moment list (k directions)
__host__ __device__ inline int mom_index(int k, int a, int b, int c, int d) {
    int t = 0;
    for (int p = 0; p < k; ++p)
        for (int q = p; q < k; ++q)
            for (int s = q; s < k; ++s)
                for (int u = s; u < k; ++u, ++t)
                    if (p == a && q == b && s == c && u == d) return t;
    return -1;
}

// M_abcd = sum_i a_i^2 v_ia v_ib v_ic v_id over the sorted tuples; V column-major n x k
template <typename T>
__global__ void __launch_bounds__(kBlock) k_grow_moments(const T *__restrict__ V, int64_t n, int k,
                                                         const int *__restrict__ sel_k,
                                                         const double *__restrict__ sel_a, DevState *st,
                                                         double *partials, double *__restrict__ mom) {
    __shared__ double shm[32];
    double acc[kGrowMom];
#pragma unroll
    for (int t = 0; t < kGrowMom; ++t) acc[t] = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        if (sel_k[i] < 0) continue;
        const double a2 = sel_a[i] * sel_a[i];
        double v[kGrowMax];
        for (int p = 0; p < k; ++p) v[p] = double(V[int64_t(p) * n + i]);
        int t = 0;
        for (int p = 0; p < k; ++p)
            for (int q = p; q < k; ++q)
                for (int s = q; s < k; ++s)
                    for (int u = s; u < k; ++u, ++t) acc[t] += a2 * v[p] * v[q] * v[s] * v[u];
    }
    int nm = 0;
    for (int p = 0; p < k; ++p)
        for (int q = p; q < k; ++q)
            for (int s = q; s < k; ++s) nm += k - s;
    double *part = partials + size_t(blockIdx.x) * kPartStride;
    for (int t = 0; t < nm; ++t) {
        const double x = block_sum(acc[t], shm);
        if (threadIdx.x == 0) part[t] = x;
    }
    if (!last_block(&st->counter[CNT_RED])) return;
    for (int t = 0; t < nm; ++t) {
        const double x = sum_partials(partials, t, shm);
        if (threadIdx.x == 0) mom[t] = x;
    }
}

// cyclic Jacobi eigendecomposition of a symmetric k x k matrix A (row-major, destroyed):
// eigenvalues on A's diagonal, eigenvectors in the columns of Q
__device__ void jacobi_eig(double *A, double *Q, int k) {
    for (int p = 0; p < k; ++p)
        for (int q = 0; q < k; ++q) Q[p * k + q] = p == q ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int p = 0; p < k; ++p)
            for (int q = 0; q < k; ++q) {
                tot += A[p * k + q] * A[p * k + q];
                if (p != q) off += A[p * k + q] * A[p * k + q];
            }
        if (off <= 1e-30 * tot || off == 0.0) return;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double apq = A[p * k + q];
                if (apq == 0.0) continue;
                // rotation that annihilates A_pq (Rutishauser's stable form)
                const double theta = (A[q * k + q] - A[p * k + p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int j = 0; j < k; ++j) {  // A <- J^T A J
                    const double x = A[p * k + j], y = A[q * k + j];
                    A[p * k + j] = c * x - s * y;
                    A[q * k + j] = s * x + c * y;
                }
                for (int j = 0; j < k; ++j) {
                    const double x = A[j * k + p], y = A[j * k + q];
                    A[j * k + p] = c * x - s * y;
                    A[j * k + q] = s * x + c * y;
                }
                for (int j = 0; j < k; ++j) {  // Q <- Q J
                    const double x = Q[j * k + p], y = Q[j * k + q];
                    Q[j * k + p] = c * x - s * y;
                    Q[j * k + q] = s * x + c * y;
                }
            }
    }
}

// B = Q diag(f(ev)) Q^T with f(x) = max(x, 0) (sqrt_mode 0) or sqrt(max(x, 0)) (sqrt_mode 1)
__device__ void psd_apply(const double *S, int k, int sqrt_mode, double *B) {
    double A[kGrowMax * kGrowMax], Q[kGrowMax * kGrowMax];
    for (int t = 0; t < k * k; ++t) A[t] = S[t];
    for (int p = 0; p < k; ++p)  // symmetrise
        for (int q = p + 1; q < k; ++q) A[p * k + q] = A[q * k + p] = 0.5 * (A[p * k + q] + A[q * k + p]);
    jacobi_eig(A, Q, k);
    for (int p = 0; p < k; ++p)
        for (int q = 0; q < k; ++q) {
            double x = 0.0;
            for (int j = 0; j < k; ++j) {
                const double ev = fmax(A[j * k + j], 0.0);
                x += Q[p * k + j] * (sqrt_mode ? sqrt(ev) : ev) * Q[q * k + j];
            }
            B[p * k + q] = x;
        }
}

// The k x k problem min_{S >= 0} f(S) = <diag(lam), S> + sigma/2 <S, M(S)>, with
// M(S)_ab = sum_cd M_abcd S_cd, by projected gradient S <- Proj_PSD(S - grad f(S) / Lip),
// Lip = sigma lambda_max of M as a k^2 x k^2 matrix (power iteration; M is PSD).  One thread.
// out: sqrtS (k x k, row-major) = S^{1/2}; info[0] = status (0 ok, 1 unbounded: M vanishes
// and some lambda < 0), info[1] = iterations; dec[0] = f(S) (the predicted decrease of L).
__global__ void k_grow_sdp(const double *__restrict__ mom, const double *__restrict__ lam, int k, double sigma,
                           int max_iter, double tol, double *__restrict__ sqrtS, int *__restrict__ info,
                           double *__restrict__ dec) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int kk = k * k;
    double H[kGrowMax * kGrowMax * kGrowMax * kGrowMax];
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b)
            for (int c = 0; c < k; ++c)
                for (int d = 0; d < k; ++d) {
                    int s[4] = {a, b, c, d};  // sort the tuple
                    for (int x = 1; x < 4; ++x)
                        for (int y = x; y > 0 && s[y - 1] > s[y]; --y) {
                            const int tmp = s[y];
                            s[y] = s[y - 1];
                            s[y - 1] = tmp;
                        }
                    H[(a * k + b) * kk + c * k + d] = mom[mom_index(k, s[0], s[1], s[2], s[3])];
                }
    // lambda_max(H) by power iteration from the all-ones vector
    double x[kGrowMax * kGrowMax], y[kGrowMax * kGrowMax];
    for (int p = 0; p < kk; ++p) x[p] = 1.0 / double(k);  // unit norm
    double lmax = 0.0;
    for (int it = 0; it < 300; ++it) {
        double nrm = 0.0;
        for (int p = 0; p < kk; ++p) {
            double t = 0.0;
            for (int q = 0; q < kk; ++q) t += H[p * kk + q] * x[q];
            y[p] = t;
            nrm += t * t;
        }
        nrm = sqrt(nrm);
        if (!(nrm > 0.0)) break;
        lmax = nrm;  // |H x| with |x| = 1
        for (int p = 0; p < kk; ++p) x[p] = y[p] / nrm;
    }
    const double Lip = sigma * lmax;
    info[0] = 0;
    info[1] = 0;
    if (!(Lip > 0.0)) {
        info[0] = 1;
        return;
    }
    double S[kGrowMax * kGrowMax], Y[kGrowMax * kGrowMax], Sn[kGrowMax * kGrowMax];
    for (int p = 0; p < kk; ++p) S[p] = 0.0;
    int it = 0;
    for (; it < max_iter; ++it) {
        for (int p = 0; p < k; ++p)
            for (int q = 0; q < k; ++q) {
                double g = p == q ? lam[p] : 0.0;
                for (int r = 0; r < kk; ++r) g += sigma * H[(p * k + q) * kk + r] * S[r];
                Y[p * k + q] = S[p * k + q] - g / Lip;
            }
        psd_apply(Y, k, 0, Sn);
        double dn = 0.0, sn = 0.0;
        for (int p = 0; p < kk; ++p) {
            dn += (Sn[p] - S[p]) * (Sn[p] - S[p]);
            sn += Sn[p] * Sn[p];
            S[p] = Sn[p];
        }
        if (sqrt(dn) <= tol * fmax(1.0, sqrt(sn))) {
            ++it;
            break;
        }
    }
    info[1] = it;
    double f = 0.0;
    for (int p = 0; p < k; ++p) f += lam[p] * S[p * k + p];
    for (int p = 0; p < kk; ++p)
        for (int q = 0; q < kk; ++q) f += 0.5 * sigma * S[p] * H[p * kk + q] * S[q];
    dec[0] = f;
    psd_apply(S, k, 1, sqrtS);
}

// dst[i, col0 + b] = sum_a V[a, i] sqrtS[a, b] (b < k): the new columns V S^{1/2}
template <typename T>
__global__ void __launch_bounds__(kBlock) k_grow_append(const T *__restrict__ V, int64_t n, int k,
                                                        const double *__restrict__ sqrtS, T *__restrict__ dst, int ld,
                                                        int col0) {
    __shared__ double s[kGrowMax * kGrowMax];
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) s[t] = sqrtS[t];
    __syncthreads();
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        double v[kGrowMax];
        for (int a = 0; a < k; ++a) v[a] = double(V[int64_t(a) * n + i]);
        for (int b = 0; b < k; ++b) {
            double x = 0.0;
            for (int a = 0; a < k; ++a) x += v[a] * s[a * k + b];
            dst[i * ld + col0 + b] = T(x);
        }
    }
}

// dst (double) <- src (working precision), n entries
template <typename T>
__global__ void __launch_bounds__(kBlock) k_to_double(const T *__restrict__ src, int64_t n, double *__restrict__ dst) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = double(src[i]);
}

// ---------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------
static int grow_grid(const LaunchCtx &c, int64_t n) {
    const int64_t need = std::max<int64_t>(1, (n + kBlock - 1) / kBlock);
    return int(std::min<int64_t>(need, c.grid));
}

template <typename T>
void launch_grow_moments(const LaunchCtx &c, const SparseView<T> &v, const T *V, int k, double *mom) {
    k_grow_moments<T><<<grow_grid(c, v.n), kBlock, 0, c.stream>>>(V, v.n, k, v.d_sel_k, v.d_sel_a, c.st, c.partials,
                                                                   mom);
    ++*c.launches;
}

void launch_grow_sdp(const LaunchCtx &c, const double *mom, const double *lam, int k, double sigma, double *sqrtS,
                     int *info, double *dec) {
    k_grow_sdp<<<1, 32, 0, c.stream>>>(mom, lam, k, sigma, 20000, 1e-13, sqrtS, info, dec);
    ++*c.launches;
}

template <typename T>
void launch_grow_append(const LaunchCtx &c, const T *V, int64_t n, int k, const double *sqrtS, T *dst, int ld,
                        int col0) {
    k_grow_append<T><<<grow_grid(c, n), kBlock, 0, c.stream>>>(V, n, k, sqrtS, dst, ld, col0);
    ++*c.launches;
}

template <typename T>
void launch_to_double(const LaunchCtx &c, const T *src, int64_t n, double *dst) {
    k_to_double<T><<<grow_grid(c, n), kBlock, 0, c.stream>>>(src, n, dst);
    ++*c.launches;
}

#define ALM_GROW_INST(T)                                                                                     \
    template void launch_grow_moments<T>(const LaunchCtx &, const SparseView<T> &, const T *, int, double *); \
    template void launch_grow_append<T>(const LaunchCtx &, const T *, int64_t, int, const double *, T *, int, int); \
    template void launch_to_double<T>(const LaunchCtx &, const T *, int64_t, double *);

ALM_GROW_INST(float)
ALM_GROW_INST(double)

}  // namespace alm
