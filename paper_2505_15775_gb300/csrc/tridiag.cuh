// Smallest eigenpair of a symmetric tridiagonal matrix in FP64 (the Lanczos matrix T
// of a restart cycle), computed by one warp: multisection on the Sturm count (32 points
// per round, the bracket shrinks 33x per round), then inverse iteration on lane 0 with a
// tridiagonal solve under partial pivoting.  Shared by the per-kernel Lanczos and the
// batched persistent solver.
#pragma once

#include <cfloat>
#include <cmath>

#include "alm_internal.h"

namespace alm {

// number of eigenvalues of the tridiagonal (a, b) smaller than x (Sturm count via the
// LDL^T pivots of T - x I)
__device__ inline int sturm_count(const double *a, const double *b, int m, double x, double tiny) {
    int cnt = 0;
    double d = a[0] - x;
    if (d == 0.0) d = -tiny;
    cnt += d < 0.0;
    for (int i = 1; i < m; ++i) {
        d = a[i] - x - b[i - 1] * b[i - 1] / d;
        if (d == 0.0) d = -tiny;
        cnt += d < 0.0;
    }
    return cnt;
}

// a[0..m-1] (diagonal) and b[0..m-2] (off-diagonal; b[m-1] = the next Lanczos beta, used
// for the residual estimate) are read by every lane; 1 <= m <= kLzMax.  Every lane of the
// calling warp must call it.  Lane 0 writes the unit eigenvector to x_out[0..m-1] and the
// residual estimate |b[m-1] x[m-1]| to *resid_out; the eigenvalue is returned to all lanes.
__device__ inline double warp_tridiag_min(const double *a, const double *b, int m, double *x_out,
                                          double *resid_out) {
    const int lane = threadIdx.x & 31;
    double lo = a[0], hi = a[0];
    for (int i = 0; i < m; ++i) {
        const double rad = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < m ? fabs(b[i]) : 0.0);
        lo = fmin(lo, a[i] - rad);
        hi = fmax(hi, a[i] + rad);
    }
    const double scale = fmax(fabs(lo), fabs(hi)) + DBL_MIN;
    const double tiny = DBL_EPSILON * scale * 1e-3 + DBL_MIN;
    for (int round = 0; round < 40 && hi - lo > 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)); ++round) {
        const double step = (hi - lo) / 33.0;
        const double x = lo + step * double(lane + 1);
        const unsigned bal = __ballot_sync(0xffffffffu, sturm_count(a, b, m, x, tiny) >= 1);
        const double xlast = __shfl_sync(0xffffffffu, x, 31);
        if (bal == 0u) {
            lo = xlast;
        } else {
            const int f = __ffs(bal) - 1;
            const double xf = __shfl_sync(0xffffffffu, x, f);
            const double xp = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
            hi = xf;
            if (f > 0) lo = xp;
        }
    }
    const double theta = 0.5 * (lo + hi);  // lo and hi are warp-uniform
    if (lane != 0) return theta;
    // inverse iteration: solve (T - theta I) x = s by Gaussian elimination with partial
    // pivoting for tridiagonal systems (a second superdiagonal appears on row swaps)
    double x[kLzMax];
    for (int i = 0; i < m; ++i) x[i] = 1.0 + 0.5 * sin(double(i) + 1.0);
    for (int sweep = 0; sweep < 3; ++sweep) {
        double dl[kLzMax], dd[kLzMax], du[kLzMax], du2[kLzMax], rhs[kLzMax];
        for (int i = 0; i < m; ++i) {
            dd[i] = a[i] - theta;
            rhs[i] = x[i];
            du2[i] = 0.0;
            dl[i] = (i + 1 < m) ? b[i] : 0.0;
            du[i] = dl[i];
        }
        for (int i = 0; i + 1 < m; ++i) {
            if (fabs(dd[i]) >= fabs(dl[i])) {
                if (dd[i] == 0.0) dd[i] = tiny;
                const double f = dl[i] / dd[i];
                dd[i + 1] -= f * du[i];
                rhs[i + 1] -= f * rhs[i];
            } else {
                const double f = dd[i] / dl[i];
                dd[i] = dl[i];
                const double t = dd[i + 1];
                dd[i + 1] = du[i] - f * t;
                if (i + 2 < m) {
                    du2[i] = du[i + 1];
                    du[i + 1] = -f * du2[i];
                }
                du[i] = t;
                const double tb = rhs[i];
                rhs[i] = rhs[i + 1];
                rhs[i + 1] = tb - f * rhs[i + 1];
            }
        }
        if (dd[m - 1] == 0.0) dd[m - 1] = tiny;
        x[m - 1] = rhs[m - 1] / dd[m - 1];
        if (m >= 2) x[m - 2] = (rhs[m - 2] - du[m - 2] * x[m - 1]) / dd[m - 2];
        for (int i = m - 3; i >= 0; --i) x[i] = (rhs[i] - du[i] * x[i + 1] - du2[i] * x[i + 2]) / dd[i];
        double nx = 0.0;
        for (int i = 0; i < m; ++i) nx += x[i] * x[i];
        nx = sqrt(nx);
        if (!(nx > 0.0) || !isfinite(nx)) {
            for (int i = 0; i < m; ++i) x[i] = (i == 0);
            break;
        }
        const double inx = 1.0 / nx;
        for (int i = 0; i < m; ++i) x[i] *= inx;
    }
    for (int i = 0; i < m; ++i) x_out[i] = x[i];
    *resid_out = fabs(b[m - 1] * x[m - 1]);
    return theta;
}

}  // namespace alm
