// Exact minimiser of the line-search quartic phi(a) = q0 + q1 a + ... + q4 a^4 over
// a >= 0 (the closed-form step of the inner loop), in FP64.  Shared by the per-kernel
// inner loop and the batched persistent solver.
#pragma once

#include <cmath>

namespace alm {

// ---------------------------------------------------------------------------------------
// exact minimiser of the quartic phi(a) = q0 + q1 a + q2 a^2 + q3 a^3 + q4 a^4 on a >= 0
// ---------------------------------------------------------------------------------------
__device__ inline int real_cubic_roots(double c3, double c2, double c1, double c0, double x[3]) {
    // c3 x^3 + c2 x^2 + c1 x + c0 = 0, c3 != 0.  Depressed cubic t^3 + p t + q = 0 with
    // x = t - B/3 (Cardano; trigonometric form when all three roots are real).
    const double B = c2 / c3, Cc = c1 / c3, Dd = c0 / c3;
    const double p = Cc - B * B / 3.0;
    const double q = 2.0 * B * B * B / 27.0 - B * Cc / 3.0 + Dd;
    const double shift = -B / 3.0;
    const double disc = q * q / 4.0 + p * p * p / 27.0;
    int nr;
    if (disc > 0.0) {
        const double sd = sqrt(disc);
        x[0] = cbrt(-q / 2.0 + sd) + cbrt(-q / 2.0 - sd) + shift;
        nr = 1;
    } else if (p == 0.0) {
        x[0] = shift;
        nr = 1;
    } else {
        const double rr = 2.0 * sqrt(-p / 3.0);
        double arg = (3.0 * q / (2.0 * p)) * sqrt(-3.0 / p);
        arg = fmin(1.0, fmax(-1.0, arg));
        const double ph = acos(arg) / 3.0;
        const double tpi3 = 2.0943951023931954923;  // 2 pi / 3
        for (int k = 0; k < 3; ++k) x[k] = rr * cos(ph - tpi3 * k) + shift;
        nr = 3;
    }
    for (int k = 0; k < nr; ++k) {  // Newton polish on the original cubic
        double t = x[k];
        for (int it = 0; it < 4; ++it) {
            const double f = ((c3 * t + c2) * t + c1) * t + c0;
            const double fp = (3.0 * c3 * t + 2.0 * c2) * t + c1;
            if (fp == 0.0) break;
            const double nt = t - f / fp;
            if (!isfinite(nt)) break;
            t = nt;
        }
        x[k] = t;
    }
    return nr;
}

__device__ __forceinline__ double quartic_drop(const double q[5], double a) {  // phi(a) - phi(0)
    return a * (q[1] + a * (q[2] + a * (q[3] + a * q[4])));
}

__device__ inline double quartic_argmin(const double q[5], int *unbounded) {
    *unbounded = 0;
    if (q[4] < 0.0 || (q[4] == 0.0 && (q[3] < 0.0 || (q[3] == 0.0 && (q[2] < 0.0 || (q[2] == 0.0 && q[1] < 0.0)))))) {
        *unbounded = 1;
        return INFINITY;
    }
    double cand[3];
    int nc = 0;
    if (q[4] > 0.0) {
        nc = real_cubic_roots(4.0 * q[4], 3.0 * q[3], 2.0 * q[2], q[1], cand);
    } else if (q[3] > 0.0) {  // phi' = 3 q3 a^2 + 2 q2 a + q1
        const double A = 3.0 * q[3], Bq = 2.0 * q[2], Cq = q[1];
        const double disc = Bq * Bq - 4.0 * A * Cq;
        if (disc >= 0.0) {
            const double sd = sqrt(disc);
            cand[0] = (-Bq - sd) / (2.0 * A);
            cand[1] = (-Bq + sd) / (2.0 * A);
            nc = 2;
        }
    } else if (q[2] > 0.0) {
        cand[0] = -q[1] / (2.0 * q[2]);
        nc = 1;
    }
    for (int a = 0; a < nc; ++a)  // ascending: the smallest of equal minima wins
        for (int b = a + 1; b < nc; ++b)
            if (cand[b] < cand[a]) { const double t = cand[a]; cand[a] = cand[b]; cand[b] = t; }
    double best = 0.0, bestv = 0.0;
    for (int k = 0; k < nc; ++k) {
        const double a = cand[k];
        if (!(a > 0.0) || !isfinite(a)) continue;
        const double v = quartic_drop(q, a);
        if (v < bestv) { best = a; bestv = v; }
    }
    return best;
}

}  // namespace alm
