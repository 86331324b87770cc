// Integer-order Bessel functions J_l(x), Y_l(x), l = 0..nmax, x > 0, in FP64.
//
// Methods (all published; constants below are exact rationals or pi, gamma):
//  * x <= 20: J. C. P. Miller's backward recurrence (1952) from an order
//    well above max(nmax, x), normalised with J_0 + 2 sum_{j>=1} J_{2j} = 1.
//    The same sweep accumulates the Neumann series of Abramowitz & Stegun
//    9.1.88,
//        (pi/2) Y_0 = (ln(x/2) + gamma) J_0 - 2 sum_{k>=1} (-1)^k J_{2k} / k,
//    and its derivative (Y_1 = -Y_0', J_{2k}' = (J_{2k-1} - J_{2k+1})/2),
//        (pi/2) Y_1 = (ln(x/2) + gamma) J_1 - J_0 / x
//                     + sum_{k>=1} (-1)^k (J_{2k-1} - J_{2k+1}) / k.
//  * x > 20: Hankel's asymptotic expansion (A&S 9.2.5, 9.2.6, 9.2.9,
//    9.2.10) for J_0, J_1, Y_0, Y_1, summed until the terms fall below
//    1e-18 (at x > 20 the smallest term is below e^{-40}); the phase
//    x - (nu/2 + 1/4) pi is formed from sin x and cos x so that no rounded
//    multiple of pi is subtracted from a large x.  J_l for l > 1 then comes
//    from the forward recurrence when nmax <= x, else from Miller's sweep.
//  * Y_l, l >= 2: forward recurrence Y_{l+1} = (2l/x) Y_l - Y_{l-1}
//    (Y is the dominant solution, so this direction is stable).
#pragma once

#include <math.h>

#define MSD_EULER_GAMMA 0.57721566490153286061

// Start order of the backward recurrence: past the turning point by a
// margin growing like sqrt(order), so that J_start / J_nmax is far below
// the FP64 unit roundoff.
__host__ __device__ __forceinline__ int miller_start(int nmax, double x) {
    double top = fmax((double)nmax, x);
    int s = (int)(top + sqrt(60.0 * top)) + 16;
    return s + (s & 1);  // even
}

// Miller sweep: J[0..nmax] normalised; s0, s1 = the two Neumann sums above
// (already divided by the normalisation).
__device__ inline void bessel_miller(double x, int nmax, double* J, double* s0, double* s1) {
    const int start = miller_start(nmax, x);
    const double big = 1e250, small = 1e-250;
    double jp1 = 0.0, jl = 1e-30, norm = 0.0, a0 = 0.0, a1 = 0.0;
    for (int l = start; l >= 1; --l) {
        if (l <= nmax) J[l] = jl;
        if ((l & 1) == 0) {
            const int k = l >> 1;
            norm += 2.0 * jl;
            a0 += ((k & 1) ? -jl : jl) / k;
        } else {
            const int k = (l - 1) >> 1;  // l = 2k + 1
            // coefficient of J_{2k+1} in sum_k (-1)^k (J_{2k-1} - J_{2k+1}) / k
            const double c = (k == 0) ? -1.0 : ((k & 1) ? 1.0 : -1.0) * (1.0 / (k + 1) + 1.0 / k);
            a1 += c * jl;
        }
        const double jm1 = (2.0 * l / x) * jl - jp1;
        jp1 = jl;
        jl = jm1;
        if (fabs(jl) > big) {
            jl *= small;
            jp1 *= small;
            norm *= small;
            a0 *= small;
            a1 *= small;
            for (int i = l; i <= nmax; ++i) J[i] *= small;
        }
    }
    norm += jl;  // + J_0
    J[0] = jl;
    const double inv = 1.0 / norm;
    for (int i = 0; i <= nmax; ++i) J[i] *= inv;
    *s0 = a0 * inv;
    *s1 = a1 * inv;
}

// Hankel's expansion for order nu in {0, 1}, x > 20.
__device__ inline void bessel_asymptotic(double x, int nu, double sx, double cx, double* Jn, double* Yn) {
    const double mu = 4.0 * nu * nu;
    const double z8 = 8.0 * x;
    double t = 1.0, P = 1.0, Q = 0.0;
    for (int k = 1; k < 80; ++k) {
        const double odd = 2.0 * k - 1.0;
        const double tn = t * (mu - odd * odd) / (k * z8);
        if (k > 2 && fabs(tn) > fabs(t)) break;
        t = tn;
        if (k & 1) Q += (((k - 1) >> 1) & 1) ? -t : t;
        else P += ((k >> 1) & 1) ? -t : t;
        if (fabs(t) < 1e-18) break;
    }
    const double r2 = 0.70710678118654752440;  // 1/sqrt(2)
    double cc, ss;                              // cos and sin of x - (nu/2 + 1/4) pi
    if (nu == 0) {
        cc = (cx + sx) * r2;
        ss = (sx - cx) * r2;
    } else {
        cc = (sx - cx) * r2;
        ss = -(sx + cx) * r2;
    }
    const double amp = sqrt(2.0 / (M_PI * x));
    *Jn = amp * (P * cc - Q * ss);
    *Yn = amp * (P * ss + Q * cc);
}

// J[0..nmax], Y[0..nmax] (caller arrays of length >= max(nmax, 1) + 1).
__device__ inline void bessel_jy(double x, int nmax, double* J, double* Y) {
    const int nm = nmax < 1 ? 1 : nmax;
    double Y0, Y1;
    if (x > 20.0) {
        double sx, cx;
        sincos(x, &sx, &cx);
        double J0, J1;
        bessel_asymptotic(x, 0, sx, cx, &J0, &Y0);
        bessel_asymptotic(x, 1, sx, cx, &J1, &Y1);
        if ((double)nm <= x) {
            J[0] = J0;
            J[1] = J1;
            for (int l = 1; l < nm; ++l) J[l + 1] = (2.0 * l / x) * J[l] - J[l - 1];
        } else {
            double s0, s1;
            bessel_miller(x, nm, J, &s0, &s1);
        }
    } else {
        double s0, s1;
        bessel_miller(x, nm, J, &s0, &s1);
        const double L = log(0.5 * x) + MSD_EULER_GAMMA;
        Y0 = (2.0 / M_PI) * (L * J[0] - 2.0 * s0);
        Y1 = (2.0 / M_PI) * (L * J[1] - J[0] / x + s1);
    }
    Y[0] = Y0;
    Y[1] = Y1;
    for (int l = 1; l < nm; ++l) Y[l + 1] = (2.0 * l / x) * Y[l] - Y[l - 1];
}
