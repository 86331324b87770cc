// K6: far field of the single-layer representation (section 4.4):
//   a_L(theta) = sum_p sum_m c^p_m(theta) rho^p_m,
//   c^p_m(theta) = i e^{-i pi/4} sqrt(a_p) / (2 sqrt k) e^{-i k theta_hat . O_p}
//                  J_m(k a_p) e^{i m (theta - pi/2)},
// or, with J_m replaced by the row factor w_L J_m - k w_M J'_m, of the
// representation u = w_L L + w_M M (the double-layer vector a_M is
// -k J'_m / J_m times the single-layer one);
// (b_p cos(theta - alpha_p) = theta_hat . O_p).  One CTA per (configuration,
// sample angle, group of 8 columns); threads stride over the disks, the
// e^{i m (theta - pi/2)} factors come from one sincos and a complex
// recurrence, and the CTA reduces its partial sums in shared memory.
#include "msd_internal.cuh"

namespace {
constexpr int kCols = 8;
constexpr int kThreads = 128;

__global__ void k_farfield(const MsdConfig* __restrict__ cfgs, const double2* __restrict__ centre,
                           const double* __restrict__ radius, const double2* __restrict__ J, int R, int T,
                           const double* __restrict__ thetas, const double2* __restrict__ rho,
                           double2* __restrict__ F) {
    const int t = blockIdx.x, ci = blockIdx.y, r0 = blockIdx.z * kCols;
    const MsdConfig c = cfgs[ci];
    const double th = thetas[t];
    double st, ct;
    sincos(th, &st, &ct);
    double s1, c1;
    sincos(th - 0.5 * M_PI, &s1, &c1);
    const double2 e1 = make_double2(c1, s1);
    // e^{-i N (theta - pi/2)}
    double sN, cN;
    sincos(-(double)c.N * (th - 0.5 * M_PI), &sN, &cN);
    const double2 eN = make_double2(cN, sN);
    const double2 pre = cscale(cmul(make_double2(0.0, 1.0), make_double2(cos(-0.25 * M_PI), sin(-0.25 * M_PI))),
                               0.5 / sqrt(c.k));
    double2 acc[kCols];
#pragma unroll
    for (int j = 0; j < kCols; ++j) acc[j] = make_double2(0.0, 0.0);
    for (int p = threadIdx.x; p < c.M; p += blockDim.x) {
        const int d = c.disk_off + p;
        const double2 O = centre[d];
        double sp, cp;
        sincos(-c.k * (ct * O.x + st * O.y), &sp, &cp);
        const double2 ph = cscale(cmul(pre, make_double2(cp, sp)), sqrt(radius[d]));
        const long long row0 = c.row_off + (long long)p * c.n;
        double2 e = eN;
        for (int mi = 0; mi < c.n; ++mi) {
            const double2 f = cmul(cmul(ph, e), J[row0 + mi]);
            const double2* rr = rho + (row0 + mi) * R;
#pragma unroll
            for (int j = 0; j < kCols; ++j)
                if (r0 + j < R) acc[j] = cadd(acc[j], cmul(f, rr[r0 + j]));
            e = cmul(e, e1);
        }
    }
    __shared__ double2 red[kThreads];
    for (int j = 0; j < kCols && r0 + j < R; ++j) {
        red[threadIdx.x] = acc[j];
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s /= 2) {
            if (threadIdx.x < s) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + s]);
            __syncthreads();
        }
        if (threadIdx.x == 0) F[((long long)ci * T + t) * R + r0 + j] = red[0];
        __syncthreads();
    }
}
}  // namespace

void launch_farfield(const MsdConfig* d_cfg, int C, const MsdConfig*, const double2* d_centre,
                     const double* d_radius, const double2* J, int R, int T, const double* d_thetas,
                     const double2* rho, double2*, double2* F, cudaStream_t s) {
    dim3 grid(T, C, (R + kCols - 1) / kCols);
    k_farfield<<<grid, kThreads, 0, s>>>(d_cfg, d_centre, d_radius, J, R, T, d_thetas, rho, F);
    g_msd_launches += 1;
}
