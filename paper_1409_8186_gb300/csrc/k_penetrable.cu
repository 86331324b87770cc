// Penetrable obstacles (section 7, Example II): u+ = L+ rho+ outside and
// u- = L- rho- inside the disks, single layers at the exterior wavenumber k+
// and the interior one k-, with the transmission rows
//   L+ rho+ - L- rho- = -U,   (-I/2 + N+) rho+ - mu (I/2 + N-) rho- = -dU.
// Every off-diagonal block is a diagonal times (S^pq)^T times sqrt(a_q)J^q:
//   L+-^pq = c J+-^p S+-^T J+-^q,  N+-^pq = k+- c J+-'^p S+-^T J+-^q,
// so the product needs one block-Toeplitz sum per wavenumber,
//   z+ = sum_q T(g+^pq)(sqrt(a) J+ rho+),  z- = sum_q T(g-^pq)(sqrt(a) J- rho-),
// and row (p, m) of B^-1 (off-diagonal part) is A [z+; z-] with
//   C = (i pi sqrt(a)/2) [[J+, -J-], [k+ J+', -mu k- J-']],  A = B^-1 C,
// B the 2 x 2 self block of the mode:
//   B = [[(i pi a/2) J+ H+, -(i pi a/2) J- H-],
//        [(i pi k+ a/2) J+ H+', -mu (1 + (i pi k- a/2) J- H-')]].
// The Krylov vectors of a transmission solve hold, per configuration c
// (row offset R0 = row_off_c, M n rows per density), rho+ in rows
// [2 R0, 2 R0 + M n) and rho- in rows [2 R0 + M n, 2 R0 + 2 M n).
#include <cuda_runtime.h>

#include "msd_internal.cuh"

namespace {

__device__ __forceinline__ double2 ci(double2 a) { return make_double2(-a.y, a.x); }  // i a
__device__ __forceinline__ double2 rc(double x) { return make_double2(x, 0.0); }

// Per-row factors, one thread per disk.
__global__ void k_pen_rows(const MsdConfig* __restrict__ cfg_p, const MsdConfig* __restrict__ cfg_m, int Mtot,
                           long long Ntot,
                           const int* __restrict__ disk_cfg, const double* __restrict__ radius,
                           const double* __restrict__ mu, const double2* __restrict__ Jp,
                           const double2* __restrict__ dJp, const double2* __restrict__ Hp,
                           const double2* __restrict__ dHp, const double2* __restrict__ Jm,
                           const double2* __restrict__ dJm, const double2* __restrict__ Hm,
                           const double2* __restrict__ dHm, double2* __restrict__ A64, float2* __restrict__ A32,
                           double2* __restrict__ S64, int* __restrict__ flags) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= Mtot) return;
    const int ci_ = disk_cfg[d];
    const MsdConfig c = cfg_p[ci_];
    const double kp = c.k, km = cfg_m[ci_].k;
    const double a = radius[d], sa = sqrt(a), m_ = mu[d];
    const long long row0 = c.row_off + (long long)(d - c.disk_off) * c.n;
    int bad = 0;
    for (int i = 0; i < c.n; ++i) {
        const long long row = row0 + i;
        const double jp = Jp[row].x, djp = dJp[row].x, jm = Jm[row].x, djm = dJm[row].x;
        const double2 hp = Hp[row], dhp = dHp[row], hm = Hm[row], dhm = dHm[row];
        const double2 b11 = ci(cscale(hp, 0.5 * M_PI * a * jp));
        const double2 b12 = cscale(ci(cscale(hm, 0.5 * M_PI * a * jm)), -1.0);
        const double2 b21 = ci(cscale(dhp, 0.5 * M_PI * kp * a * jp));
        const double2 b22 = cscale(cadd(rc(1.0), ci(cscale(dhm, 0.5 * M_PI * km * a * jm))), -m_);
        const double2 inv = cinv(csub(cmul(b11, b22), cmul(b12, b21)));
        // B^-1 = inv [[b22, -b12], [-b21, b11]]
        const double2 i11 = cmul(inv, b22), i12 = cscale(cmul(inv, b12), -1.0);
        const double2 i21 = cscale(cmul(inv, b21), -1.0), i22 = cmul(inv, b11);
        const double pre = 0.5 * M_PI * sa;
        const double2 c11 = ci(rc(pre * jp)), c12 = ci(rc(-pre * jm));
        const double2 c21 = ci(rc(pre * kp * djp)), c22 = ci(rc(-pre * m_ * km * djm));
        double2 A[4];
        A[0] = cadd(cmul(i11, c11), cmul(i12, c21));
        A[1] = cadd(cmul(i11, c12), cmul(i12, c22));
        A[2] = cadd(cmul(i21, c11), cmul(i22, c21));
        A[3] = cadd(cmul(i21, c12), cmul(i22, c22));
        // right-hand side: B^-1 [-U; -dU] = d * (-B^-1 [J+; k+ J+'])
        const double2 s1 = cscale(cadd(cscale(i11, jp), cscale(i12, kp * djp)), -1.0);
        const double2 s2 = cscale(cadd(cscale(i21, jp), cscale(i22, kp * djp)), -1.0);
        for (int t = 0; t < 4; ++t) {
            if (!isfinite(A[t].x) || !isfinite(A[t].y)) bad = 1;
            A64[row * 4 + t] = A[t];
            A32[row * 4 + t] = make_float2((float)A[t].x, (float)A[t].y);
        }
        if (!isfinite(s1.x) || !isfinite(s1.y) || !isfinite(s2.x) || !isfinite(s2.y)) bad = 1;
        S64[row] = s1;
        S64[Ntot + row] = s2;
    }
    if (bad) atomicOr(flags, 1);
}

// Configuration of parent row `row` (binary search on the row offsets).
__device__ __forceinline__ int cfg_of_row(const MsdConfig* __restrict__ cfg, int C, long long row) {
    int lo = 0, hi = C - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cfg[mid].row_off <= row) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Rows of the two densities of parent row `row` in the transmission layout.
__device__ __forceinline__ void pen_rows(const MsdConfig* __restrict__ cfg, int C, long long row, long long& sp,
                                         long long& sm) {
    const MsdConfig c = cfg[cfg_of_row(cfg, C, row)];
    sp = 2 * c.row_off + (row - c.row_off);
    sm = sp + (long long)c.M * c.n;
}

// xs+[row][r] = rf+[row] rho+, xs-[row][r] = rf-[row] rho- (parent layout)
template <typename V, typename S>
__global__ void k_pen_scale(const MsdConfig* __restrict__ cfg, int C, long long Ntot, int R, const S* __restrict__ rfp,
                            const S* __restrict__ rfm, const V* __restrict__ x, V* __restrict__ xsp,
                            V* __restrict__ xsm) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Ntot * R) return;
    const long long row = t / R;
    const int r = (int)(t % R);
    long long sp, sm;
    pen_rows(cfg, C, row, sp, sm);
    const V vp = x[sp * R + r], vm = x[sm * R + r];
    const S fp = rfp[row], fm = rfm[row];
    xsp[t] = V{vp.x * fp, vp.y * fp};
    xsm[t] = V{vm.x * fm, vm.y * fm};
}

template <typename V>
__device__ __forceinline__ V vmul(V a, V b) {
    return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// y = x + A [z+; z-], z+- the sums of the splits of each product
template <typename V>
__global__ void k_pen_finalize(const MsdConfig* __restrict__ cfg, int C, long long Ntot, int R,
                               const V* __restrict__ A, const V* __restrict__ x, const V* __restrict__ partp,
                               int nsp, const V* __restrict__ partm, int nsm, V* __restrict__ y) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Ntot * R) return;
    const long long row = t / R;
    const int r = (int)(t % R);
    const long long tot = Ntot * R;
    V zp{0, 0}, zm{0, 0};
    for (int k = 0; k < nsp; ++k) {
        const V v = partp[k * tot + t];
        zp.x += v.x;
        zp.y += v.y;
    }
    for (int k = 0; k < nsm; ++k) {
        const V v = partm[k * tot + t];
        zm.x += v.x;
        zm.y += v.y;
    }
    long long sp, sm;
    pen_rows(cfg, C, row, sp, sm);
    const V a0 = A[row * 4], a1 = A[row * 4 + 1], a2 = A[row * 4 + 2], a3 = A[row * 4 + 3];
    const V u = vmul(a0, zp), v = vmul(a1, zm), w = vmul(a2, zp), q = vmul(a3, zm);
    const V xp = x[sp * R + r], xm = x[sm * R + r];
    y[sp * R + r] = V{xp.x + u.x + v.x, xp.y + u.y + v.y};
    y[sm * R + r] = V{xm.x + w.x + q.x, xm.y + w.y + q.y};
}

// between the transmission layout and two parent-layout arrays
__global__ void k_pen_layout(const MsdConfig* __restrict__ cfg, int C, long long Ntot, int R, int to_pen,
                             double2* __restrict__ pen, double2* __restrict__ xp, double2* __restrict__ xm) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= Ntot * R) return;
    const long long row = t / R;
    const int r = (int)(t % R);
    long long sp, sm;
    pen_rows(cfg, C, row, sp, sm);
    if (to_pen) {
        pen[sp * R + r] = xp[t];
        pen[sm * R + r] = xm[t];
    } else {
        xp[t] = pen[sp * R + r];
        xm[t] = pen[sm * R + r];
    }
}

}  // namespace

void launch_pen_rows(const MsdConfig* cfg_p, const MsdConfig* cfg_m, int Mtot, long long Ntot, const int* disk_cfg,
                     const double* radius, const double* mu, const double2* Jp, const double2* dJp,
                     const double2* Hp, const double2* dHp, const double2* Jm, const double2* dJm,
                     const double2* Hm, const double2* dHm, double2* A64, float2* A32, double2* S64, int* flags,
                     cudaStream_t s) {
    k_pen_rows<<<(Mtot + 63) / 64, 64, 0, s>>>(cfg_p, cfg_m, Mtot, Ntot, disk_cfg, radius, mu, Jp, dJp, Hp, dHp, Jm, dJm,
                                               Hm, dHm, A64, A32, S64, flags);
    g_msd_launches += 1;
}

void launch_pen_scale(bool fp64, const MsdConfig* cfg, int C, long long Ntot, int R, const void* rfp,
                      const void* rfm, const void* x, void* xsp, void* xsm, cudaStream_t s) {
    const unsigned blocks = (unsigned)((Ntot * R + 255) / 256);
    if (fp64)
        k_pen_scale<double2, double><<<blocks, 256, 0, s>>>(cfg, C, Ntot, R, (const double*)rfp, (const double*)rfm,
                                                             (const double2*)x, (double2*)xsp, (double2*)xsm);
    else
        k_pen_scale<float2, float><<<blocks, 256, 0, s>>>(cfg, C, Ntot, R, (const float*)rfp, (const float*)rfm,
                                                           (const float2*)x, (float2*)xsp, (float2*)xsm);
    g_msd_launches += 1;
}

void launch_pen_finalize(bool fp64, const MsdConfig* cfg, int C, long long Ntot, int R, const void* A, const void* x,
                         const void* partp, int nsp, const void* partm, int nsm, void* y, cudaStream_t s) {
    const unsigned blocks = (unsigned)((Ntot * R + 255) / 256);
    if (fp64)
        k_pen_finalize<double2><<<blocks, 256, 0, s>>>(cfg, C, Ntot, R, (const double2*)A, (const double2*)x,
                                                       (const double2*)partp, nsp, (const double2*)partm, nsm,
                                                       (double2*)y);
    else
        k_pen_finalize<float2><<<blocks, 256, 0, s>>>(cfg, C, Ntot, R, (const float2*)A, (const float2*)x,
                                                      (const float2*)partp, nsp, (const float2*)partm, nsm,
                                                      (float2*)y);
    g_msd_launches += 1;
}

void launch_pen_layout(const MsdConfig* cfg, int C, long long Ntot, int R, bool to_pen, double2* pen, double2* xp,
                       double2* xm, cudaStream_t s) {
    k_pen_layout<<<(unsigned)((Ntot * R + 255) / 256), 256, 0, s>>>(cfg, C, Ntot, R, to_pen ? 1 : 0, pen, xp, xm);
    g_msd_launches += 1;
}
