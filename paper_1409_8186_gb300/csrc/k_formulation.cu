// Integral-equation formulations (sections 3, 4.2, 5): the rows of the disks
// with boundary condition c carry the linear combination
//   w_I I + w_L L + w_M M + w_N N + w_D D
// of the section 4.2 blocks, the right-hand side -(w_U U + w_dU dU), and
// the fields come from u = w_L' L dens + w_M' M dens.  Every off-diagonal
// block of every operator is a diagonal times (S^pq)^T times a diagonal,
// with the diagonals J or J' on either side:
//   L^pq = c J^p S^T J^q,  M^pq = -k c J^p S^T J'^q,
//   N^pq = k c J'^p S^T J^q,  D^pq = -k^2 c J'^p S^T J'^q,  c = i pi sqrt(a_p a_q)/2,
// so one block-Toeplitz product over 2R columns (sqrt(a) J x and
// sqrt(a) J' x, the same generators g^pq) gives z1 and z2, and row p of the
// preconditioned product is
//   y = x + l1 z1 + l2 z2,
//   l1 = (i pi sqrt(a_p)/2)(w_L J + k w_N J') / P,
//   l2 = (i pi sqrt(a_p)/2)(-k w_M J - k^2 w_D J') / P,
// with P the (diagonal) self block of the combination:
//   P = w_I + w_L (i pi a/2) J H + w_M (-1/2 - (i pi k a/2) J H')
//       + w_N (1/2 + (i pi k a/2) J H') - w_D (i pi k^2 a/2) J' H'.
// The D diagonal takes the sign of its definition (the normal derivative of
// the double-layer potential); the printed diagonal has the opposite sign.
#include <cuda_runtime.h>

#include "msd_internal.cuh"

namespace {

__device__ __forceinline__ double2 cmulr(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 ci(double2 a) { return make_double2(-a.y, a.x); }  // i a

// Per-row factors of a formulation, one thread per disk (modes in order).
__global__ void k_form_rows(const MsdConfig* __restrict__ cfg, int Mtot, const int* __restrict__ disk_cfg,
                            const double* __restrict__ radius, const int8_t* __restrict__ bc,
                            const double2* __restrict__ J, const double2* __restrict__ dJ,
                            const double2* __restrict__ H, const double2* __restrict__ dH, MsdFormulation w,
                            double2* __restrict__ l1_64, double2* __restrict__ l2_64, float2* __restrict__ l1_32,
                            float2* __restrict__ l2_32, double* __restrict__ rf2_64, float* __restrict__ rf2_32,
                            double2* __restrict__ rhs_scale, double2* __restrict__ ff, double2* __restrict__ diag,
                            int* __restrict__ flags) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= Mtot) return;
    const MsdConfig c = cfg[disk_cfg[d]];
    const double a = radius[d], k = c.k, sa = sqrt(a);
    const int cls = bc[d] == MSD_NEUMANN ? 1 : 0;
    double2 std_op[5], std_rhs[2], std_rep[2];
    const double2* op = w.op[cls];  // I, L, M, N, D
    const double2* rhs = w.rhs[cls];
    const double2* rep = w.rep;
    if (w.kind >= 0) {  // named formulation; eta = i k of this configuration unless given
        msd_standard_weights(w.kind, w.alpha, w.eta_ik ? make_double2(0.0, k) : w.eta, cls, std_op, std_rhs,
                             std_rep);
        op = std_op;
        rhs = std_rhs;
        rep = std_rep;
    }
    const double2 wU = rhs[0], wdU = rhs[1];
    const long long row0 = c.row_off + (long long)(d - c.disk_off) * c.n;
    const double hpa = 0.5 * M_PI * a, hpka = 0.5 * M_PI * k * a, hpk2a = 0.5 * M_PI * k * k * a;
    int bad = 0;
    for (int i = 0; i < c.n; ++i) {
        const long long row = row0 + i;
        const double Jm = J[row].x, dJm = dJ[row].x;
        const double2 Hm = H[row], dHm = dH[row];
        // self block of the combination
        const double2 iJH = ci(cmulr(Hm, hpa * Jm));      // (i pi a/2) J H
        const double2 iJdH = ci(cmulr(dHm, hpka * Jm));   // (i pi k a/2) J H'
        const double2 idJdH = ci(cmulr(dHm, hpk2a * dJm));  // (i pi k^2 a/2) J' H'
        double2 P = op[0];
        P = cadd(P, cmul(op[1], iJH));
        P = cadd(P, cmul(op[2], csub(make_double2(-0.5, 0.0), iJdH)));
        P = cadd(P, cmul(op[3], cadd(make_double2(0.5, 0.0), iJdH)));
        P = csub(P, cmul(op[4], idJdH));
        const double2 inv = cinv(P);
        const double pre = 0.5 * M_PI * sa;  // times i below
        const double2 c1 = cadd(cmulr(op[1], Jm), cmulr(op[3], k * dJm));
        const double2 c2 = cadd(cmulr(op[2], -k * Jm), cmulr(op[4], -k * k * dJm));
        const double2 l1 = cmul(ci(cmulr(c1, pre)), inv);
        const double2 l2 = cmul(ci(cmulr(c2, pre)), inv);
        const double2 rs = cmul(cadd(cmulr(wU, -Jm), cmulr(wdU, -k * dJm)), inv);
        if (!isfinite(l1.x) || !isfinite(l1.y) || !isfinite(l2.x) || !isfinite(l2.y) || !isfinite(rs.x) ||
            !isfinite(rs.y))
            bad = 1;
        l1_64[row] = l1;
        l2_64[row] = l2;
        l1_32[row] = make_float2((float)l1.x, (float)l1.y);
        l2_32[row] = make_float2((float)l2.x, (float)l2.y);
        rf2_64[row] = sa * dJm;
        rf2_32[row] = (float)(sa * dJm);
        rhs_scale[row] = rs;
        ff[row] = cadd(cmulr(rep[0], Jm), cmulr(rep[1], -k * dJm));
        diag[row] = P;
    }
    if (bad) atomicOr(flags, 1);
}

// xs[row][r] = rf[row] x[row][r], xs[row][R + r] = rf2[row] x[row][r]
template <typename V, typename S>
__global__ void k_form_scale(long long Ntot, int R, const S* __restrict__ rf, const S* __restrict__ rf2,
                             const V* __restrict__ x, V* __restrict__ xs) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Ntot * R) return;
    const long long row = i / R;
    const int r = (int)(i % R);
    const V v = x[i];
    const S f1 = rf[row], f2 = rf2[row];
    xs[row * 2 * R + r] = V{v.x * f1, v.y * f1};
    xs[row * 2 * R + R + r] = V{v.x * f2, v.y * f2};
}

// y = x + l1 .* sum_s part[s][.][0:R] + l2 .* sum_s part[s][.][R:2R]
template <typename V>
__global__ void k_form_finalize(long long Ntot, int R, int nsplit, const V* __restrict__ l1, const V* __restrict__ l2,
                                const V* __restrict__ x, const V* __restrict__ part, V* __restrict__ y) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Ntot * R) return;
    const long long row = i / R;
    const int r = (int)(i % R);
    const long long stride = Ntot * 2 * R;
    V s1{0, 0}, s2{0, 0};
    for (int k = 0; k < nsplit; ++k) {
        const V a = part[k * stride + row * 2 * R + r], b = part[k * stride + row * 2 * R + R + r];
        s1.x += a.x;
        s1.y += a.y;
        s2.x += b.x;
        s2.y += b.y;
    }
    const V p = l1[row], q = l2[row], v = x[i];
    y[i] = V{v.x + (p.x * s1.x - p.y * s1.y) + (q.x * s2.x - q.y * s2.y),
             v.y + (p.x * s1.y + p.y * s1.x) + (q.x * s2.y + q.y * s2.x)};
}

}  // namespace

void launch_form_rows(const MsdConfig* d_cfg, int Mtot, const int* d_disk_cfg, const double* d_radius,
                      const int8_t* d_bc, const double2* J, const double2* dJ, const double2* H, const double2* dH,
                      const MsdFormulation& w, double2* l1_64, double2* l2_64, float2* l1_32, float2* l2_32,
                      double* rf2_64, float* rf2_32, double2* rhs_scale, double2* ff, double2* diag, int* d_flags,
                      cudaStream_t s) {
    k_form_rows<<<(Mtot + 63) / 64, 64, 0, s>>>(d_cfg, Mtot, d_disk_cfg, d_radius, d_bc, J, dJ, H, dH, w, l1_64, l2_64,
                                                l1_32, l2_32, rf2_64, rf2_32, rhs_scale, ff, diag, d_flags);
    g_msd_launches += 1;
}

void launch_form_scale(bool fp64, long long Ntot, int R, const void* rf, const void* rf2, const void* x, void* xs,
                       cudaStream_t s) {
    const long long tot = Ntot * R;
    const unsigned blocks = (unsigned)((tot + 255) / 256);
    if (fp64)
        k_form_scale<double2, double><<<blocks, 256, 0, s>>>(Ntot, R, (const double*)rf, (const double*)rf2,
                                                              (const double2*)x, (double2*)xs);
    else
        k_form_scale<float2, float><<<blocks, 256, 0, s>>>(Ntot, R, (const float*)rf, (const float*)rf2,
                                                            (const float2*)x, (float2*)xs);
    g_msd_launches += 1;
}

void launch_form_finalize(bool fp64, long long Ntot, int R, int nsplit, const void* l1, const void* l2,
                          const void* x, const void* part, void* y, cudaStream_t s) {
    const long long tot = Ntot * R;
    const unsigned blocks = (unsigned)((tot + 255) / 256);
    if (fp64)
        k_form_finalize<double2><<<blocks, 256, 0, s>>>(Ntot, R, nsplit, (const double2*)l1, (const double2*)l2,
                                                        (const double2*)x, (const double2*)part, (double2*)y);
    else
        k_form_finalize<float2><<<blocks, 256, 0, s>>>(Ntot, R, nsplit, (const float2*)l1, (const float2*)l2,
                                                       (const float2*)x, (const float2*)part, (float2*)y);
    g_msd_launches += 1;
}
