// Set-up kernels of the hot path:
//   K1 disk diagonals (section 4.2: J^p, J'^p, H^p, H'^p) and the row/column
//      factors of the single-scattering-preconditioned operator (section 5);
//   K2 Toeplitz generators g^pq_l = H_l(k b_pq) e^{i l alpha_pq} of every
//      ordered pair (section 4.2, the separation matrix S^pq);
//   K5 preconditioned plane-wave right-hand sides (Prop. 4.1).
#include "bessel.cuh"
#include "msd_internal.cuh"

#define MAXL (2 * MSD_MAX_N + 2)

// Flags written by set-up kernels (bitwise OR into d_flags[0]).
#define FLAG_NONFINITE 1
#define FLAG_RANGE32 2

// ---------------------------------------------------------------- K1

// One thread per disk.  For m = -N..N (Z_{-m} = (-1)^m Z_m, Z' = (Z_{m-1} - Z_{m+1})/2):
//   J, J', H = J + iY, H' at x = k a_p;
//   rf  = sqrt(a_p) J_m                               (column factor r^p_m)
//   lf  = 1/(sqrt(a_p) H_m)           (Dirichlet)     (row factor l^p_m)
//       = J'_m/(sqrt(a_p) J_m H'_m)   (Neumann)
//   rhs = 2i/(pi a_p H_m)            (Dirichlet)     (P^-1 applied to -U / d)
//       = 2i J'_m/(pi a_p J_m H'_m)   (Neumann)
// Dividing the off-diagonal blocks of section 4.2 by the diagonal block
// (i pi a_p/2) J^p H^p (Dirichlet) or (i pi k a_p/2) J^p H'^p (Neumann)
// leaves exactly l^p_m g_{n-m} r^q_n: the J_m of Dirichlet rows cancels
// analytically instead of being divided out.
__global__ void k_disk_diagonals(const MsdConfig* __restrict__ cfg, int Mtot,
                                 const int* __restrict__ disk_cfg, const double* __restrict__ radius,
                                 const int8_t* __restrict__ bc, double2* J_, double2* dJ_, double2* H_,
                                 double2* dH_, double2* lf64, double* rf64, float2* lf32, float* rf32,
                                 double2* rhs_scale, int* flags) {
    int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= Mtot) return;
    const MsdConfig c = cfg[disk_cfg[d]];
    const int N = c.N;
    const double a = radius[d];
    const double x = c.k * a;
    double J[MSD_MAX_N + 2], Y[MSD_MAX_N + 2];
    bessel_jy(x, N + 1, J, Y);
    const double sa = sqrt(a);
    const bool neumann = bc[d] == MSD_NEUMANN;
    const long long row0 = c.row_off + (long long)(d - c.disk_off) * c.n;
    int bad = 0;
    for (int mm = -N; mm <= N; ++mm) {
        int m = mm < 0 ? -mm : mm;
        double sgn = (mm < 0 && (m & 1)) ? -1.0 : 1.0;
        double Jm = J[m], Ym = Y[m];
        double dJm, dYm;
        if (m == 0) {
            dJm = -J[1];
            dYm = -Y[1];
        } else {
            dJm = 0.5 * (J[m - 1] - J[m + 1]);
            dYm = 0.5 * (Y[m - 1] - Y[m + 1]);
        }
        // derivative of Z_{-m} = (-1)^m Z_m is (-1)^m Z'_m
        Jm *= sgn; Ym *= sgn; dJm *= sgn; dYm *= sgn;
        const double2 Hm = make_double2(Jm, Ym), dHm = make_double2(dJm, dYm);
        const long long row = row0 + (mm + N);
        J_[row] = make_double2(Jm, 0.0);
        dJ_[row] = make_double2(dJm, 0.0);
        H_[row] = Hm;
        dH_[row] = dHm;
        double2 l, rs;
        if (!neumann) {
            l = cscale(cinv(Hm), 1.0 / sa);
            rs = cscale(cinv(Hm), 2.0 / (M_PI * a));
            rs = make_double2(-rs.y, rs.x);  // * i
        } else {
            double2 q = cinv(cscale(dHm, Jm));   // 1/(J_m H'_m)
            l = cscale(q, dJm / sa);
            rs = cscale(q, 2.0 * dJm / (M_PI * a));
            rs = make_double2(-rs.y, rs.x);
        }
        if (!isfinite(l.x) || !isfinite(l.y) || !isfinite(rs.x) || !isfinite(rs.y)) bad = 1;
        lf64[row] = l;
        rf64[row] = sa * Jm;
        lf32[row] = make_float2((float)l.x, (float)l.y);
        rf32[row] = (float)(sa * Jm);
        rhs_scale[row] = rs;
    }
    if (bad) atomicOr(flags, FLAG_NONFINITE);
}

// Per-disk truncation orders (section 5): the rows of modes |m| > N_p of
// disk p get zero row and column factors and a zero right-hand-side scale,
// so they form an identity block with a zero right-hand side that no product
// couples to the other rows: the padded system has the solution of the one
// truncated at N_p on every disk, and zeros on the dropped modes.
__global__ void k_mask_rows(const MsdConfig* __restrict__ cfg, int Mtot, const int* __restrict__ disk_cfg,
                            const int* __restrict__ Np, double2* lf64, float2* lf32, double* rf64, float* rf32,
                            double2* rhs_scale) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= Mtot) return;
    const MsdConfig c = cfg[disk_cfg[d]];
    const long long row0 = c.row_off + (long long)(d - c.disk_off) * c.n;
    const int np = Np[d];
    for (int i = 0; i < c.n; ++i) {
        const int m = i - c.N;
        if (m >= -np && m <= np) continue;
        const long long row = row0 + i;
        lf64[row] = make_double2(0.0, 0.0);
        lf32[row] = make_float2(0.f, 0.f);
        rf64[row] = 0.0;
        rf32[row] = 0.f;
        rhs_scale[row] = make_double2(0.0, 0.0);
    }
}

void launch_mask_rows(const MsdConfig* d_cfg, int Mtot, const int* d_disk_cfg, const int* d_Np, double2* lf64,
                      float2* lf32, double* rf64, float* rf32, double2* rhs_scale, cudaStream_t s) {
    k_mask_rows<<<(Mtot + 127) / 128, 128, 0, s>>>(d_cfg, Mtot, d_disk_cfg, d_Np, lf64, lf32, rf64, rf32, rhs_scale);
    g_msd_launches += 1;
}

void launch_disk_diagonals(const MsdConfig* d_cfg, int Mtot, const int* d_disk_cfg,
                           const double* d_radius, const int8_t* d_bc, int /*Nmax*/,
                           double2* J, double2* dJ, double2* H, double2* dH,
                           double2* lf64, double* rf64, float2* lf32, float* rf32,
                           double2* rhs_scale, int* d_flags, cudaStream_t s) {
    int threads = 128;
    int blocks = (Mtot + threads - 1) / threads;
    k_disk_diagonals<<<blocks, threads, 0, s>>>(d_cfg, Mtot, d_disk_cfg, d_radius, d_bc, J, dJ, H,
                                                 dH, lf64, rf64, lf32, rf32, rhs_scale, d_flags);
    g_msd_launches += 1;
}

// ---------------------------------------------------------------- K2

// One thread per ordered pair (q, p) of a generator block: configuration
// g.cfg, sources q in [Q0, Q0+Qb), targets p in [P0, P0+Pc) (P0, Pc
// multiples of 32, p may reach into the padding p >= M).  Output
// out[g.out_off + ((q-Q0) Pc + (p-P0)) L + l + 2N].  The whole-problem
// array is one block per configuration (P0 = Q0 = 0, Pc = Mp, Qb = M,
// out_off = gen_off); recomputed products use blocks of a chunk.
// b_pq = O_p - O_q, e^{i alpha_pq} = b_pq/|b_pq|; for l >= 0:
// g_l = H_l(k b) e^{i l alpha}, g_{-l} = (-1)^l H_l(k b) e^{-i l alpha}.
// Padded targets (p >= M) and the diagonal p == q get zeros.
//
// Far pairs (x = k b > 20 and 2N <= x: J and Y both by forward recurrence
// from Hankel's expansion of orders 0 and 1) are done by their own thread;
// near pairs (Miller's backward sweep, ~100 FP64 steps) are collected per
// block and done afterwards by the first threads of the block, so that a
// warp of far pairs never waits on a near one.  F32: the far pairs of a
// complex64-only build use FP32 arithmetic after an FP64 phase (sin/cos of
// x and the unit vector b/|b|); relative error ~1e-6, for products that run
// in FP32 anyway.
namespace {

constexpr int kGenThreads = 128;

struct PairRef {
    GenBlock g;
    long long li;
    int q, p;
};

__device__ __forceinline__ PairRef resolve_pair(const GenBlock* __restrict__ blocks, int nblocks, long long idx) {
    int lo = 0, hi = nblocks - 1;  // last block with item_off <= idx
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blocks[mid].item_off <= idx) lo = mid;
        else hi = mid - 1;
    }
    PairRef r;
    r.g = blocks[lo];
    r.li = idx - r.g.item_off;
    r.q = r.g.Q0 + (int)(r.li / r.g.Pc);
    r.p = r.g.P0 + (int)(r.li % r.g.Pc);
    return r;
}

// Hankel's expansion in FP32 (the FP64 routine's steps), x > 20.
__device__ inline void bessel_asymptotic_f32(float x, int nu, float sx, float cx, float* Jn, float* Yn) {
    const float mu = 4.0f * nu * nu;
    const float z8 = 8.0f * x;
    float t = 1.0f, P = 1.0f, Q = 0.0f;
    for (int k = 1; k < 40; ++k) {
        const float odd = 2.0f * k - 1.0f;
        const float tn = t * (mu - odd * odd) / (k * z8);
        if (k > 2 && fabsf(tn) > fabsf(t)) break;
        t = tn;
        if (k & 1) Q += (((k - 1) >> 1) & 1) ? -t : t;
        else P += ((k >> 1) & 1) ? -t : t;
        if (fabsf(t) < 1e-9f) break;
    }
    const float r2 = 0.70710678f;
    float cc, ss;
    if (nu == 0) {
        cc = (cx + sx) * r2;
        ss = (sx - cx) * r2;
    } else {
        cc = (sx - cx) * r2;
        ss = -(sx + cx) * r2;
    }
    const float amp = sqrtf(2.0f / (3.14159265f * x));
    *Jn = amp * (P * cc - Q * ss);
    *Yn = amp * (P * ss + Q * cc);
}

template <bool F32>
__global__ void __launch_bounds__(kGenThreads)
    k_pair_generators(const MsdConfig* __restrict__ cfg, const GenBlock* __restrict__ blocks, int nblocks,
                      long long nitems, const double2* __restrict__ centre, double2* G64, float2* G32, int* flags) {
    __shared__ int near_list[kGenThreads];
    __shared__ int n_near;
    if (threadIdx.x == 0) n_near = 0;
    __syncthreads();
    int bad = 0;
    const long long idx = (long long)blockIdx.x * kGenThreads + threadIdx.x;
    if (idx < nitems) {
        const PairRef r = resolve_pair(blocks, nblocks, idx);
        const MsdConfig c = cfg[r.g.cfg];
        const int L = c.L, lmax = 2 * c.N;
        const long long base = r.g.out_off + r.li * L;
        if (r.p >= c.M || r.p == r.q) {
            for (int l = 0; l < L; ++l) {
                if (G64) G64[base + l] = make_double2(0.0, 0.0);
                if (G32) G32[base + l] = make_float2(0.f, 0.f);
            }
        } else {
            const double2 Op = centre[c.disk_off + r.p], Oq = centre[c.disk_off + r.q];
            const double dx = Op.x - Oq.x, dy = Op.y - Oq.y;
            const double b = hypot(dx, dy);
            const double x = c.k * b;
            if (!(x > 20.0 && (double)lmax <= x)) {
                near_list[atomicAdd(&n_near, 1)] = threadIdx.x;
            } else if (F32) {
                double sxd, cxd;
                sincos(x, &sxd, &cxd);
                const float xf = (float)x;
                float J0, J1, Y0, Y1;
                bessel_asymptotic_f32(xf, 0, (float)sxd, (float)cxd, &J0, &Y0);
                bessel_asymptotic_f32(xf, 1, (float)sxd, (float)cxd, &J1, &Y1);
                const float2 e1 = make_float2((float)(dx / b), (float)(dy / b));
                const float two_x = 2.0f / xf;
                float2 e = make_float2(1.f, 0.f);
                auto put = [&](int l, float Jl, float Yl) {
                    const float2 gp = make_float2(Jl * e.x - Yl * e.y, Jl * e.y + Yl * e.x);
                    float2 gm = make_float2(Jl * e.x + Yl * e.y, Yl * e.x - Jl * e.y);
                    if (l & 1) gm = make_float2(-gm.x, -gm.y);
                    G32[base + lmax + l] = gp;
                    G32[base + lmax - l] = gm;
                    e = make_float2(e.x * e1.x - e.y * e1.y, e.x * e1.y + e.y * e1.x);
                };
                put(0, J0, Y0);
                for (int l = 1; l <= lmax; ++l) {
                    put(l, J1, Y1);
                    const float f = l * two_x;
                    const float J2 = f * J1 - J0, Y2 = f * Y1 - Y0;
                    J0 = J1;
                    J1 = J2;
                    Y0 = Y1;
                    Y1 = Y2;
                }
            } else {
                const double2 e1 = make_double2(dx / b, dy / b);
                double2 e = make_double2(1.0, 0.0);  // e^{i l alpha}
                auto put = [&](int l, double Jl, double Yl) {
                    const double2 H = make_double2(Jl, Yl);
                    const double2 gp = cmul(H, e);                  // g_l
                    double2 gm = cmul(H, cconj(e));                 // H_l e^{-i l alpha}
                    if (l & 1) gm = make_double2(-gm.x, -gm.y);    // g_{-l} = (-1)^l H_l e^{-i l alpha}
                    if (G64) {
                        G64[base + lmax + l] = gp;
                        G64[base + lmax - l] = gm;
                    }
                    if (G32) {
                        G32[base + lmax + l] = make_float2((float)gp.x, (float)gp.y);
                        G32[base + lmax - l] = make_float2((float)gm.x, (float)gm.y);
                    }
                    e = cmul(e, e1);
                };
                double sx, cx, J0, J1, Y0, Y1;
                sincos(x, &sx, &cx);
                bessel_asymptotic(x, 0, sx, cx, &J0, &Y0);
                bessel_asymptotic(x, 1, sx, cx, &J1, &Y1);
                put(0, J0, Y0);
                for (int l = 1; l <= lmax; ++l) {
                    put(l, J1, Y1);
                    const double f = 2.0 * l / x;
                    const double J2 = f * J1 - J0, Y2 = f * Y1 - Y0;
                    J0 = J1;
                    J1 = J2;
                    Y0 = Y1;
                    Y1 = Y2;
                }
            }
        }
    }
    __syncthreads();
    // the near pairs of this block, one per thread, in FP64 (Miller's sweep)
    if ((int)threadIdx.x < n_near) {
        const long long nidx = (long long)blockIdx.x * kGenThreads + near_list[threadIdx.x];
        const PairRef r = resolve_pair(blocks, nblocks, nidx);
        const MsdConfig c = cfg[r.g.cfg];
        const int L = c.L, lmax = 2 * c.N;
        const long long base = r.g.out_off + r.li * L;
        const double2 Op = centre[c.disk_off + r.p], Oq = centre[c.disk_off + r.q];
        const double dx = Op.x - Oq.x, dy = Op.y - Oq.y;
        const double b = hypot(dx, dy);
        const double2 e1 = make_double2(dx / b, dy / b);
        double J[MAXL], Y[MAXL];
        bessel_jy(c.k * b, lmax, J, Y);
        double2 e = make_double2(1.0, 0.0);
        for (int l = 0; l <= lmax; ++l) {
            const double2 H = make_double2(J[l], Y[l]);
            const double2 gp = cmul(H, e);
            double2 gm = cmul(H, cconj(e));
            if (l & 1) gm = make_double2(-gm.x, -gm.y);
            if (G64) {
                G64[base + lmax + l] = gp;
                G64[base + lmax - l] = gm;
            }
            if (G32) {
                if (!(fabs(gp.x) < 3.0e38 && fabs(gp.y) < 3.0e38)) bad = 1;
                G32[base + lmax + l] = make_float2((float)gp.x, (float)gp.y);
                G32[base + lmax - l] = make_float2((float)gm.x, (float)gm.y);
            }
            e = cmul(e, e1);
        }
    }
    if (bad) atomicOr(flags, FLAG_RANGE32);
}

// ---------------------------------------------------------------- near field (Prop. 4.3)

// W[row][r] = c^p_m rho^p_m[r] with c^p_m = (i pi a_p / 2) f^p_m / sqrt(2 pi a_p):
// the weight of H_m(k r_p) e^{i m theta_p} in the potential, f = J_m(k a_p)
// for the single-layer potential, w_L J_m - k w_M J'_m for u = w_L L + w_M M
// (the double-layer term of Prop. 4.3 is -(i pi k a_p / 2) J'_m).
__global__ void k_nf_weights(const MsdConfig* __restrict__ cfg, int ci, const double* __restrict__ radius,
                             const double2* __restrict__ J, const double2* __restrict__ rho, int R,
                             double2* __restrict__ W) {
    const MsdConfig c = cfg[ci];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)c.M * c.n * R) return;
    const long long lrow = t / R;
    const int p = (int)(lrow / c.n);
    const long long row = c.row_off + lrow;
    const double a = radius[c.disk_off + p];
    const double s = 0.5 * M_PI * a / sqrt(2.0 * M_PI * a);
    const double2 cm = make_double2(-s * J[row].y, s * J[row].x);  // i s J_m
    W[row * R + (t % R)] = cmul(cm, rho[row * R + (t % R)]);
}

// u(x)[r] = sum_p sum_m W^p_m[r] H_m(k r_p) e^{i m theta_p}, x = points[t],
// for x outside every disk (points inside a disk get 0).  One thread per
// point, disks in order (the warp reads the same disk's weights together).
// Far pairs (k r > 20, N <= k r): J_m, Y_m by FP32 forward recurrence from
// Hankel's expansion after an FP64 phase; near pairs: FP64 (Miller).  The m
// sum of one disk is formed in FP32 (far) or FP64 (near) and added to FP64
// sums per point.  Columns r0 .. r0 + RC - 1 of R.
template <int RC>
__global__ void __launch_bounds__(128) k_nearfield(const MsdConfig* __restrict__ cfg, int ci,
                                                   const double2* __restrict__ centre,
                                                   const double* __restrict__ radius,
                                                   const double2* __restrict__ W, int R, int r0, int ncol,
                                                   const double2* __restrict__ pts, long long P,
                                                   double2* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P) return;
    const MsdConfig c = cfg[ci];
    const int N = c.N, n = c.n;
    const double2 x = pts[t];
    double2 u[RC];
#pragma unroll
    for (int j = 0; j < RC; ++j) u[j] = make_double2(0.0, 0.0);
    bool inside = false;
    for (int p = 0; p < c.M && !inside; ++p) {
        const double2 O = centre[c.disk_off + p];
        const double dx = x.x - O.x, dy = x.y - O.y;
        const double r = hypot(dx, dy);
        if (r <= radius[c.disk_off + p]) {
            inside = true;
            break;
        }
        const double kr = c.k * r;
        const double2* w = W + (c.row_off + (long long)p * n + N) * R + r0;  // mode m = 0
        if (kr > 20.0 && (double)(N < 1 ? 1 : N) <= kr) {
            double sxd, cxd;
            sincos(kr, &sxd, &cxd);
            const float xf = (float)kr;
            float J0, J1, Y0, Y1;
            bessel_asymptotic_f32(xf, 0, (float)sxd, (float)cxd, &J0, &Y0);
            bessel_asymptotic_f32(xf, 1, (float)sxd, (float)cxd, &J1, &Y1);
            const float2 e1 = make_float2((float)(dx / r), (float)(dy / r));
            const float two_x = 2.0f / xf;
            float2 e = make_float2(1.f, 0.f);
            float2 acc[RC];
#pragma unroll
            for (int j = 0; j < RC; ++j) {
                const double2 w0 = w[j];
                acc[j] = make_float2((float)(w0.x * J0 - w0.y * Y0), (float)(w0.x * Y0 + w0.y * J0));
            }
            for (int m = 1; m <= N; ++m) {
                e = make_float2(e.x * e1.x - e.y * e1.y, e.x * e1.y + e.y * e1.x);
                // H_m e^{i m th} and H_{-m} e^{-i m th} = (-1)^m H_m e^{-i m th}
                const float2 hp = make_float2(J1 * e.x - Y1 * e.y, J1 * e.y + Y1 * e.x);
                float2 hm = make_float2(J1 * e.x + Y1 * e.y, Y1 * e.x - J1 * e.y);
                if (m & 1) hm = make_float2(-hm.x, -hm.y);
#pragma unroll
                for (int j = 0; j < RC; ++j) {
                    if (j >= ncol) break;
                    const double2 wp = w[(long long)m * R + j], wm = w[-(long long)m * R + j];
                    const float2 a = make_float2((float)wp.x, (float)wp.y), b = make_float2((float)wm.x, (float)wm.y);
                    acc[j].x += a.x * hp.x - a.y * hp.y + b.x * hm.x - b.y * hm.y;
                    acc[j].y += a.x * hp.y + a.y * hp.x + b.x * hm.y + b.y * hm.x;
                }
                const float f = m * two_x;
                const float J2 = f * J1 - J0, Y2 = f * Y1 - Y0;
                J0 = J1;
                J1 = J2;
                Y0 = Y1;
                Y1 = Y2;
            }
#pragma unroll
            for (int j = 0; j < RC; ++j) {
                u[j].x += acc[j].x;
                u[j].y += acc[j].y;
            }
        } else {
            double J[MAXL], Y[MAXL];
            bessel_jy(kr, N, J, Y);
            const double2 e1 = make_double2(dx / r, dy / r);
            double2 e = make_double2(1.0, 0.0);
            for (int m = 0; m <= N; ++m) {
                const double2 H = make_double2(J[m], Y[m]);
                const double2 hp = cmul(H, e);
                double2 hm = cmul(H, cconj(e));
                if (m & 1) hm = make_double2(-hm.x, -hm.y);
#pragma unroll
                for (int j = 0; j < RC; ++j) {
                    if (j >= ncol) break;
                    u[j] = cadd(u[j], cmul(w[(long long)m * R + j], hp));
                    if (m > 0) u[j] = cadd(u[j], cmul(w[-(long long)m * R + j], hm));
                }
                e = cmul(e, e1);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < RC; ++j) {
        if (j >= ncol) break;
        out[t * R + r0 + j] = inside ? make_double2(0.0, 0.0) : u[j];
    }
}

// Interior field of penetrable obstacles (section 7, Example II):
// u-(x) = L- rho- at points x inside the disks, the single layers of every
// circle at the interior wavenumber k-.  For x inside disk p the own circle
// takes the interior expansion (Graf's theorem with x and y exchanged),
//   V^p_m J_m(k- r_p) e^{i m theta_p},   V^p_m = (i pi a_p/2) H_m(k- a_p) rho-^p_m / sqrt(2 pi a_p),
// the other circles the exterior one, W^q_m H_m(k- r_q) e^{i m theta_q} with
// W^q_m = (i pi a_q/2) J_m(k- a_q) rho-^q_m / sqrt(2 pi a_q).  Points outside
// every disk get 0.  One thread per point and column block, FP64.
template <int RC>
__global__ void __launch_bounds__(128) k_nearfield_inside(const MsdConfig* __restrict__ cfg, int ci, double km,
                                                          const double2* __restrict__ centre,
                                                          const double* __restrict__ radius,
                                                          const double2* __restrict__ W, const double2* __restrict__ V,
                                                          int R, int r0, int ncol, const double2* __restrict__ pts,
                                                          long long P, double2* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P) return;
    const MsdConfig c = cfg[ci];
    const int N = c.N, n = c.n;
    const double2 x = pts[t];
    int own = -1;
    for (int p = 0; p < c.M; ++p) {
        const double2 O = centre[c.disk_off + p];
        if (hypot(x.x - O.x, x.y - O.y) <= radius[c.disk_off + p]) {
            own = p;
            break;
        }
    }
    double2 u[RC];
#pragma unroll
    for (int j = 0; j < RC; ++j) u[j] = make_double2(0.0, 0.0);
    if (own >= 0) {
        for (int q = 0; q < c.M; ++q) {
            const double2 O = centre[c.disk_off + q];
            const double dx = x.x - O.x, dy = x.y - O.y;
            const double r = hypot(dx, dy);
            const double kr = km * r;
            const bool self = q == own;
            const double2* w = (self ? V : W) + (c.row_off + (long long)q * n + N) * R + r0;  // mode m = 0
            double J[MAXL], Y[MAXL];
            bessel_jy(kr > 1e-300 ? kr : 1e-300, N, J, Y);
            // angle of x - O_q (any angle at the centre: only m = 0 survives there)
            const double2 e1 = r > 0.0 ? make_double2(dx / r, dy / r) : make_double2(1.0, 0.0);
            double2 e = make_double2(1.0, 0.0);
            for (int m = 0; m <= N; ++m) {
                const double2 Z = self ? make_double2(J[m], 0.0) : make_double2(J[m], Y[m]);
                const double2 zp = cmul(Z, e);
                double2 zm = cmul(Z, cconj(e));
                if (m & 1) zm = make_double2(-zm.x, -zm.y);  // Z_{-m} = (-1)^m Z_m
#pragma unroll
                for (int j = 0; j < RC; ++j) {
                    if (j >= ncol) break;
                    u[j] = cadd(u[j], cmul(w[(long long)m * R + j], zp));
                    if (m > 0) u[j] = cadd(u[j], cmul(w[-(long long)m * R + j], zm));
                }
                e = cmul(e, e1);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < RC; ++j) {
        if (j >= ncol) break;
        out[t * R + r0 + j] = u[j];
    }
}

}  // namespace

void launch_nearfield_inside(const MsdConfig* d_cfg, int ci, const MsdConfig& h_cfg, double km, const double2* d_centre,
                             const double* d_radius, const double2* Jm, const double2* Hm, const double2* rho_minus,
                             int R, double2* W, double2* V, const double2* d_pts, long long P, double2* out,
                             cudaStream_t s) {
    const long long nw = (long long)h_cfg.M * h_cfg.n * R;
    k_nf_weights<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(d_cfg, ci, d_radius, Jm, rho_minus, R, W);
    k_nf_weights<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(d_cfg, ci, d_radius, Hm, rho_minus, R, V);
    const unsigned blocks = (unsigned)((P + 127) / 128);
    for (int r0 = 0; r0 < R; r0 += 4) {
        const int nc = R - r0 < 4 ? R - r0 : 4;
        if (nc <= 1)
            k_nearfield_inside<1><<<blocks, 128, 0, s>>>(d_cfg, ci, km, d_centre, d_radius, W, V, R, r0, nc, d_pts, P,
                                                         out);
        else
            k_nearfield_inside<4><<<blocks, 128, 0, s>>>(d_cfg, ci, km, d_centre, d_radius, W, V, R, r0, nc, d_pts, P,
                                                         out);
        g_msd_launches += 1;
    }
    g_msd_launches += 2;
}

void launch_generator_blocks(const MsdConfig* d_cfg, const GenBlock* d_blocks, int nblocks, long long nitems,
                             const double2* d_centre, double2* G64, float2* G32, int* d_flags, cudaStream_t s,
                             bool f32_math) {
    if (nitems <= 0) return;
    const long long blocks = (nitems + kGenThreads - 1) / kGenThreads;
    if (f32_math && !G64 && G32)
        k_pair_generators<true><<<(unsigned)blocks, kGenThreads, 0, s>>>(d_cfg, d_blocks, nblocks, nitems, d_centre,
                                                                         G64, G32, d_flags);
    else
        k_pair_generators<false><<<(unsigned)blocks, kGenThreads, 0, s>>>(d_cfg, d_blocks, nblocks, nitems,
                                                                          d_centre, G64, G32, d_flags);
    g_msd_launches += 1;
}

// ---------------------------------------------------------------- true residual

// Unpreconditioned norms of two vectors: the single-scattering preconditioner
// P is the diagonal of the self blocks (section 4.2), P_mm = (i pi a/2)
// J_m H_m on Dirichlet rows and (i pi k a/2) J_m H'_m on Neumann rows, so
// ||P u||^2 = sum |P_row|^2 |u_row|^2.  One CTA per row chunk; part[chunk][r]
// = (sum |P|^2 |u|^2, sum |P|^2 |v|^2) over the chunk's rows.
__global__ void k_weighted_norms(const MsdConfig* __restrict__ cfg, const RowChunk* __restrict__ chunks, int R,
                                 const double* __restrict__ radius, const int8_t* __restrict__ bc,
                                 const double2* __restrict__ J, const double2* __restrict__ H,
                                 const double2* __restrict__ dH, const double2* __restrict__ diag,
                                 const double2* __restrict__ u, const double2* __restrict__ v,
                                 double2* __restrict__ part) {
    __shared__ double su[64], sv[64];
    for (int t = threadIdx.x; t < R; t += blockDim.x) su[t] = sv[t] = 0.0;
    __syncthreads();
    const RowChunk ch = chunks[blockIdx.x];
    const MsdConfig c = cfg[ch.cfg];
    const long long tot = (ch.row1 - ch.row0) * R;
    for (long long t = threadIdx.x; t < tot; t += blockDim.x) {
        const long long row = ch.row0 + t / R;
        const int r = (int)(t % R);
        const int p = (int)((row - c.row_off) / c.n);
        const double a = radius[c.disk_off + p];
        double w2;
        if (diag) {
            w2 = cabs2(diag[row]);
        } else {
            const double2 jj = J[row];
            const double2 hh = bc[c.disk_off + p] ? dH[row] : H[row];
            const double sc = bc[c.disk_off + p] ? 0.5 * M_PI * c.k * a : 0.5 * M_PI * a;
            w2 = sc * sc * cabs2(jj) * cabs2(hh);
        }
        atomicAdd(&su[r], w2 * cabs2(u[row * R + r]));
        atomicAdd(&sv[r], w2 * cabs2(v[row * R + r]));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < R; t += blockDim.x)
        part[(long long)blockIdx.x * R + t] = make_double2(su[t], sv[t]);
}

void launch_weighted_norms(const MsdConfig* d_cfg, const RowChunk* d_chunks, int nchunk, int R,
                           const double* d_radius, const int8_t* d_bc, const double2* J, const double2* H,
                           const double2* dH, const double2* diag, const double2* u, const double2* v,
                           double2* part, cudaStream_t s) {
    k_weighted_norms<<<nchunk, 256, 0, s>>>(d_cfg, d_chunks, R, d_radius, d_bc, J, H, dH, diag, u, v, part);
    g_msd_launches += 1;
}

void launch_nearfield(const MsdConfig* d_cfg, int ci, const MsdConfig& h_cfg, const double2* d_centre,
                      const double* d_radius, const double2* J, const double2* rho, int R, double2* W,
                      const double2* d_pts, long long P, double2* out, cudaStream_t s) {
    const long long nw = (long long)h_cfg.M * h_cfg.n * R;
    k_nf_weights<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(d_cfg, ci, d_radius, J, rho, R, W);
    const unsigned blocks = (unsigned)((P + 127) / 128);
    for (int r0 = 0; r0 < R; r0 += 8) {
        const int nc = R - r0 < 8 ? R - r0 : 8;
        if (nc <= 1)
            k_nearfield<1><<<blocks, 128, 0, s>>>(d_cfg, ci, d_centre, d_radius, W, R, r0, nc, d_pts, P, out);
        else if (nc <= 4)
            k_nearfield<4><<<blocks, 128, 0, s>>>(d_cfg, ci, d_centre, d_radius, W, R, r0, nc, d_pts, P, out);
        else
            k_nearfield<8><<<blocks, 128, 0, s>>>(d_cfg, ci, d_centre, d_radius, W, R, r0, nc, d_pts, P, out);
        g_msd_launches += 1;
    }
    g_msd_launches += 1;
}

// ---------------------------------------------------------------- K5

// One thread per (disk, column r).  d^p_m = sqrt(2 pi a_p) e^{i k beta_hat . O_p}
// e^{i m (pi/2 - beta)} (Prop. 4.1); out = rhs_scale * d, i.e. P^-1(-U)
// (Dirichlet rows) or P^-1(-dU) (Neumann rows).
__global__ void k_rhs_planewave(const MsdConfig* __restrict__ cfg, int Mtot,
                                const int* __restrict__ disk_cfg, const double2* __restrict__ centre,
                                const double* __restrict__ radius, const double2* __restrict__ rhs_scale,
                                int R, const double* __restrict__ betas, double2* out) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)Mtot * R) return;
    const int d = (int)(idx / R), r = (int)(idx % R);
    const int ci = disk_cfg[d];
    const MsdConfig c = cfg[ci];
    const double beta = betas[(long long)ci * R + r];
    const double2 O = centre[d];
    const double a = radius[d];
    double sb, cb;
    sincos(beta, &sb, &cb);
    double sp, cp;
    sincos(c.k * (cb * O.x + sb * O.y), &sp, &cp);
    const double amp = sqrt(2.0 * M_PI * a);
    const long long row0 = c.row_off + (long long)(d - c.disk_off) * c.n;
    for (int mm = -c.N; mm <= c.N; ++mm) {
        double s, co;
        sincos(mm * (0.5 * M_PI - beta), &s, &co);
        const double2 dm = cscale(cmul(make_double2(cp, sp), make_double2(co, s)), amp);
        const long long row = row0 + (mm + c.N);
        out[row * R + r] = cmul(rhs_scale[row], dm);
    }
}

// Point sources (section 4.3, point-source proposition): u_inc = (i/4)
// H_0(k |x - s|).  One thread per (disk, column r) with source s = src[cfg][r]:
// d'_m = (i/4) sqrt(2 pi a_p) H_m(k b) e^{-i m phi}, (b, phi) the polar
// coordinates of s - O_p (Graf, b > a_p), H_{-m} = (-1)^m H_m; out =
// rhs_scale * d', i.e. P^-1(-U) or P^-1(-dU) as for plane waves.
__global__ void k_rhs_pointsource(const MsdConfig* __restrict__ cfg, int Mtot, const int* __restrict__ disk_cfg,
                                  const double2* __restrict__ centre, const double* __restrict__ radius,
                                  const double2* __restrict__ rhs_scale, int R, const double2* __restrict__ src,
                                  double2* out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)Mtot * R) return;
    const int d = (int)(idx / R), r = (int)(idx % R);
    const int ci = disk_cfg[d];
    const MsdConfig c = cfg[ci];
    const double2 s = src[(long long)ci * R + r];
    const double2 O = centre[d];
    const double dx = s.x - O.x, dy = s.y - O.y;
    const double b = hypot(dx, dy);
    const double2 e1 = make_double2(dx / b, dy / b);  // e^{i phi}
    double J[MAXL], Y[MAXL];
    bessel_jy(c.k * b, c.N, J, Y);
    const double amp = 0.25 * sqrt(2.0 * M_PI * radius[d]);
    const long long row0 = c.row_off + (long long)(d - c.disk_off) * c.n + c.N;  // mode 0
    double2 e = make_double2(1.0, 0.0);  // e^{i m phi}
    for (int m = 0; m <= c.N; ++m) {
        const double2 iH = make_double2(-amp * Y[m], amp * J[m]);  // (i/4) sqrt(2 pi a) H_m
        const double2 dp = cmul(iH, cconj(e));                      // m: e^{-i m phi}
        out[(row0 + m) * R + r] = cmul(rhs_scale[row0 + m], dp);
        if (m > 0) {
            double2 dm = cmul(iH, e);  // -m: (-1)^m H_m e^{+i m phi}
            if (m & 1) dm = make_double2(-dm.x, -dm.y);
            out[(row0 - m) * R + r] = cmul(rhs_scale[row0 - m], dm);
        }
        e = cmul(e, e1);
    }
}

void launch_rhs_pointsource(const MsdConfig* d_cfg, int Mtot, const int* d_disk_cfg, const double2* d_centre,
                            const double* d_radius, const double2* rhs_scale, int R, const double2* d_src,
                            double2* out, cudaStream_t s) {
    const long long n = (long long)Mtot * R;
    k_rhs_pointsource<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(d_cfg, Mtot, d_disk_cfg, d_centre, d_radius,
                                                                  rhs_scale, R, d_src, out);
    g_msd_launches += 1;
}

void launch_rhs_planewave(const MsdConfig* d_cfg, int Mtot, const int* d_disk_cfg,
                          const double2* d_centre, const double* d_radius,
                          const double2* rhs_scale, int /*Nmax*/, int R, const double* d_betas,
                          double2* out, cudaStream_t s) {
    long long n = (long long)Mtot * R;
    int threads = 128;
    long long blocks = (n + threads - 1) / threads;
    k_rhs_planewave<<<(unsigned)blocks, threads, 0, s>>>(d_cfg, Mtot, d_disk_cfg, d_centre, d_radius,
                                                          rhs_scale, R, d_betas, out);
    g_msd_launches += 1;
}
