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
__global__ void k_pair_generators(const MsdConfig* __restrict__ cfg, const GenBlock* __restrict__ blocks,
                                  int nblocks, long long nitems, const double2* __restrict__ centre,
                                  double2* G64, float2* G32, int* flags) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nitems) return;
    int lo = 0, hi = nblocks - 1;  // last block with item_off <= idx
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blocks[mid].item_off <= idx) lo = mid;
        else hi = mid - 1;
    }
    const GenBlock g = blocks[lo];
    const MsdConfig c = cfg[g.cfg];
    const long long li = idx - g.item_off;
    const int q = g.Q0 + (int)(li / g.Pc);
    const int p = g.P0 + (int)(li % g.Pc);
    const int N = c.N, L = c.L, lmax = 2 * N;
    const long long base = g.out_off + li * L;
    if (p >= c.M || p == q) {
        for (int l = 0; l < L; ++l) {
            if (G64) G64[base + l] = make_double2(0.0, 0.0);
            if (G32) G32[base + l] = make_float2(0.f, 0.f);
        }
        return;
    }
    const double2 Op = centre[c.disk_off + p], Oq = centre[c.disk_off + q];
    const double dx = Op.x - Oq.x, dy = Op.y - Oq.y;
    const double b = hypot(dx, dy);
    const double2 e1 = make_double2(dx / b, dy / b);
    const double x = c.k * b;
    double2 e = make_double2(1.0, 0.0);  // e^{i l alpha}
    int bad = 0;
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
            if (!(fabs(gp.x) < 3.0e38 && fabs(gp.y) < 3.0e38)) bad = 1;
            G32[base + lmax + l] = make_float2((float)gp.x, (float)gp.y);
            G32[base + lmax - l] = make_float2((float)gm.x, (float)gm.y);
        }
        e = cmul(e, e1);
    };
    if (x > 20.0 && (double)(lmax < 1 ? 1 : lmax) <= x) {
        // far pair: J and Y both by forward recurrence from Hankel's
        // expansion of orders 0 and 1 (the same steps as bessel_jy), on the fly
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
    } else {
        double J[MAXL], Y[MAXL];
        bessel_jy(x, lmax, J, Y);
        for (int l = 0; l <= lmax; ++l) put(l, J[l], Y[l]);
    }
    if (bad) atomicOr(flags, FLAG_RANGE32);
}

void launch_generator_blocks(const MsdConfig* d_cfg, const GenBlock* d_blocks, int nblocks, long long nitems,
                             const double2* d_centre, double2* G64, float2* G32, int* d_flags, cudaStream_t s) {
    if (nitems <= 0) return;
    const int threads = 128;
    const long long blocks = (nitems + threads - 1) / threads;
    k_pair_generators<<<(unsigned)blocks, threads, 0, s>>>(d_cfg, d_blocks, nblocks, nitems, d_centre, G64, G32,
                                                            d_flags);
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
