// K7: gradient of the far-field misfit J = sum_{t,r} |F(theta_t; beta_r) - F*_{tr}|^2
// with respect to the disk centres, radii and the wavenumber, by the adjoint
// method on the blocks of section 4.2, the plane-wave coefficients of
// Prop. 4.1 and the far-field coefficients of section 4.4:
//
//   dJ = 2 Re[ w^H dC rho + lam^H (db - dA rho) ],  A^H lam = C^H w,  w = F - F*.
//
// With A = P A' (P the block-diagonal part, A' the preconditioned operator
// l .* T(g) .* r of the product kernel), lam = P^-H mu where A'^H mu = C^H w.
// Every term then reduces to quantities the product kernels already make:
//   * generator derivatives (centres, k): per ordered pair the correlation
//     c_l = sum_{n-m=l} conj(mu^_m) rho^_n  (mu^ = conj(l) .* mu, rho^ = r .* rho)
//     contracted with dg_l/db_x = (k/2)(g_{l-1} - g_{l+1}),
//     dg_l/db_y = (i k/2)(g_{l-1} + g_{l+1}),
//     dg_l/dk   = (|b|/2)(g_{l-1} e^{i alpha} - g_{l+1} e^{-i alpha});
//   * row factors f = (i pi/2) sqrt(a) left (left = J or k J'): conj(lam) df s,
//     with s the raw forward Toeplitz sums of rho^;
//   * column factors r = sqrt(a) J: conj(t) dr rho, with t the raw adjoint
//     sums of mu^;
//   * diagonal blocks, right-hand sides and far-field coefficients: per row.
// Second derivatives come from Bessel's equation Z'' = -Z'/x - (1 - m^2/x^2) Z.
#include "msd_internal.cuh"

namespace {

constexpr int kThreads = 128;

__device__ __forceinline__ double2 cexpi(double t) {
    double s, c;
    sincos(t, &s, &c);
    return make_double2(c, s);
}

// ---------------------------------------------------------------- adjoint generators

// GA[p][q][l + 2N] = conj(g^pq_{-l}) = conj(G[q][p][2N - l]) for q < M, q != p;
// zero elsewhere (padded targets and the diagonal).
template <typename V>
__global__ void k_adjoint_generators(const MsdConfig* __restrict__ cfg, int ci, const V* __restrict__ G,
                                     V* __restrict__ GA) {
    const MsdConfig c = cfg[ci];
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)c.M * c.Mp) return;
    const int p = (int)(idx / c.Mp), q = (int)(idx % c.Mp);
    const int L = c.L;
    V* dst = GA + c.gen_off + ((long long)p * c.Mp + q) * L;
    if (q >= c.M || q == p) {
        for (int l = 0; l < L; ++l) dst[l] = V{0, 0};
        return;
    }
    const V* src = G + c.gen_off + ((long long)q * c.Mp + p) * L;
    for (int l = 0; l < L; ++l) {
        const V v = src[L - 1 - l];
        dst[l] = V{v.x, -v.y};
    }
}

// ---------------------------------------------------------------- far-field pieces

// E[c][m][t] = e^{i m (theta_t - pi/2)}, m = -N..N of configuration c (rows nmax apart)
__global__ void k_ff_table(const MsdConfig* __restrict__ cfg, int C, int nmax, int T,
                           const double* __restrict__ th, double2* __restrict__ E) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)C * nmax * T) return;
    const int t = (int)(idx % T);
    const int mi = (int)((idx / T) % nmax);
    const int c = (int)(idx / ((long long)T * nmax));
    const MsdConfig g = cfg[c];
    if (mi >= g.n) return;
    const int m = mi - g.N;
    E[idx] = cexpi(m * (th[t] - 0.5 * M_PI));
}

// w = F - F*, and J_c = sum |w|^2 per configuration (atomic)
__global__ void k_misfit(int C, int T, int R, const double2* __restrict__ F, const double2* __restrict__ Ft,
                         double2* __restrict__ w, double* __restrict__ J) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)C * T * R) return;
    const double2 d = csub(F[idx], Ft[idx]);
    w[idx] = d;
    atomicAdd(&J[idx / ((long long)T * R)], cabs2(d));
}

// Adjoint right-hand side u = C^H w: one block per (disk, column); the block
// stages v_t = e^{i k theta_hat_t . O_p} w_t and each thread sums one mode.
__global__ void k_farfield_adj(const MsdConfig* __restrict__ cfg, const int* __restrict__ disk_cfg,
                               const double2* __restrict__ centre, const double* __restrict__ radius,
                               const double2* __restrict__ Jrow, int nmax, int T, int R,
                               const double* __restrict__ th, const double2* __restrict__ E,
                               const double2* __restrict__ w, double2* __restrict__ u) {
    extern __shared__ double2 v[];
    const int d = blockIdx.x, r = blockIdx.y;
    const int ci = disk_cfg[d];
    const MsdConfig c = cfg[ci];
    const double2 O = centre[d];
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        double st, ct;
        sincos(th[t], &st, &ct);
        v[t] = cmul(cexpi(c.k * (ct * O.x + st * O.y)), w[((long long)ci * T + t) * R + r]);
    }
    __syncthreads();
    // conj of i e^{-i pi/4} sqrt(a) / (2 sqrt k)
    const double2 K0c = cscale(cconj(cmul(make_double2(0.0, 1.0), cexpi(-0.25 * M_PI))),
                               sqrt(radius[d]) / (2.0 * sqrt(c.k)));
    const long long row0 = c.row_off + (long long)(d - c.disk_off) * c.n;
    const double2* Ec = E + (long long)ci * nmax * T;
    for (int mi = threadIdx.x; mi < c.n; mi += blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        const double2* Em = Ec + (long long)mi * T;
        for (int t = 0; t < T; ++t) acc = cadd(acc, cmul(cconj(Em[t]), v[t]));
        u[(row0 + mi) * R + r] = cmul(K0c, cscale(acc, Jrow[row0 + mi].x));
    }
}

// Far-field term of the gradient, w^H dC rho, per (disk, column): one block,
// threads over the sample angles.
__global__ void k_farfield_grad(const MsdConfig* __restrict__ cfg, const int* __restrict__ disk_cfg,
                                const double2* __restrict__ centre, const double* __restrict__ radius,
                                const double2* __restrict__ Jrow, const double2* __restrict__ dJrow, int nmax,
                                int T, int R, const double* __restrict__ th, const double2* __restrict__ E,
                                const double2* __restrict__ w, const double2* __restrict__ rho,
                                double* __restrict__ gO, double* __restrict__ ga, double* __restrict__ gk) {
    const int d = blockIdx.x, r = blockIdx.y;
    const int ci = disk_cfg[d];
    const MsdConfig c = cfg[ci];
    const double2 O = centre[d];
    const double a = radius[d];
    const long long row0 = c.row_off + (long long)(d - c.disk_off) * c.n;
    const double2* Ec = E + (long long)ci * nmax * T;
    const double2 K0 = cscale(cmul(make_double2(0.0, 1.0), cexpi(-0.25 * M_PI)), sqrt(a) / (2.0 * sqrt(c.k)));
    double gx = 0, gy = 0, gaa = 0, gkk = 0;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        double st, ct;
        sincos(th[t], &st, &ct);
        const double proj = ct * O.x + st * O.y;
        const double2 ph = cmul(K0, cexpi(-c.k * proj));
        double2 S1 = make_double2(0.0, 0.0), S2 = make_double2(0.0, 0.0);
        for (int mi = 0; mi < c.n; ++mi) {
            const double2 e = Ec[(long long)mi * T + t];
            const double2 rr = rho[(row0 + mi) * R + r];
            const double2 er = cmul(e, rr);
            S1 = cadd(S1, cscale(er, Jrow[row0 + mi].x));
            S2 = cadd(S2, cscale(er, dJrow[row0 + mi].x));
        }
        const double2 Fp = cmul(ph, S1);                      // sum_m C^p_m rho_m
        const double2 Fd = cmul(ph, S2);                      // same with J_m -> J'_m
        const double2 wc = cconj(w[((long long)ci * T + t) * R + r]);
        // d/dO: -i k theta_hat C;  d/da: C/(2a) + k (J' part);  d/dk: -C/(2k) - i proj C + a (J' part)
        const double2 mik = make_double2(0.0, -c.k);
        gx += 2.0 * cmul(wc, cscale(cmul(mik, Fp), ct)).x;
        gy += 2.0 * cmul(wc, cscale(cmul(mik, Fp), st)).x;
        gaa += 2.0 * cmul(wc, cadd(cscale(Fp, 0.5 / a), cscale(Fd, c.k))).x;
        const double2 Fk = cadd(cadd(cscale(Fp, -0.5 / c.k), cmul(make_double2(0.0, -proj), Fp)), cscale(Fd, a));
        gkk += 2.0 * cmul(wc, Fk).x;
    }
    __shared__ double red[4][kThreads];
    red[0][threadIdx.x] = gx;
    red[1][threadIdx.x] = gy;
    red[2][threadIdx.x] = gaa;
    red[3][threadIdx.x] = gkk;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s /= 2) {
        if (threadIdx.x < s)
            for (int j = 0; j < 4; ++j) red[j][threadIdx.x] += red[j][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&gO[2 * d], red[0][0]);
        atomicAdd(&gO[2 * d + 1], red[1][0]);
        atomicAdd(&ga[d], red[2][0]);
        atomicAdd(&gk[ci], red[3][0]);
    }
}

// ---------------------------------------------------------------- pair term

// One warp per ordered pair (q source, p target) of configuration ci, p != q:
// correlation c_l of mu^p and rho^q over all columns, contracted with the
// generator derivatives.  Adds -2 Re S_x, -2 Re S_y to the centre gradient of
// p, +2 Re S to that of q, and -2 Re S_k to the wavenumber gradient.
__global__ void k_pair_grad(const MsdConfig* __restrict__ cfg, int ci, const double2* __restrict__ centre,
                            const double2* __restrict__ G, int R, const double2* __restrict__ muh,
                            const double2* __restrict__ rhoh, double* __restrict__ gO, double* __restrict__ gk) {
    const MsdConfig c = cfg[ci];
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (long long)c.M * c.M) return;
    const int q = (int)(wid / c.M), p = (int)(wid % c.M);
    if (p == q) return;
    const int N = c.N, n = c.n, L = c.L, lmax = 2 * N;
    const double2 Op = centre[c.disk_off + p], Oq = centre[c.disk_off + q];
    const double bx = Op.x - Oq.x, by = Op.y - Oq.y;
    const double b = hypot(bx, by);
    const double2 e1 = make_double2(bx / b, by / b), em1 = cconj(e1);
    const double x = c.k * b;
    const double2* g = G + c.gen_off + ((long long)q * c.Mp + p) * L;  // g[l + 2N]
    // g_{l} for l = -2N-1 .. 2N+1 via one recurrence step at each end
    auto gval = [&](int l) -> double2 {
        if (l >= -lmax && l <= lmax) return g[l + lmax];
        if (l > 0) return csub(cscale(cmul(g[lmax + lmax], e1), 2.0 * lmax / x), cmul(g[lmax + lmax - 1], cmul(e1, e1)));
        return csub(cscale(cmul(g[0], em1), -2.0 * lmax / x), cmul(g[1], cmul(em1, em1)));
    };
    const long long rp = c.row_off + (long long)p * n, rq = c.row_off + (long long)q * n;
    double2 Sx = make_double2(0.0, 0.0), Sy = Sx, Sk = Sx;
    for (int l = -lmax + lane; l <= lmax; l += 32) {
        // c_l = sum over columns and m of conj(mu^p_m) rho^q_{m+l}
        double2 cl = make_double2(0.0, 0.0);
        const int m_lo = l < 0 ? -l : 0, m_hi = l < 0 ? n : n - l;
        for (int m = m_lo; m < m_hi; ++m) {
            const double2* mu = muh + (rp + m) * R;
            const double2* rh = rhoh + (rq + m + l) * R;
            for (int r = 0; r < R; ++r) cl = cadd(cl, cmul(cconj(mu[r]), rh[r]));
        }
        const double2 gm = gval(l - 1), gp = gval(l + 1);
        const double2 dx = cscale(csub(gm, gp), 0.5 * c.k);
        const double2 dy = cmul(make_double2(0.0, 0.5 * c.k), cadd(gm, gp));
        const double2 dk = cscale(csub(cmul(gm, e1), cmul(gp, em1)), 0.5 * b);
        Sx = cadd(Sx, cmul(dx, cl));
        Sy = cadd(Sy, cmul(dy, cl));
        Sk = cadd(Sk, cmul(dk, cl));
    }
    for (int off = 16; off > 0; off >>= 1) {
        Sx.x += __shfl_xor_sync(0xffffffffu, Sx.x, off);
        Sy.x += __shfl_xor_sync(0xffffffffu, Sy.x, off);
        Sk.x += __shfl_xor_sync(0xffffffffu, Sk.x, off);
    }
    if (lane == 0) {
        const int dp = c.disk_off + p, dq = c.disk_off + q;
        atomicAdd(&gO[2 * dp], -2.0 * Sx.x);
        atomicAdd(&gO[2 * dp + 1], -2.0 * Sy.x);
        atomicAdd(&gO[2 * dq], 2.0 * Sx.x);
        atomicAdd(&gO[2 * dq + 1], 2.0 * Sy.x);
        atomicAdd(&gk[ci], -2.0 * Sk.x);
    }
}

// ---------------------------------------------------------------- per-row terms

// One thread per disk: right-hand side, diagonal block, row factor (with the
// raw forward sums s) and column factor (with the raw adjoint sums t).
__global__ void k_grad_rows(const MsdConfig* __restrict__ cfg, int Mtot, const int* __restrict__ disk_cfg,
                            const double2* __restrict__ centre, const double* __restrict__ radius,
                            const int8_t* __restrict__ bc, const double2* __restrict__ J_, const double2* __restrict__ dJ_,
                            const double2* __restrict__ H_, const double2* __restrict__ dH_, int R,
                            const double* __restrict__ betas, const double2* __restrict__ mu,
                            const double2* __restrict__ rho, const double2* __restrict__ s,
                            const double2* __restrict__ t, double* __restrict__ gO, double* __restrict__ ga,
                            double* __restrict__ gk) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= Mtot) return;
    const int ci = disk_cfg[d];
    const MsdConfig c = cfg[ci];
    const double a = radius[d], k = c.k, sa = sqrt(a), xa = k * a;
    const double2 O = centre[d];
    const bool neu = bc[d] == MSD_NEUMANN;
    const long long row0 = c.row_off + (long long)(d - c.disk_off) * c.n;
    const double2 ipi2 = make_double2(0.0, 0.5 * M_PI);
    double gx = 0, gy = 0, gaa = 0, gkk = 0;
    for (int mi = 0; mi < c.n; ++mi) {
        const int m = mi - c.N;
        const long long row = row0 + mi;
        const double Jm = J_[row].x, dJm = dJ_[row].x;
        const double2 Hm = H_[row], dHm = dH_[row];
        const double q2 = 1.0 - (double)m * m / (xa * xa);
        const double ddJm = -dJm / xa - q2 * Jm;
        const double2 ddHm = csub(cscale(dHm, -1.0 / xa), cscale(Hm, q2));
        // row factor f = (i pi/2) sqrt(a) left and derivatives; diagonal P and derivatives
        double left, dl_a, dl_k;
        double2 P, P_a, P_k;
        if (!neu) {
            left = Jm;
            dl_a = k * dJm;
            dl_k = a * dJm;
            P = cmul(ipi2, cscale(Hm, a * Jm));
            P_a = cmul(ipi2, cadd(cscale(Hm, Jm), cscale(cadd(cscale(Hm, dJm), cscale(dHm, Jm)), a * k)));
            P_k = cmul(ipi2, cscale(cadd(cscale(Hm, dJm), cscale(dHm, Jm)), a * a));
        } else {
            left = k * dJm;
            dl_a = k * k * ddJm;
            dl_k = dJm + k * a * ddJm;
            P = cmul(ipi2, cscale(dHm, k * a * Jm));
            const double2 inner = cadd(cscale(dHm, dJm), cscale(ddHm, Jm));
            P_a = cmul(ipi2, cscale(cadd(cscale(dHm, Jm), cscale(inner, a * k)), k));
            P_k = cmul(ipi2, cscale(cadd(cscale(dHm, Jm), cscale(inner, k * a)), a));
        }
        const double2 f_a = cscale(ipi2, left / (2.0 * sa) + sa * dl_a);
        const double2 f_k = cscale(ipi2, sa * dl_k);
        // column factor r = sqrt(a) J
        const double r_a = Jm / (2.0 * sa) + sa * k * dJm;
        const double r_k = sa * a * dJm;
        const double2 Pc = cconj(P);
        for (int rr = 0; rr < R; ++rr) {
            const long long i = row * R + rr;
            const double2 lam = (Pc.x == 0.0 && Pc.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(mu[i], Pc);
            const double2 lc = cconj(lam), rh = rho[i];
            // plane-wave coefficients b = -d left, d = sqrt(2 pi a) e^{i k beta_hat.O} e^{i m (pi/2 - beta)}
            const double beta = betas[(long long)ci * R + rr];
            double sb, cb;
            sincos(beta, &sb, &cb);
            const double proj = cb * O.x + sb * O.y;
            const double2 dm = cscale(cmul(cexpi(k * proj), cexpi(m * (0.5 * M_PI - beta))), sqrt(2.0 * M_PI * a));
            const double2 bm = cscale(dm, -left);
            const double2 ikb = make_double2(0.0, k);
            const double2 db_x = cscale(cmul(ikb, bm), cb);
            const double2 db_y = cscale(cmul(ikb, bm), sb);
            const double2 db_a = cscale(cadd(cscale(dm, left / (2.0 * a)), cscale(dm, dl_a)), -1.0);
            const double2 db_k = cscale(cadd(cmul(make_double2(0.0, proj), cscale(dm, left)), cscale(dm, dl_k)), -1.0);
            gx += 2.0 * cmul(lc, db_x).x;
            gy += 2.0 * cmul(lc, db_y).x;
            gaa += 2.0 * cmul(lc, db_a).x;
            gkk += 2.0 * cmul(lc, db_k).x;
            // - lam^H (dP rho + df s) - conj(t) dr rho
            const double2 sv = s[i], tc = cconj(t[i]);
            gaa -= 2.0 * (cmul(lc, cadd(cmul(P_a, rh), cmul(f_a, sv))).x + cmul(tc, cscale(rh, r_a)).x);
            gkk -= 2.0 * (cmul(lc, cadd(cmul(P_k, rh), cmul(f_k, sv))).x + cmul(tc, cscale(rh, r_k)).x);
        }
    }
    atomicAdd(&gO[2 * d], gx);
    atomicAdd(&gO[2 * d + 1], gy);
    atomicAdd(&ga[d], gaa);
    atomicAdd(&gk[ci], gkk);
}

// mu^ = conj(l) .* mu  and  rho^ = r .* rho  (the scaled vectors of the correlation)
__global__ void k_scale_pair_inputs(long long Ntot, int R, const double2* __restrict__ lf,
                                    const double* __restrict__ rf, const double2* __restrict__ mu,
                                    const double2* __restrict__ rho, double2* __restrict__ muh,
                                    double2* __restrict__ rhoh) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Ntot * R) return;
    const long long row = i / R;
    muh[i] = cmul(cconj(lf[row]), mu[i]);
    rhoh[i] = cscale(rho[i], rf[row]);
}

__global__ void k_conj_rows(long long n, const double2* __restrict__ a, double2* __restrict__ ca,
                            float2* __restrict__ ca32) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 v = cconj(a[i]);
    ca[i] = v;
    ca32[i] = make_float2((float)v.x, (float)v.y);
}

inline unsigned blocks_for(long long n, int th) { return (unsigned)((n + th - 1) / th); }

}  // namespace

void launch_adjoint_generators_f64(const MsdConfig* d_cfg, int C, const MsdConfig* h_cfg, const double2* G,
                                   double2* GA, cudaStream_t s) {
    for (int ci = 0; ci < C; ++ci) {
        const long long n = (long long)h_cfg[ci].M * h_cfg[ci].Mp;
        k_adjoint_generators<double2><<<blocks_for(n, 128), 128, 0, s>>>(d_cfg, ci, G, GA);
    }
    g_msd_launches += C;
}

void launch_adjoint_generators_f32(const MsdConfig* d_cfg, int C, const MsdConfig* h_cfg, const float2* G,
                                   float2* GA, cudaStream_t s) {
    for (int ci = 0; ci < C; ++ci) {
        const long long n = (long long)h_cfg[ci].M * h_cfg[ci].Mp;
        k_adjoint_generators<float2><<<blocks_for(n, 128), 128, 0, s>>>(d_cfg, ci, G, GA);
    }
    g_msd_launches += C;
}

void launch_conj_rows(long long n, const double2* a, double2* ca, float2* ca32, cudaStream_t s) {
    k_conj_rows<<<blocks_for(n, 256), 256, 0, s>>>(n, a, ca, ca32);
    g_msd_launches += 1;
}

void launch_ff_table(const MsdConfig* d_cfg, int C, int nmax, int T, const double* th, double2* E, cudaStream_t s) {
    const long long n = (long long)C * nmax * T;
    k_ff_table<<<blocks_for(n, 256), 256, 0, s>>>(d_cfg, C, nmax, T, th, E);
    g_msd_launches += 1;
}

void launch_misfit(int C, int T, int R, const double2* F, const double2* Ft, double2* w, double* J, cudaStream_t s) {
    const long long n = (long long)C * T * R;
    k_misfit<<<blocks_for(n, 256), 256, 0, s>>>(C, T, R, F, Ft, w, J);
    g_msd_launches += 1;
}

void launch_farfield_adj(const MsdConfig* d_cfg, int Mtot, const int* disk_cfg, const double2* centre,
                         const double* radius, const double2* J, int nmax, int T, int R, const double* th,
                         const double2* E, const double2* w, double2* u, cudaStream_t s) {
    k_farfield_adj<<<dim3(Mtot, R), kThreads, (size_t)T * sizeof(double2), s>>>(d_cfg, disk_cfg, centre, radius, J,
                                                                              nmax, T, R, th, E, w, u);
    g_msd_launches += 1;
}

void launch_farfield_grad(const MsdConfig* d_cfg, int Mtot, const int* disk_cfg, const double2* centre,
                          const double* radius, const double2* J, const double2* dJ, int nmax, int T, int R,
                          const double* th, const double2* E, const double2* w, const double2* rho, double* gO,
                          double* ga, double* gk, cudaStream_t s) {
    k_farfield_grad<<<dim3(Mtot, R), kThreads, 0, s>>>(d_cfg, disk_cfg, centre, radius, J, dJ, nmax, T, R, th, E, w,
                                                      rho, gO, ga, gk);
    g_msd_launches += 1;
}

void launch_pair_grad(const MsdConfig* d_cfg, int C, const MsdConfig* h_cfg, const double2* centre, const double2* G,
                      int R, const double2* muh, const double2* rhoh, double* gO, double* gk, cudaStream_t s) {
    for (int ci = 0; ci < C; ++ci) {
        const long long warps = (long long)h_cfg[ci].M * h_cfg[ci].M;
        k_pair_grad<<<blocks_for(warps * 32, 256), 256, 0, s>>>(d_cfg, ci, centre, G, R, muh, rhoh, gO, gk);
    }
    g_msd_launches += C;
}

void launch_grad_rows(const MsdConfig* d_cfg, int Mtot, const int* disk_cfg, const double2* centre,
                      const double* radius, const int8_t* bc, const double2* J, const double2* dJ, const double2* H,
                      const double2* dH, int R, const double* betas, const double2* mu, const double2* rho,
                      const double2* sv, const double2* tv, double* gO, double* ga, double* gk, cudaStream_t s) {
    k_grad_rows<<<blocks_for(Mtot, 64), 64, 0, s>>>(d_cfg, Mtot, disk_cfg, centre, radius, bc, J, dJ, H, dH, R, betas,
                                                   mu, rho, sv, tv, gO, ga, gk);
    g_msd_launches += 1;
}

void launch_scale_pair_inputs(long long Ntot, int R, const double2* lf, const double* rf, const double2* mu,
                              const double2* rho, double2* muh, double2* rhoh, cudaStream_t s) {
    k_scale_pair_inputs<<<blocks_for(Ntot * R, 256), 256, 0, s>>>(Ntot, R, lf, rf, mu, rho, muh, rhoh);
    g_msd_launches += 1;
}
