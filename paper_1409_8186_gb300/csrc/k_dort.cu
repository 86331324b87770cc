// Time reversal (section 7, DORT): the time-reversal matrix T = conj(F)^T F
// of every configuration's far-field matrix F [n][n] (row i: far field at
// alpha_i + pi; column j: incidence alpha_j) and the eigenvalues of T.
//
// Eigenvalues: T is Hermitian.  Householder reflections reduce it to a
// Hermitian tridiagonal matrix (n - 2 steps; step k maps column k below the
// diagonal onto a multiple of e_1 with H = I - tau v v^H and applies
// H B H = B - v w^H - w v^H to the trailing block B, p = tau B v,
// w = p - (tau/2)(v^H p) v), all steps in one persistent cooperative launch
// with one grid barrier per step (between p and its use).  A diagonal unitary
// similarity makes the off-diagonal entries real and non-negative (their
// moduli), and the eigenvalues of that real symmetric tridiagonal matrix
// are bracketed by Sturm counts (the number of sign changes of the leading
// principal minors of the shifted matrix is the number of eigenvalues below
// the shift), one warp per eigenvalue with 32 shifts per round.  Every
// kernel runs over all configurations at once.
#include <cuda_runtime.h>

#include <algorithm>

#include "msd_internal.cuh"

namespace {

constexpr int kGramTile = 16;

// T[c][i][j] = sum_t conj(F[c][t][i]) F[c][t][j], 16 x 16 output tiles.
__global__ void __launch_bounds__(kGramTile* kGramTile)
    k_dort_gram(int n, const double2* __restrict__ F, double2* __restrict__ T) {
    __shared__ double2 Fi[kGramTile][kGramTile + 1], Fj[kGramTile][kGramTile + 1];
    const int c = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i = blockIdx.y * kGramTile + ty, j = blockIdx.x * kGramTile + tx;
    const double2* Fc = F + (long long)c * n * n;
    double2 s = make_double2(0.0, 0.0);
    for (int t0 = 0; t0 < n; t0 += kGramTile) {
        const int t = t0 + ty;
        const int ci = blockIdx.y * kGramTile + tx, cj = blockIdx.x * kGramTile + tx;
        Fi[ty][tx] = (t < n && ci < n) ? Fc[(long long)t * n + ci] : make_double2(0.0, 0.0);
        Fj[ty][tx] = (t < n && cj < n) ? Fc[(long long)t * n + cj] : make_double2(0.0, 0.0);
        __syncthreads();
#pragma unroll 4
        for (int u = 0; u < kGramTile; ++u) s = cadd(s, cmul(cconj(Fi[u][ty]), Fj[u][tx]));
        __syncthreads();
    }
    if (i < n && j < n) T[((long long)c * n + i) * n + j] = s;
}

constexpr int kTdThreads = 128;
constexpr int kTdWarps = kTdThreads / 32;  // one warp per row of the trailing block
constexpr long long kBarrierCycles = 2000000000LL;  // ~1 s at 2 GHz

__device__ double block_sum_td(double v, double* red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kTdWarps; ++w) s += red[w];
    __syncthreads();
    return s;
}

// Grid-wide barrier of a cooperative launch: the counter reaches
// gridDim.x * epoch when every CTA has arrived at barrier number epoch.
// The wait is bounded (~1 s of SM clock); on expiry *err is set, and once
// it is set no CTA waits again (the results are then invalid and the host
// reports the error).
// expire_test (msd_test_expire_waits): the first barrier waits for one CTA
// more than the grid has, with a limit of kTestWaitCycles, so that the
// expiry path runs without any fault.
constexpr long long kTestWaitCycles = 20000;

__device__ __forceinline__ void grid_barrier(unsigned* counter, unsigned epoch, int* err, int expire_test) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(counter, 1u);
        const bool test = expire_test && epoch == 1;
        const unsigned target = gridDim.x * epoch + (test ? 1u : 0u);
        const long long limit = test ? kTestWaitCycles : kBarrierCycles;
        if (!*(volatile int*)err) {
            const long long t0 = clock64();
            while (*(volatile unsigned*)counter < target) {
                if (clock64() - t0 > limit) {
                    atomicExch(err, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// B[r][j] - v_r conj(w_j) - w_r conj(v_j): one entry of H B H (8 FMAs).
__device__ __forceinline__ double2 rank2(double2 b, double2 vr, double2 wr, double2 wj, double2 vj) {
    double re = fma(-wr.y, vj.y, b.x);
    re = fma(-wr.x, vj.x, re);
    re = fma(-vr.y, wj.y, re);
    re = fma(-vr.x, wj.x, re);
    double im = fma(wr.x, vj.y, b.y);
    im = fma(-wr.y, vj.x, im);
    im = fma(vr.x, wj.y, im);
    im = fma(-vr.y, wj.x, im);
    return make_double2(re, im);
}

constexpr int kTdBatch = 8;  // row entries per lane whose loads are issued together

// Householder tridiagonalisation of C Hermitian matrices A [C][n][n] in
// place, one persistent cooperative launch, one grid barrier per step.
// Row R of every matrix belongs to warp R mod (4 gridDim.x) for all steps.
// Every CTA holds x_k = A[k+1:, k] (the column the reflector of step k
// maps onto a multiple of e_1) in shared memory and derives v, tau from it
// itself.  Step k, per configuration:
//   1. p_r = tau (B v)_r for the warp's rows of B = A[k+1:, k+1:]
//      (written to pbuf[k & 1]);  grid barrier;
//   2. every CTA reads all of p, forms w = p - (tau/2)(v^H p) v, applies
//      B <- B - v w^H - w v^H to its own rows (writing the new A[R][k+2] to
//      colbuf[k & 1] as well) and computes x_{k+1} = (new B)[1:, 0] from
//      the column written one step earlier and v, w.
// pbuf and colbuf alternate between steps, so that a buffer is rewritten
// only after every CTA has passed the barrier that follows its last read.
// e_k = sigma_k = ||x_k|| goes to e_all; the diagonal entries are final in
// A once their step is done.  Dynamic shared memory: x for two steps of
// every configuration, w, and tau and ||x_k||^2 per configuration.
__global__ void __launch_bounds__(kTdThreads)
    k_dort_tridiag(int C, int n, double2* __restrict__ Aall, double2* __restrict__ pbuf,
                   double2* __restrict__ colbuf, double* __restrict__ e_all, double* __restrict__ tau_all,
                   double2* __restrict__ ph_all, unsigned* __restrict__ bar, int* __restrict__ err, int expire_test) {
    extern __shared__ double2 td_sh[];
    double2* xs = td_sh;                    // [2][C][n]
    double2* w_sh = td_sh + 2 * (size_t)C * n;  // [n]
    double* tau_sh = (double*)(w_sh + n);   // [C]
    double* nrm_sh = tau_sh + C;            // [C] ||x_k||^2
    __shared__ double red[kTdWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kTdWarps + warp, GW = gridDim.x * kTdWarps;
    auto X = [&](int par, int c) { return xs + ((size_t)par * C + c) * n; };
    // x_0 = A[1:, 0]; the column 1 below row 1 (needed by step 0) in X(1, c)
    for (int c = 0; c < C; ++c) {
        const double2* A = Aall + (long long)c * n * n;
        double nrm2 = 0.0;
        for (int r = threadIdx.x; r < n - 1; r += kTdThreads) {
            const double2 a = A[(long long)(1 + r) * n];
            X(0, c)[r] = a;
            nrm2 += cabs2(a);
        }
        for (int r = threadIdx.x; r < n - 2; r += kTdThreads) X(1, c)[r] = A[(long long)(2 + r) * n + 1];
        nrm2 = block_sum_td(nrm2, red);
        if (threadIdx.x == 0) nrm_sh[c] = nrm2;
    }
    __syncthreads();
    unsigned epoch = 0;
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1, par = k & 1;
        const int R0 = k + 1 + ((gw - (k + 1)) % GW + GW) % GW;  // first own row >= k+1
        for (int c = 0; c < C; ++c) {
            double2* x = X(par, c);
            const double sigma = sqrt(nrm_sh[c]);
            const double2 x0 = x[0];
            const double ax0 = sqrt(cabs2(x0));
            // v = x + e^{i arg x0} sigma e_1 maps x onto -e^{i arg x0} sigma e_1;
            // ||v||^2 = 2 sigma (sigma + |x0|), tau = 2 / ||v||^2
            const double tau = sigma > 0.0 ? 1.0 / (sigma * (sigma + ax0)) : 0.0;
            __syncthreads();  // every thread has read x[0]
            if (threadIdx.x == 0) {
                if (sigma > 0.0) {
                    const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
                    x[0] = cadd(x0, cscale(ph, sigma));  // x now holds v
                }
                tau_sh[c] = tau;
                if (blockIdx.x == 0) {
                    // the reflector of this step, for eigenvectors: tau, the phase of
                    // x0 (the new sub-diagonal entry is -phase sigma); v goes to row k
                    e_all[(long long)c * n + k] = sigma;
                    tau_all[(long long)c * n + k] = tau;
                    ph_all[(long long)c * n + k] =
                        ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
                }
            }
            __syncthreads();
            const double2* A = Aall + (long long)c * n * n;
            for (int R = R0; R < n; R += GW) {
                const double2* row = A + (long long)R * n + (k + 1);
                double2 s = make_double2(0.0, 0.0);
                for (int j0 = lane; j0 < m; j0 += 32 * kTdBatch) {
                    double2 a[kTdBatch];
#pragma unroll
                    for (int u = 0; u < kTdBatch; ++u) {
                        const int j = j0 + 32 * u;
                        a[u] = j < m ? row[j] : make_double2(0.0, 0.0);
                    }
#pragma unroll
                    for (int u = 0; u < kTdBatch; ++u) {
                        const int j = j0 + 32 * u;
                        if (j < m) cfma(s, a[u], x[j]);
                    }
                }
                for (int off = 16; off > 0; off >>= 1) {
                    s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
                    s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
                }
                if (lane == 0) pbuf[((size_t)par * C + c) * n + (R - k - 1)] = cscale(s, tau);
            }
        }
        grid_barrier(bar, ++epoch, err, expire_test);
        for (int c = 0; c < C; ++c) {
            const double2* v = X(par, c);
            const double tau = tau_sh[c];
            const double2* p = pbuf + ((size_t)par * C + c) * n;
            double vp_re = 0.0;  // Re(v^H p); v^H p = tau v^H B v is real
            for (int r = threadIdx.x; r < m; r += kTdThreads) {
                const double2 pr = p[r], vr = v[r];
                w_sh[r] = pr;
                vp_re += vr.x * pr.x + vr.y * pr.y;
            }
            vp_re = block_sum_td(vp_re, red);
            const double K = 0.5 * tau * vp_re;
            for (int r = threadIdx.x; r < m; r += kTdThreads) w_sh[r] = csub(w_sh[r], cscale(v[r], K));
            __syncthreads();
            double2* A = Aall + (long long)c * n * n;
            // v of this step into row k right of the diagonal: no step reads or
            // writes that part of row k after step k - 1
            if (blockIdx.x == 0)
                for (int r = threadIdx.x; r < m; r += kTdThreads) A[(long long)k * n + k + 1 + r] = v[r];
            double2* col_out = colbuf + ((size_t)par * C + c) * n;
            for (int R = R0; R < n; R += GW) {
                const int r = R - k - 1;
                const double2 vr = v[r], wr = w_sh[r];
                double2* row = A + (long long)R * n + (k + 1);
                for (int j0 = lane; j0 < m; j0 += 32 * kTdBatch) {
                    double2 a[kTdBatch];
#pragma unroll
                    for (int u = 0; u < kTdBatch; ++u) {
                        const int j = j0 + 32 * u;
                        a[u] = j < m ? row[j] : make_double2(0.0, 0.0);
                    }
#pragma unroll
                    for (int u = 0; u < kTdBatch; ++u) {
                        const int j = j0 + 32 * u;
                        if (j < m) {
                            const double2 b = rank2(a[u], vr, wr, w_sh[j], v[j]);
                            row[j] = b;
                            if (j == 1) col_out[R] = b;
                        }
                    }
                }
            }
            // x_{k+1}[i] = new A[k+2+i][k+1], from the column written by the
            // previous step (step 0: the copy taken before the first step)
            double2* xn = X(par ^ 1, c);
            const double2* col_in = colbuf + ((size_t)(par ^ 1) * C + c) * n;
            const double2 w0 = w_sh[0], v0 = v[0];
            double nrm2 = 0.0;  // ||x_{k+1}||^2 for the next step
            for (int i = threadIdx.x; i < m - 1; i += kTdThreads) {
                const double2 old = k == 0 ? xn[i] : col_in[k + 2 + i];
                const double2 xi = rank2(old, v[i + 1], w_sh[i + 1], w0, v0);
                xn[i] = xi;
                nrm2 += cabs2(xi);
            }
            nrm2 = block_sum_td(nrm2, red);
            if (threadIdx.x == 0) nrm_sh[c] = nrm2;
            __syncthreads();
        }
    }
}

__device__ __forceinline__ int sign_bit(double x) { return (int)((unsigned)__double2hiint(x) >> 31); }
__device__ __forceinline__ int biased_exponent(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }

// Sturm count of the symmetric tridiagonal matrix (d, e) at x: the number
// of sign changes of p_{-1} = 1, p_0 = d_0 - x,
// p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2}, the leading principal minors
// of the shifted matrix, which equals the number of eigenvalues below x.
// No division: the pair (p_{i-1}, p_i) is rescaled by a power of two when
// p_i leaves [2^-511, 2^512]; a zero p_i counts with the sign opposite to
// p_{i-1} (it is replaced by -2^-300 p_{i-1}).
__device__ int sturm_count(int n, const double* d, const double* e2, double x) {
    double pm = 1.0, p = d[0] - x;
    if (biased_exponent(p) == 0) p = -0x1p-300;
    int cnt = sign_bit(p);
    for (int i = 1; i < n; ++i) {
        double q = fma(d[i] - x, p, -e2[i - 1] * pm);
        int ex = biased_exponent(q);
        if (ex == 0) {  // zero (or below the normal range)
            q = -0x1p-300 * p;
            ex = biased_exponent(q);
        }
        cnt += sign_bit(q) ^ sign_bit(p);
        if (ex > 1023 + 512 || ex < 1023 - 511) {
            const double f = __hiloint2double((2046 - ex) << 20, 0);  // 2^-(ex - 1023)
            q *= f;
            p *= f;
        }
        pm = p;
        p = q;
    }
    return cnt;
}

constexpr int kBsWarps = 4;  // eigenvalues per CTA

// Eigenvalue i (largest first) of configuration blockIdx.y, one warp per
// eigenvalue: 32-point multisection of its bracket [lo, hi]
// (count(lo) <= j < count(hi), j = n - 1 - i its ascending index), each
// lane evaluating the Sturm count at one interior point, until the bracket
// is a few ulps wide or 2^-60 of the norm bound wide.  The matrix is scaled
// by a power of two so that its Gershgorin interval lies in [-1, 1].  The
// diagonal and the last off-diagonal entry are read from the reduced
// matrix; the other off-diagonal moduli come from the Householder steps.
// Dynamic shared memory: d [n] and e^2 [n].
__global__ void __launch_bounds__(kBsWarps * 32)
    k_dort_bisect(int n, const double2* __restrict__ Aall, const double* __restrict__ e_all,
                  double* __restrict__ eig) {
    extern __shared__ double de_sh[];
    double* d = de_sh;
    double* e2 = de_sh + n;
    __shared__ double lo_w[kBsWarps], hi_w[kBsWarps];
    __shared__ double lo_sh, hi_sh;
    const int c = blockIdx.y;
    const double2* A = Aall + (long long)c * n * n;
    const int nh = n > 2 ? n - 2 : 0;  // entries produced by the Householder steps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double e_abs[2];
    double lo = 1e308, hi = -1e308;
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = A[(long long)i * n + i].x;
    for (int i = threadIdx.x; i < n - 1; i += blockDim.x) {
        const double ei = i < nh ? e_all[(long long)c * n + i] : sqrt(cabs2(A[(long long)(i + 1) * n + i]));
        e2[i] = ei;  // |e_i| for now
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {  // Gershgorin discs
        e_abs[0] = i > 0 ? e2[i - 1] : 0.0;
        e_abs[1] = i < n - 1 ? e2[i] : 0.0;
        lo = fmin(lo, d[i] - e_abs[0] - e_abs[1]);
        hi = fmax(hi, d[i] + e_abs[0] + e_abs[1]);
    }
    for (int off = 16; off > 0; off >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, off));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if (lane == 0) {
        lo_w[warp] = lo;
        hi_w[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kBsWarps; ++w) {
            lo = fmin(lo, lo_w[w]);
            hi = fmax(hi, hi_w[w]);
        }
        lo_sh = lo;
        hi_sh = hi;
    }
    __syncthreads();
    const double bound = fmax(fabs(lo_sh), fabs(hi_sh));
    const int i = blockIdx.x * kBsWarps + warp;
    if (bound == 0.0) {  // zero matrix
        if (i < n && lane == 0) eig[(long long)c * n + i] = 0.0;
        return;
    }
    const int sc = ilogb(bound) + 1;  // 2^sc > bound
    const double inv = ldexp(1.0, -sc);
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        d[t] *= inv;
        if (t < n - 1) e2[t] = (e2[t] * inv) * (e2[t] * inv);
    }
    __syncthreads();
    if (i >= n) return;
    const int j = n - 1 - i;
    lo = lo_sh * inv - 0x1p-50;
    hi = hi_sh * inv + 0x1p-50;
    for (int round = 0; round < 64; ++round) {
        const double x = lo + (hi - lo) * ((double)(lane + 1) * (1.0 / 33.0));
        const int cnt = sturm_count(n, d, e2, x);
        const unsigned le = __ballot_sync(0xffffffffu, cnt <= j);
        const int L = le ? 31 - __clz(le) : -1;  // highest lane with count <= j
        const double xl = __shfl_sync(0xffffffffu, x, L < 0 ? 0 : L);
        const double xh = __shfl_sync(0xffffffffu, x, L < 31 ? L + 1 : 31);
        const double nlo = L >= 0 ? fmax(lo, xl) : lo;
        const double nhi = L < 31 ? fmin(hi, xh) : hi;
        if (nlo == lo && nhi == hi) break;  // the bracket cannot be split further
        lo = nlo;
        hi = nhi;
        // converged: a few ulps of the eigenvalue, or 2^-60 of the scaled
        // norm bound (below the tridiagonalisation's own error)
        if (hi - lo <= fmax(0x1p-51 * fmax(fabs(lo), fabs(hi)), 0x1p-60)) break;
    }
    if (lane == 0) eig[(long long)c * n + i] = ldexp(0.5 * (lo + hi), sc);
}

// ---------------------------------------------------------------- eigenvectors
//
// After the reduction T' = Q^H T Q with Q = H_0 H_1 ... H_{n-3}
// (H_k = I - tau_k v_k v_k^H on indices k+1..n-1), T' is Hermitian
// tridiagonal with sub-diagonal beta_k = -ph_k sigma_k (k < n - 2) and
// beta_{n-2} = A[n-1][n-2]; with D = diag(delta), delta_0 = 1,
// delta_{k+1} = delta_k beta_k / |beta_k|, T' = D S D^H for the real
// symmetric tridiagonal S with off-diagonal |beta_k| (the matrix whose
// eigenvalues the bisection found).  An eigenvector y of S gives the
// eigenvector Q D y of T.

__device__ __forceinline__ double2 beta_of(int k, int n, const double2* A, const double* e, const double2* ph) {
    if (k < n - 2) return cscale(ph[k], -e[k]);
    return A[(long long)(k + 1) * n + k];
}

// Eigenvectors y of S for the K largest eigenvalues, one warp per
// configuration, in order: inverse iteration (three solves with
// (S - lambda I) by Gaussian elimination with partial pivoting of the
// tridiagonal, a zero pivot replaced by eps ||S||), each iterate
// orthogonalised against the earlier vectors whose eigenvalues lie within
// 1e-3 ||S|| (a cluster) and normalised.  Scratch: 5 n doubles per
// configuration (sub-diagonal after elimination, diagonal, two
// super-diagonals, pivots).
__global__ void __launch_bounds__(32) k_dort_trivec(int n, int K, const double2* __restrict__ Aall,
                                                    const double* __restrict__ e_all, const double2* __restrict__ ph_all,
                                                    const double* __restrict__ eig, double* __restrict__ scratch,
                                                    double* __restrict__ Y) {
    const int c = blockIdx.x, lane = threadIdx.x;
    const double2* A = Aall + (long long)c * n * n;
    const double* e = e_all + (long long)c * n;
    const double2* ph = ph_all + (long long)c * n;
    double* dl = scratch + (long long)c * 5 * n;
    double* dd = dl + n;
    double* du = dd + n;
    double* du2 = du + n;
    double* piv = du2 + n;
    double* Yc = Y + (long long)c * K * n;
    // norm bound of S (Gershgorin)
    double nb = 0.0;
    for (int j = lane; j < n; j += 32) {
        double r = fabs(A[(long long)j * n + j].x);
        if (j > 0) r += sqrt(cabs2(beta_of(j - 1, n, A, e, ph)));
        if (j < n - 1) r += sqrt(cabs2(beta_of(j, n, A, e, ph)));
        nb = fmax(nb, r);
    }
    for (int off = 16; off > 0; off >>= 1) nb = fmax(nb, __shfl_xor_sync(0xffffffffu, nb, off));
    if (nb == 0.0) nb = 1.0;
    const double tiny = 0x1p-52 * nb;
    for (int i = 0; i < K; ++i) {
        const double lam = eig[(long long)c * n + i];
        double* y = Yc + (long long)i * n;
        if (lane == 0) {
            // factor S - lam I = P L U (rows i, i+1 swapped where the
            // sub-diagonal entry is the larger), U with two super-diagonals
            for (int j = 0; j < n; ++j) {
                dd[j] = A[(long long)j * n + j].x - lam;
                if (j < n - 1) dl[j] = du[j] = sqrt(cabs2(beta_of(j, n, A, e, ph)));
                du2[j] = 0.0;
            }
            for (int j = 0; j < n - 1; ++j) {
                if (fabs(dd[j]) >= fabs(dl[j])) {
                    piv[j] = 0.0;
                    if (dd[j] == 0.0) dd[j] = tiny;
                    const double f = dl[j] / dd[j];
                    dl[j] = f;
                    dd[j + 1] -= f * du[j];
                } else {
                    piv[j] = 1.0;
                    const double f = dd[j] / dl[j];
                    dd[j] = dl[j];
                    dl[j] = f;
                    const double t = du[j];
                    du[j] = dd[j + 1];
                    dd[j + 1] = t - f * dd[j + 1];
                    if (j < n - 2) {
                        du2[j] = du[j + 1];
                        du[j + 1] = -f * du[j + 1];
                    }
                }
            }
            if (dd[n - 1] == 0.0) dd[n - 1] = tiny;
            for (int j = 0; j < n; ++j) y[j] = 1.0 + 0.25 * sin(1.0 + j);  // fixed start vector
        }
        __syncwarp();
        for (int it = 0; it < 3; ++it) {
            if (lane == 0) {
                // forward: apply P and L^-1; backward: U^-1
                for (int j = 0; j < n - 1; ++j) {
                    if (piv[j] == 0.0) {
                        y[j + 1] -= dl[j] * y[j];
                    } else {
                        const double t = y[j];
                        y[j] = y[j + 1];
                        y[j + 1] = t - dl[j] * y[j];
                    }
                }
                y[n - 1] /= dd[n - 1];
                if (n > 1) y[n - 2] = (y[n - 2] - du[n - 2] * y[n - 1]) / dd[n - 2];
                for (int j = n - 3; j >= 0; --j) y[j] = (y[j] - du[j] * y[j + 1] - du2[j] * y[j + 2]) / dd[j];
            }
            __syncwarp();
            // orthogonalise against earlier vectors of the cluster, then normalise
            for (int j = 0; j < i; ++j) {
                if (fabs(eig[(long long)c * n + j] - lam) > 1e-3 * nb) continue;
                const double* yj = Yc + (long long)j * n;
                double dot = 0.0;
                for (int t = lane; t < n; t += 32) dot += yj[t] * y[t];
                for (int off = 16; off > 0; off >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, off);
                for (int t = lane; t < n; t += 32) y[t] -= dot * yj[t];
                __syncwarp();
            }
            double nrm = 0.0;
            for (int t = lane; t < n; t += 32) nrm += y[t] * y[t];
            for (int off = 16; off > 0; off >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, off);
            const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
            for (int t = lane; t < n; t += 32) y[t] *= inv;
            __syncwarp();
        }
    }
}

constexpr int kBtThreads = 256;

// u = Q D y for eigenvector i of configuration c (grid: K x C): the phases
// delta, then the reflectors applied last to first; finally the phase of the
// vector is fixed (its largest-modulus entry real and positive).  Dynamic
// shared memory: z [n] complex.
__global__ void __launch_bounds__(kBtThreads) k_dort_backtransform(int n, int K, const double2* __restrict__ Aall,
                                                                   const double* __restrict__ e_all,
                                                                   const double* __restrict__ tau_all,
                                                                   const double2* __restrict__ ph_all,
                                                                   const double* __restrict__ Y,
                                                                   double2* __restrict__ U) {
    extern __shared__ double2 z[];
    __shared__ double2 red[kBtThreads / 32];
    __shared__ double2 dot_sh;
    const int i = blockIdx.x, c = blockIdx.y, t = threadIdx.x;
    const double2* A = Aall + (long long)c * n * n;
    const double* e = e_all + (long long)c * n;
    const double2* ph = ph_all + (long long)c * n;
    const double* y = Y + ((long long)c * K + i) * n;
    if (t == 0) {
        double2 delta = make_double2(1.0, 0.0);
        for (int k = 0; k < n; ++k) {
            z[k] = cscale(delta, y[k]);
            if (k < n - 1) {
                const double2 b = beta_of(k, n, A, e, ph);
                const double ab = sqrt(cabs2(b));
                if (ab > 0.0) delta = cmul(delta, make_double2(b.x / ab, b.y / ab));
            }
        }
    }
    __syncthreads();
    for (int k = n - 3; k >= 0; --k) {
        const int m = n - k - 1;
        const double tau = tau_all[(long long)c * n + k];
        const double2* v = A + (long long)k * n + k + 1;
        double2 s = make_double2(0.0, 0.0);  // v^H z[k+1:]
        for (int r = t; r < m; r += kBtThreads) s = cadd(s, cmul(cconj(v[r]), z[k + 1 + r]));
        for (int off = 16; off > 0; off >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
        }
        if ((t & 31) == 0) red[t >> 5] = s;
        __syncthreads();
        if (t == 0) {
            double2 a = make_double2(0.0, 0.0);
            for (int w = 0; w < kBtThreads / 32; ++w) a = cadd(a, red[w]);
            dot_sh = cscale(a, tau);
        }
        __syncthreads();
        const double2 f = dot_sh;
        for (int r = t; r < m; r += kBtThreads) z[k + 1 + r] = csub(z[k + 1 + r], cmul(v[r], f));
        __syncthreads();
    }
    // phase: the entry of largest modulus real and positive
    if (t == 0) {
        int jm = 0;
        double am = -1.0;
        for (int j = 0; j < n; ++j) {
            const double a2 = cabs2(z[j]);
            if (a2 > am) {
                am = a2;
                jm = j;
            }
        }
        const double a = sqrt(am);
        dot_sh = a > 0.0 ? make_double2(z[jm].x / a, -z[jm].y / a) : make_double2(1.0, 0.0);
    }
    __syncthreads();
    const double2 f = dot_sh;
    for (int j = t; j < n; j += kBtThreads) U[((long long)c * K + i) * n + j] = cmul(z[j], f);
}

// Discrete Herglotz waves (section 7): u[p][r] = h sum_j g[r][j]
// exp(i k (x_p cos a_j + y_p sin a_j)), a_j = 2 pi j / na, h = 2 pi / na.
__global__ void k_herglotz(double k, int na, int K, const double2* __restrict__ g, long long P,
                           const double2* __restrict__ pts, double2* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= P * K) return;
    const long long p = t / K;
    const int r = (int)(t - p * K);
    const double2 x = pts[p];
    const double h = 2.0 * M_PI / na;
    double2 u = make_double2(0.0, 0.0);
    for (int j = 0; j < na; ++j) {
        double sa, ca;
        sincospi(2.0 * j / na, &sa, &ca);
        double sp, cp;
        sincos(k * (x.x * ca + x.y * sa), &sp, &cp);
        u = cadd(u, cmul(g[(long long)r * na + j], make_double2(cp, sp)));
    }
    out[p * K + r] = cscale(u, h);
}

}  // namespace

size_t dort_work_bytes(int C, int n) {
    // T copy, p and column buffers (two each), e, tau, phases, barrier counter and error flag
    return (size_t)C * n * n * 16 + 4 * (size_t)C * n * 16 + (size_t)C * n * 8 + (size_t)C * n * 8 +
           (size_t)C * n * 16 + 16;
}

namespace {
constexpr size_t kTdSmemMax = 220 * 1024;
size_t tridiag_smem(int Cg, int n) { return (2 * (size_t)Cg * n + n) * 16 + (size_t)Cg * 16; }
int tridiag_group(int C, int n) {
    int g = (int)((kTdSmemMax / 16 - n) / (2 * (size_t)n + 1));
    return std::max(1, std::min(C, g));
}
}  // namespace

cudaError_t dort_set_smem_limits(int n) {
    // the tridiagonalisation's shared memory: x of two steps per configuration, w, tau
    return cudaFuncSetAttribute(k_dort_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTdSmemMax);
}

cudaError_t launch_dort(int C, int n, const double2* F, double2* T, void* work, double* eig, int* err_host_flag,
                        cudaStream_t s) {
    char* w = (char*)work;
    double2* A = (double2*)w;
    w += (size_t)C * n * n * 16;
    double2* pbuf = (double2*)w;  // [2][C][n]
    w += 2 * (size_t)C * n * 16;
    double2* colbuf = (double2*)w;  // [2][C][n]
    w += 2 * (size_t)C * n * 16;
    double2* ph = (double2*)w;  // 16-byte aligned: it follows the complex buffers
    w += (size_t)C * n * 16;
    double* e = (double*)w;
    w += (size_t)C * n * 8;
    double* tau = (double*)w;
    w += (size_t)C * n * 8;
    unsigned* bar = (unsigned*)w;
    int* err = (int*)(w + 4);
    const int tiles = (n + kGramTile - 1) / kGramTile;
    k_dort_gram<<<dim3(tiles, tiles, C), dim3(kGramTile, kGramTile), 0, s>>>(n, F, T);
    cudaError_t ce = cudaMemcpyAsync(A, T, (size_t)C * n * n * 16, cudaMemcpyDeviceToDevice, s);
    if (ce != cudaSuccess) return ce;
    ce = cudaMemsetAsync(bar, 0, 8, s);
    if (ce != cudaSuccess) return ce;
    long long launches = 2;
    if (n > 2) {
        // persistent grid, every CTA co-resident (cooperative launch); the
        // configurations in groups whose x buffers fit in shared memory
        int dev = 0, sms = 0;
        if ((ce = cudaGetDevice(&dev)) != cudaSuccess) return ce;
        if ((ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return ce;
        const int G = tridiag_group(C, n);
        for (int c0 = 0; c0 < C; c0 += G) {
            int Cg = std::min(G, C - c0);
            const size_t smem = tridiag_smem(Cg, n);
            int per_sm = 0;
            if ((ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dort_tridiag, kTdThreads, smem)) !=
                cudaSuccess)
                return ce;
            const int need = (n - 1 + kTdWarps - 1) / kTdWarps;
            const int grid = std::max(1, std::min(need, per_sm * sms));
            if (c0 > 0 && (ce = cudaMemsetAsync(bar, 0, 4, s)) != cudaSuccess) return ce;
            double2* Ag = A + (size_t)c0 * n * n;
            double* eg = e + (size_t)c0 * n;
            double* tg = tau + (size_t)c0 * n;
            double2* pg = ph + (size_t)c0 * n;
            int expire_test = g_msd_expire_waits.load();
            void* args[] = {&Cg, (void*)&n, &Ag, &pbuf, &colbuf, &eg, &tg, &pg, &bar, &err, &expire_test};
            ce = cudaLaunchCooperativeKernel((const void*)k_dort_tridiag, dim3(grid), dim3(kTdThreads), args, smem, s);
            if (ce != cudaSuccess) return ce;
            ++launches;
        }
    }
    k_dort_bisect<<<dim3((n + kBsWarps - 1) / kBsWarps, C), kBsWarps * 32, (size_t)n * 16, s>>>(n, A, e, eig);
    g_msd_launches += launches;
    return cudaMemcpyAsync(err_host_flag, err, 4, cudaMemcpyDeviceToHost, s);
}

// Eigenvectors of the K largest eigenvalues after launch_dort with the same
// work buffer (reflectors, taus, phases and the reduced matrices kept there):
// U [C][K][n] complex128, unit 2-norm, the largest-modulus entry real positive.
// scratch: dort_vec_scratch_bytes(C, n, K).
size_t dort_vec_scratch_bytes(int C, int n, int K) { return (size_t)C * 5 * n * 8 + (size_t)C * K * n * 8; }

cudaError_t launch_dort_vectors(int C, int n, int K, void* work, const double* eig, void* scratch, double2* U,
                                cudaStream_t s) {
    char* w = (char*)work;
    double2* A = (double2*)w;
    w += (size_t)C * n * n * 16 + 4 * (size_t)C * n * 16;
    double2* ph = (double2*)w;
    w += (size_t)C * n * 16;
    double* e = (double*)w;
    w += (size_t)C * n * 8;
    double* tau = (double*)w;
    double* lu = (double*)scratch;
    double* Y = lu + (size_t)C * 5 * n;
    k_dort_trivec<<<C, 32, 0, s>>>(n, K, A, e, ph, eig, lu, Y);
    k_dort_backtransform<<<dim3(K, C), kBtThreads, (size_t)n * 16, s>>>(n, K, A, e, tau, ph, Y, U);
    g_msd_launches += 2;
    return cudaGetLastError();
}

void launch_herglotz(double k, int na, int K, const double2* g, long long P, const double2* pts, double2* out,
                     cudaStream_t s) {
    const long long tot = P * K;
    if (tot <= 0) return;
    k_herglotz<<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(k, na, K, g, P, pts, out);
    g_msd_launches += 1;
}
