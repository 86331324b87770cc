// Time reversal (section 7, DORT): the time-reversal matrix T = conj(F)^T F
// of every configuration's far-field matrix F [n][n] (row i: far field at
// alpha_i + pi; column j: incidence alpha_j) and the eigenvalues of T.
//
// Eigenvalues: T is Hermitian.  Householder reflections reduce it to a
// Hermitian tridiagonal matrix (n - 2 steps; step k maps column k below the
// diagonal onto a multiple of e_1 with H = I - tau v v^H and applies
// H B H = B - v w^H - w v^H to the trailing block B, p = tau B v,
// w = p - (tau/2)(v^H p) v).  A diagonal unitary similarity makes the
// off-diagonal entries real and non-negative (their moduli), and the
// eigenvalues of that real symmetric tridiagonal matrix are found one per
// thread by bisection on the Sturm count (the number of negative pivots of
// the LDL^T factorisation of the shifted matrix is the number of
// eigenvalues below the shift).  Every step runs over all configurations
// at once (grid.y = configuration).
#include <cuda_runtime.h>

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

constexpr int kHhThreads = 256;
constexpr int kHhRows = kHhThreads / 32;  // one warp per row

__device__ double block_sum_256(double v, double* red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kHhThreads / 32; ++w) s += red[w];
    __syncthreads();
    return s;
}

// Householder step k, part 1: every CTA builds v and tau from column k
// (rows k+1..n-1, untouched by this step) and forms p = tau B v for its
// rows of the trailing block B = A[k+1:, k+1:].  CTA 0 stores v, tau,
// d_k = Re A[k][k] and e_k = ||A[k+1:, k]||.  Dynamic shared memory: the
// m = n - k - 1 entries of v.
__global__ void __launch_bounds__(kHhThreads)
    k_dort_hh_mv(int n, int k, double2* __restrict__ Aall, double2* __restrict__ vall, double2* __restrict__ pall,
                 double* __restrict__ tau_all, double* __restrict__ d_all, double* __restrict__ e_all) {
    extern __shared__ double2 v_sh[];
    __shared__ double red[kHhThreads / 32];
    const int c = blockIdx.y, m = n - k - 1;
    double2* A = Aall + (long long)c * n * n;
    double nrm2 = 0.0;
    for (int r = threadIdx.x; r < m; r += kHhThreads) {
        const double2 x = A[(long long)(k + 1 + r) * n + k];
        v_sh[r] = x;
        nrm2 += cabs2(x);
    }
    nrm2 = block_sum_256(nrm2, red);
    const double sigma = sqrt(nrm2);
    const double2 x0 = A[(long long)(k + 1) * n + k];
    const double ax0 = sqrt(cabs2(x0));
    // v = x + e^{i arg x0} sigma e_1 maps x onto -e^{i arg x0} sigma e_1;
    // ||v||^2 = 2 sigma (sigma + |x0|), tau = 2 / ||v||^2
    const double tau = sigma > 0.0 ? 1.0 / (sigma * (sigma + ax0)) : 0.0;
    if (threadIdx.x == 0 && sigma > 0.0) {
        const double2 ph = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
        v_sh[0] = cadd(x0, cscale(ph, sigma));
    }
    __syncthreads();
    if (blockIdx.x == 0) {
        for (int r = threadIdx.x; r < m; r += kHhThreads) vall[(long long)c * n + r] = v_sh[r];
        if (threadIdx.x == 0) {
            tau_all[c] = tau;
            d_all[(long long)c * n + k] = A[(long long)k * n + k].x;
            e_all[(long long)c * n + k] = sigma;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * kHhRows + warp;
    if (r >= m) return;
    const double2* row = A + (long long)(k + 1 + r) * n + (k + 1);
    double2 s = make_double2(0.0, 0.0);
    for (int j = lane; j < m; j += 32) s = cadd(s, cmul(row[j], v_sh[j]));
    for (int off = 16; off > 0; off >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
    }
    if (lane == 0) pall[(long long)c * n + r] = cscale(s, tau);
}

// Householder step k, part 2: w = p - (tau/2)(v^H p) v (every CTA), then
// B <- B - v w^H - w v^H on the CTA's rows.  Dynamic shared memory: v and w.
__global__ void __launch_bounds__(kHhThreads)
    k_dort_hh_update(int n, int k, double2* __restrict__ Aall, const double2* __restrict__ vall,
                     const double2* __restrict__ pall, const double* __restrict__ tau_all) {
    extern __shared__ double2 vw_sh[];
    __shared__ double red[kHhThreads / 32];
    const int c = blockIdx.y, m = n - k - 1;
    const double tau = tau_all[c];
    if (tau == 0.0) return;  // column already reduced: H = I
    double2* v_sh = vw_sh;
    double2* w_sh = vw_sh + m;
    double vp_re = 0.0;  // Re(v^H p); v^H p = tau v^H B v is real
    for (int r = threadIdx.x; r < m; r += kHhThreads) {
        const double2 v = vall[(long long)c * n + r], p = pall[(long long)c * n + r];
        v_sh[r] = v;
        w_sh[r] = p;
        vp_re += v.x * p.x + v.y * p.y;
    }
    vp_re = block_sum_256(vp_re, red);
    const double K = 0.5 * tau * vp_re;
    for (int r = threadIdx.x; r < m; r += kHhThreads) w_sh[r] = csub(w_sh[r], cscale(v_sh[r], K));
    __syncthreads();
    double2* A = Aall + (long long)c * n * n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * kHhRows + warp;
    if (r >= m) return;
    const double2 vr = v_sh[r], wr = w_sh[r];
    double2* row = A + (long long)(k + 1 + r) * n + (k + 1);
    for (int j = lane; j < m; j += 32)
        row[j] = csub(row[j], cadd(cmul(vr, cconj(w_sh[j])), cmul(wr, cconj(v_sh[j]))));
}

// Sturm count: the number of eigenvalues of the symmetric tridiagonal
// matrix (d, e) below x.
__device__ int sturm_count(int n, const double* d, const double* e2, double x, double pivmin) {
    int cnt = 0;
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++cnt;
    for (int i = 1; i < n; ++i) {
        q = (d[i] - x) - e2[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// Eigenvalue i (largest first) of configuration blockIdx.y by bisection.
// The last two diagonal entries and the last off-diagonal one are read
// from the reduced matrix; the others come from the Householder steps.
// Dynamic shared memory: d [n] and e^2 [n].
__global__ void k_dort_bisect(int n, const double2* __restrict__ Aall, const double* __restrict__ d_all,
                              const double* __restrict__ e_all, double* __restrict__ eig) {
    extern __shared__ double de_sh[];
    double* d = de_sh;
    double* e2 = de_sh + n;
    __shared__ double lo_sh, hi_sh, pivmin_sh;
    const int c = blockIdx.y;
    const double2* A = Aall + (long long)c * n * n;
    const int nh = n > 2 ? n - 2 : 0;  // entries produced by the Householder steps
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        d[i] = i < nh ? d_all[(long long)c * n + i] : A[(long long)i * n + i].x;
        if (i < n - 1) {
            const double ei = i < nh ? e_all[(long long)c * n + i] : sqrt(cabs2(A[(long long)(i + 1) * n + i]));
            e2[i] = ei * ei;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // Gershgorin interval and pivot floor
        double lo = d[0], hi = d[0], emax2 = 1.0;
        for (int i = 0; i < n; ++i) {
            const double r = (i > 0 ? sqrt(e2[i - 1]) : 0.0) + (i < n - 1 ? sqrt(e2[i]) : 0.0);
            lo = fmin(lo, d[i] - r);
            hi = fmax(hi, d[i] + r);
            if (i < n - 1) emax2 = fmax(emax2, e2[i]);
        }
        const double w = fmax(fabs(lo), fabs(hi));
        lo_sh = lo - 4e-16 * w - 1e-300;
        hi_sh = hi + 4e-16 * w + 1e-300;
        pivmin_sh = 1e-290 * emax2;
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = n - 1 - i;  // ascending index of the eigenvalue
    double lo = lo_sh, hi = hi_sh;  // count(lo) <= j < count(hi)
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;  // interval at the last bit
        if (sturm_count(n, d, e2, mid, pivmin_sh) <= j) lo = mid;
        else hi = mid;
    }
    eig[(long long)c * n + i] = 0.5 * (lo + hi);
}

}  // namespace

size_t dort_work_bytes(int C, int n) {
    // T copy, v, p, tau, d, e
    return (size_t)C * n * n * 16 + 2 * (size_t)C * n * 16 + (size_t)C * 8 + 2 * (size_t)C * n * 8;
}

void launch_dort(int C, int n, const double2* F, double2* T, void* work, double* eig, cudaStream_t s) {
    char* w = (char*)work;
    double2* A = (double2*)w;
    w += (size_t)C * n * n * 16;
    double2* v = (double2*)w;
    w += (size_t)C * n * 16;
    double2* p = (double2*)w;
    w += (size_t)C * n * 16;
    double* tau = (double*)w;
    w += (size_t)C * 8;
    double* d = (double*)w;
    w += (size_t)C * n * 8;
    double* e = (double*)w;
    const int tiles = (n + kGramTile - 1) / kGramTile;
    k_dort_gram<<<dim3(tiles, tiles, C), dim3(kGramTile, kGramTile), 0, s>>>(n, F, T);
    cudaMemcpyAsync(A, T, (size_t)C * n * n * 16, cudaMemcpyDeviceToDevice, s);
    long long launches = 1;
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        const dim3 grid((m + kHhRows - 1) / kHhRows, C);
        k_dort_hh_mv<<<grid, kHhThreads, (size_t)m * 16, s>>>(n, k, A, v, p, tau, d, e);
        k_dort_hh_update<<<grid, kHhThreads, (size_t)m * 32, s>>>(n, k, A, v, p, tau);
        launches += 2;
    }
    k_dort_bisect<<<dim3((n + 31) / 32, C), 32, (size_t)n * 16, s>>>(n, A, d, e, eig);
    g_msd_launches += launches + 1;
}

cudaError_t dort_set_smem_limits(int n) {
    // dynamic shared memory above 48 KB needs an opt-in (n > 1536 for the update)
    const int need = n * 32;
    if (need <= 48 * 1024) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_dort_hh_update, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_dort_hh_mv, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_dort_bisect, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
}
