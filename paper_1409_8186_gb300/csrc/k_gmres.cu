// K4: batched restarted GMRES on the device (section 5: preconditioned
// Krylov solve; the restarted GMRES call of section 6.2).
//
// A "system" is one (configuration, column) pair s = cfg*R + r; all systems
// advance in lock step (one block matvec per Arnoldi step serves all of
// them) and each carries its own Hessenberg matrix, Givens rotations and
// convergence state.  Orthogonalisation is classical Gram-Schmidt applied
// twice (CGS2); dot products accumulate in FP64 whatever the storage type of
// the basis.  Vectors are [rows][R] with R innermost; reductions run over
// row chunks that never straddle two configurations.
#include "msd_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kIChunk = 8;  // basis vectors handled per pass of a reduction

template <typename V> __device__ __forceinline__ double2 to_d2(V v) { return make_double2(v.x, v.y); }

// Column lanes: RC = min(R, 32) (power of two not required), rows lanes RY.
__host__ __device__ inline int col_lanes(int R) { return R < 32 ? R : 32; }

// Partial sums of conj(V_i) * w over one chunk of rows (blockIdx.x), for the
// kIChunk basis vectors i in [blockIdx.z * kIChunk, ...), columns of group
// blockIdx.y.  Each block reads its w chunk once per vector group.
template <typename V>
__global__ void k_multidot_part(const RowChunk* __restrict__ chunks, int R, const V* __restrict__ Vb,
                                long long vstride, int nv, const V* __restrict__ w,
                                double2* __restrict__ part) {
    const RowChunk ch = chunks[blockIdx.x];
    const int RC = col_lanes(R);
    int RY = 1;  // row lanes: a power of two so that the tree below is exact
    while (RY * 2 * RC <= (int)blockDim.x) RY *= 2;
    const int tx = threadIdx.x % RC, ty = threadIdx.x / RC;
    const int r = blockIdx.y * RC + tx;
    const int i0 = blockIdx.z * kIChunk;
    __shared__ double2 red[kThreads];
    double2 acc[kIChunk];
#pragma unroll
    for (int ii = 0; ii < kIChunk; ++ii) acc[ii] = make_double2(0.0, 0.0);
    if (ty < RY && r < R) {
        for (long long row = ch.row0 + ty; row < ch.row1; row += RY) {
            const double2 wv = to_d2(w[row * R + r]);
#pragma unroll
            for (int ii = 0; ii < kIChunk; ++ii) {
                if (i0 + ii < nv) {
                    const double2 vv = to_d2(Vb[(long long)(i0 + ii) * vstride + row * R + r]);
                    acc[ii].x += vv.x * wv.x + vv.y * wv.y;  // conj(v) * w
                    acc[ii].y += vv.x * wv.y - vv.y * wv.x;
                }
            }
        }
    }
    for (int ii = 0; ii < kIChunk && i0 + ii < nv; ++ii) {
        red[threadIdx.x] = acc[ii];
        __syncthreads();
        for (int st = RY / 2; st > 0; st /= 2) {
            if (ty < st) {
                double2 o = red[threadIdx.x + st * RC];
                red[threadIdx.x].x += o.x;
                red[threadIdx.x].y += o.y;
            }
            __syncthreads();
        }
        if (ty == 0 && r < R) part[((long long)blockIdx.x * nv + (i0 + ii)) * R + r] = red[tx];
        __syncthreads();
    }
}

// h[s][i] = sum over the chunks of cfg(s) of part[chunk][i][r] (+= if accumulate)
__global__ void k_multidot_fin(int C, int R, int nv, const int* __restrict__ cfg_chunk_off,
                               const double2* __restrict__ part, double2* __restrict__ h, int hstride,
                               int accumulate) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= C * R * nv) return;
    const int i = idx % nv;
    const int s = idx / nv;
    const int c = s / R, r = s % R;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = cfg_chunk_off[c]; k < cfg_chunk_off[c + 1]; ++k) {
        const double2 v = part[((long long)k * nv + i) * R + r];
        acc.x += v.x;
        acc.y += v.y;
    }
    double2* dst = h + (long long)s * hstride + i;
    if (accumulate) {
        dst->x += acc.x;
        dst->y += acc.y;
    } else {
        *dst = acc;
    }
}

// w[row][r] -= sum_i V_i[row][r] h[s][i]   (s = cfg(row)*R + r)
template <typename V>
__global__ void k_update(const RowChunk* __restrict__ chunks, int R, const V* __restrict__ Vb,
                         long long vstride, int nv, const double2* __restrict__ h, int hstride,
                         V* __restrict__ w) {
    const RowChunk ch = chunks[blockIdx.x];
    const int RC = col_lanes(R);
    const int RY = blockDim.x / RC;
    const int tx = threadIdx.x % RC, ty = threadIdx.x / RC;
    const int r = blockIdx.y * RC + tx;
    if (ty >= RY || r >= R) return;
    const double2* hs = h + (long long)(ch.cfg * R + r) * hstride;
    for (long long row = ch.row0 + ty; row < ch.row1; row += RY) {
        // four independent partial sums keep several loads of V in flight
        double2 a[4] = {to_d2(w[row * R + r]), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
                        make_double2(0.0, 0.0)};
        const V* vp = Vb + row * R + r;
        int i = 0;
        for (; i + 4 <= nv; i += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double2 vv = to_d2(vp[(long long)(i + u) * vstride]);
                const double2 hh = hs[i + u];
                a[u].x -= vv.x * hh.x - vv.y * hh.y;
                a[u].y -= vv.x * hh.y + vv.y * hh.x;
            }
        }
        for (; i < nv; ++i) {
            const double2 vv = to_d2(vp[(long long)i * vstride]);
            const double2 hh = hs[i];
            a[0].x -= vv.x * hh.x - vv.y * hh.y;
            a[0].y -= vv.x * hh.y + vv.y * hh.x;
        }
        const double ax = (a[0].x + a[1].x) + (a[2].x + a[3].x);
        const double ay = (a[0].y + a[1].y) + (a[2].y + a[3].y);
        w[row * R + r] = V{(decltype(V{}.x))ax, (decltype(V{}.x))ay};
    }
}

// v = w * scale[s] for active systems, 0 otherwise.  Input FP64 or T, output T.
template <typename Vin, typename Vout>
__global__ void k_scale(const RowChunk* __restrict__ chunks, int R, const Vin* __restrict__ w,
                        const double* __restrict__ scale, const int* __restrict__ active,
                        Vout* __restrict__ v) {
    const RowChunk ch = chunks[blockIdx.x];
    const int RC = col_lanes(R);
    const int RY = blockDim.x / RC;
    const int tx = threadIdx.x % RC, ty = threadIdx.x / RC;
    const int r = blockIdx.y * RC + tx;
    if (ty >= RY || r >= R) return;
    const int s = ch.cfg * R + r;
    const double f = active[s] ? scale[s] : 0.0;
    for (long long row = ch.row0 + ty; row < ch.row1; row += RY) {
        const double2 a = to_d2(w[row * R + r]);
        v[row * R + r] = Vout{(decltype(Vout{}.x))(a.x * f), (decltype(Vout{}.x))(a.y * f)};
    }
}

// x[row][r] += sum_{i < kconv[s]} V_i[row][r] y[s][i]
template <typename V>
__global__ void k_xupdate(const RowChunk* __restrict__ chunks, int R, const V* __restrict__ Vb,
                          long long vstride, const double2* __restrict__ y, int ystride,
                          const int* __restrict__ kconv, double2* __restrict__ x) {
    const RowChunk ch = chunks[blockIdx.x];
    const int RC = col_lanes(R);
    const int RY = blockDim.x / RC;
    const int tx = threadIdx.x % RC, ty = threadIdx.x / RC;
    const int r = blockIdx.y * RC + tx;
    if (ty >= RY || r >= R) return;
    const int s = ch.cfg * R + r;
    const int k = kconv[s];
    if (k == 0) return;
    const double2* ys = y + (long long)s * ystride;
    for (long long row = ch.row0 + ty; row < ch.row1; row += RY) {
        double2 acc = x[row * R + r];
        for (int i = 0; i < k; ++i) {
            const double2 vv = to_d2(Vb[(long long)i * vstride + row * R + r]);
            acc.x += vv.x * ys[i].x - vv.y * ys[i].y;
            acc.y += vv.x * ys[i].y + vv.y * ys[i].x;
        }
        x[row * R + r] = acc;
    }
}

// Start of a cycle: beta = ||r||; systems whose residual already meets
// tol_abs are done.  g = [beta, 0, ...], scale = 1/beta.
__global__ void k_start(int S, int m, const double2* __restrict__ rr, int hstride,
                        const double* __restrict__ tol_abs, double* __restrict__ beta_out,
                        double* __restrict__ vscale, double2* __restrict__ g, int* __restrict__ active,
                        int* __restrict__ kconv, int* __restrict__ any_active) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const double beta = sqrt(rr[(long long)s * hstride].x);
    beta_out[s] = beta;
    kconv[s] = 0;
    const int act = (beta > tol_abs[s]) && isfinite(beta);
    active[s] = act;
    vscale[s] = act ? 1.0 / beta : 0.0;
    double2* gs = g + (long long)s * (m + 1);
    gs[0] = make_double2(act ? beta : 0.0, 0.0);
    for (int i = 1; i <= m; ++i) gs[i] = make_double2(0.0, 0.0);
    if (act) atomicOr(any_active, 1);
}

// Arnoldi step j: column h = h1 + h2 (CGS2), h[j+1] = ||w||; apply the previous
// rotations, make a new one, update g and the convergence state.
__global__ void k_givens(int S, int m, int j, const double2* __restrict__ h1, const double2* __restrict__ h2,
                         int hstride, const double2* __restrict__ wn2, const double* __restrict__ tol_cycle,
                         double2* __restrict__ H, double2* __restrict__ cs, double2* __restrict__ sn,
                         double2* __restrict__ g, double* __restrict__ vscale, int* __restrict__ active,
                         int* __restrict__ kconv, int* __restrict__ iters, int* __restrict__ any_active,
                         int* __restrict__ nonfinite) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    if (!active[s]) return;
    double2* Hc = H + ((long long)s * m + j) * (m + 1);  // column j, rows 0..j+1
    const double2* a = h1 + (long long)s * hstride;
    const double2* b = h2 + (long long)s * hstride;
    for (int i = 0; i <= j; ++i) Hc[i] = make_double2(a[i].x + b[i].x, a[i].y + b[i].y);
    const double hn = sqrt(fmax(wn2[(long long)s * hstride].x, 0.0));
    double2* csj = cs + (long long)s * m;
    double2* snj = sn + (long long)s * m;
    for (int i = 0; i < j; ++i) {
        const double2 c = csj[i], sn_ = snj[i];
        const double2 hi = Hc[i], hi1 = Hc[i + 1];
        // [c s; -conj(s) c] with c real
        Hc[i] = cadd(cscale(hi, c.x), cmul(sn_, hi1));
        Hc[i + 1] = csub(cscale(hi1, c.x), cmul(cconj(sn_), hi));
    }
    const double2 hjj = Hc[j];
    const double ajj = sqrt(cabs2(hjj));
    const double den = hypot(ajj, hn);
    double2 c, sv;
    if (den == 0.0) {
        c = make_double2(1.0, 0.0);
        sv = make_double2(0.0, 0.0);
    } else if (ajj == 0.0) {
        c = make_double2(0.0, 0.0);
        sv = make_double2(1.0, 0.0);  // hn real and positive
    } else {
        const double2 ph = cscale(hjj, 1.0 / ajj);
        c = make_double2(ajj / den, 0.0);
        sv = cscale(ph, hn / den);  // ph * conj(hn) / den, hn real
    }
    csj[j] = c;
    snj[j] = sv;
    Hc[j] = cadd(cscale(hjj, c.x), cscale(sv, hn));
    Hc[j + 1] = make_double2(0.0, 0.0);
    double2* gs = g + (long long)s * (m + 1);
    const double2 gj = gs[j];
    gs[j + 1] = cscale(cmul(cconj(sv), gj), -1.0);
    gs[j] = cscale(gj, c.x);
    iters[s] += 1;
    const double res = sqrt(cabs2(gs[j + 1]));
    const bool bad = !isfinite(res) || !isfinite(Hc[j].x) || !isfinite(Hc[j].y);
    if (bad) atomicOr(nonfinite, 1);
    if (bad || res <= tol_cycle[s] || hn == 0.0 || j + 1 == m) {
        active[s] = 0;
        kconv[s] = j + 1;
        vscale[s] = 0.0;
    } else {
        vscale[s] = 1.0 / hn;
        atomicOr(any_active, 1);
    }
}

// Back substitution H y = g on the leading kconv x kconv triangle.
__global__ void k_lsq(int S, int m, const double2* __restrict__ H, const double2* __restrict__ g,
                      const int* __restrict__ kconv, double2* __restrict__ y) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const int k = kconv[s];
    const double2* Hs = H + (long long)s * m * (m + 1);
    const double2* gs = g + (long long)s * (m + 1);
    double2* ys = y + (long long)s * m;
    for (int i = k - 1; i >= 0; --i) {
        double2 acc = gs[i];
        for (int jj = i + 1; jj < k; ++jj) acc = csub(acc, cmul(Hs[(long long)jj * (m + 1) + i], ys[jj]));
        const double2 d = Hs[(long long)i * (m + 1) + i];
        ys[i] = (d.x == 0.0 && d.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(acc, d);
    }
}

__global__ void k_residual(long long n, const double2* __restrict__ b, const double2* __restrict__ Ax,
                           double2* __restrict__ r) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = csub(b[i], Ax[i]);
}

__global__ void k_zero(long long n, double2* __restrict__ x) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = make_double2(0.0, 0.0);
}

__global__ void k_cast_f32(long long n, const double2* __restrict__ a, float2* __restrict__ b) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

inline dim3 grid_for(const GmresDims& d) { return dim3(d.nchunk, (d.R + col_lanes(d.R) - 1) / col_lanes(d.R)); }
inline unsigned blocks_for(long long n, int th) { return (unsigned)((n + th - 1) / th); }

}  // namespace

// ---------------------------------------------------------------- host wrappers

template <typename V>
void gm_multidot(const GmresDims& d, const RowChunk* chunks, const int* cfg_chunk_off, const V* Vb,
                 long long vstride, int nv, const V* w, double2* part, double2* h, int hstride,
                 int accumulate, cudaStream_t s) {
    dim3 g = grid_for(d);
    g.z = (nv + kIChunk - 1) / kIChunk;
    k_multidot_part<V><<<g, kThreads, 0, s>>>(chunks, d.R, Vb, vstride, nv, w, part);
    const int tot = d.S * nv;
    k_multidot_fin<<<blocks_for(tot, 128), 128, 0, s>>>(d.C, d.R, nv, cfg_chunk_off, part, h, hstride,
                                                        accumulate);
    g_msd_launches += 2;
}

template <typename V>
void gm_update(const GmresDims& d, const RowChunk* chunks, const V* Vb, long long vstride, int nv,
               const double2* h, int hstride, V* w, cudaStream_t s) {
    k_update<V><<<grid_for(d), kThreads, 0, s>>>(chunks, d.R, Vb, vstride, nv, h, hstride, w);
    g_msd_launches += 1;
}

template <typename Vin, typename Vout>
void gm_scale(const GmresDims& d, const RowChunk* chunks, const Vin* w, const double* scale,
              const int* active, Vout* v, cudaStream_t s) {
    k_scale<Vin, Vout><<<grid_for(d), kThreads, 0, s>>>(chunks, d.R, w, scale, active, v);
    g_msd_launches += 1;
}

template <typename V>
void gm_xupdate(const GmresDims& d, const RowChunk* chunks, const V* Vb, long long vstride,
                const double2* y, const int* kconv, double2* x, cudaStream_t s) {
    k_xupdate<V><<<grid_for(d), kThreads, 0, s>>>(chunks, d.R, Vb, vstride, y, d.m, kconv, x);
    g_msd_launches += 1;
}

void gm_start(const GmresDims& d, const double2* rr, int hstride, const double* tol_abs, double* beta,
              double* vscale, double2* g, int* active, int* kconv, int* any_active, cudaStream_t s) {
    k_start<<<blocks_for(d.S, 128), 128, 0, s>>>(d.S, d.m, rr, hstride, tol_abs, beta, vscale, g, active,
                                                 kconv, any_active);
    g_msd_launches += 1;
}

void gm_givens(const GmresDims& d, int j, const double2* h1, const double2* h2, int hstride,
               const double2* wn2, const double* tol_cycle, double2* H, double2* cs, double2* sn,
               double2* g, double* vscale, int* active, int* kconv, int* iters, int* any_active,
               int* nonfinite, cudaStream_t s) {
    k_givens<<<blocks_for(d.S, 128), 128, 0, s>>>(d.S, d.m, j, h1, h2, hstride, wn2, tol_cycle, H, cs, sn,
                                                  g, vscale, active, kconv, iters, any_active, nonfinite);
    g_msd_launches += 1;
}

void gm_lsq(const GmresDims& d, const double2* H, const double2* g, const int* kconv, double2* y,
            cudaStream_t s) {
    k_lsq<<<blocks_for(d.S, 128), 128, 0, s>>>(d.S, d.m, H, g, kconv, y);
    g_msd_launches += 1;
}

void gm_residual(long long n, const double2* b, const double2* Ax, double2* r, cudaStream_t s) {
    k_residual<<<blocks_for(n, 256), 256, 0, s>>>(n, b, Ax, r);
    g_msd_launches += 1;
}
void gm_zero(long long n, double2* x, cudaStream_t s) {
    k_zero<<<blocks_for(n, 256), 256, 0, s>>>(n, x);
    g_msd_launches += 1;
}
void gm_cast_f32(long long n, const double2* a, float2* b, cudaStream_t s) {
    k_cast_f32<<<blocks_for(n, 256), 256, 0, s>>>(n, a, b);
    g_msd_launches += 1;
}

template void gm_multidot<double2>(const GmresDims&, const RowChunk*, const int*, const double2*, long long,
                                   int, const double2*, double2*, double2*, int, int, cudaStream_t);
template void gm_multidot<float2>(const GmresDims&, const RowChunk*, const int*, const float2*, long long,
                                  int, const float2*, double2*, double2*, int, int, cudaStream_t);
template void gm_update<double2>(const GmresDims&, const RowChunk*, const double2*, long long, int,
                                 const double2*, int, double2*, cudaStream_t);
template void gm_update<float2>(const GmresDims&, const RowChunk*, const float2*, long long, int,
                                const double2*, int, float2*, cudaStream_t);
template void gm_scale<double2, double2>(const GmresDims&, const RowChunk*, const double2*, const double*,
                                         const int*, double2*, cudaStream_t);
template void gm_scale<double2, float2>(const GmresDims&, const RowChunk*, const double2*, const double*,
                                        const int*, float2*, cudaStream_t);
template void gm_scale<float2, float2>(const GmresDims&, const RowChunk*, const float2*, const double*,
                                       const int*, float2*, cudaStream_t);
template void gm_xupdate<double2>(const GmresDims&, const RowChunk*, const double2*, long long,
                                  const double2*, const int*, double2*, cudaStream_t);
template void gm_xupdate<float2>(const GmresDims&, const RowChunk*, const float2*, long long,
                                 const double2*, const int*, double2*, cudaStream_t);
