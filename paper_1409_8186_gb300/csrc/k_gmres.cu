// K4: batched restarted GMRES on the device (section 5: preconditioned
// Krylov solve; the restarted GMRES call of section 6.2).
//
// A "system" is one (configuration, column) pair s = cfg*R + r; all systems
// advance in lock step (one block product per Arnoldi step serves all of
// them) and each carries its own Hessenberg matrix, Givens rotations and
// convergence state.
//
// Orthogonalisation is classical Gram-Schmidt with one selective
// re-orthogonalisation pass (Daniel-Gragg-Kaufman-Stewart criterion: repeat
// the projection when it left less than a fraction eta2 of ||w||^2, by
// default one half; the solver option reorth sets eta2).  Per-thread
// sums of dot products and updates run in the storage precision of the
// basis (FP32 for the inner sweeps of a mixed solve, whose FP64 pipe would
// otherwise bound them) and cross-thread reductions in FP64.  Vectors are
// [rows][R] with R innermost; reductions run over row chunks that never
// straddle two configurations; projections V^H w and updates w -= V h are
// tiled over (row chunk, group of basis vectors) so that long Krylov bases
// are read with the whole GPU.
//
// The Givens rotations of a new Hessenberg column form the first-order
// linear recurrence z_{i+1} = -conj(s_i) z_i + c_i h_{i+1} (z_0 = h_0,
// rotated entry i = c_i z_i + s_i h_{i+1}); it is evaluated with a
// parallel scan of affine maps over one CTA per system (warp shuffles, then
// across warps), so a step costs O(j / threads + log threads) instead of a
// j-long dependency chain.
#include "msd_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kI = 8;    // basis vectors per dot-product block
constexpr int kU = 16;   // basis vectors per update block

template <typename V> __device__ __forceinline__ double2 to_d2(V v) { return make_double2(v.x, v.y); }

// Column lanes RC = the smallest power of two >= min(R, 32), so that lanes
// of one column are xor-shuffle partners.
__host__ __device__ inline int col_lanes(int R) {
    int c = 1;
    while (c < R && c < 32) c *= 2;
    return c;
}

__device__ __forceinline__ void atomic_add_v(double2* p, double2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}
__device__ __forceinline__ void atomic_add_v(float2* p, double2 v) {
    atomicAdd(&p->x, (float)v.x);
    atomicAdd(&p->y, (float)v.y);
}

// Partial sums over one chunk of rows (blockIdx.x), columns of group
// blockIdx.y, and the kI "vectors" i in [blockIdx.z * kI, ...) of the
// list V_0..V_{nv-1} followed, when self != 0, by w itself:
//   part[chunk][i][r] = sum_rows conj(u_i[row][r]) * w[row][r].
// Systems with skip[s] != 0 contribute zeros.
template <typename V>
__global__ void k_dots_part(const RowChunk* __restrict__ chunks, int R, const V* __restrict__ Vb,
                            long long vstride, int nv, int self, const V* __restrict__ w,
                            const int* __restrict__ skip, int skipval, double2* __restrict__ part) {
    const RowChunk ch = chunks[blockIdx.x];
    const int RC = col_lanes(R);
    const int RY = blockDim.x / RC;  // kThreads and RC are powers of two
    const int tx = threadIdx.x % RC, ty = threadIdx.x / RC;
    const int r = blockIdx.y * RC + tx;
    const int i0 = blockIdx.z * kI;
    const int nvv = nv + self;
    constexpr int kWarps = kThreads / 32;
    __shared__ double2 red[kWarps][32][kI];
    // Per-thread sums run in the storage precision (a handful of rows per
    // thread); they are widened to FP64 for the cross-lane and cross-warp
    // reduction.  An FP32 basis therefore costs FP32 arithmetic: the FP64
    // pipe of this GPU is a small fraction of the FP32 one.
    typedef decltype(V{}.x) A;
    A ax[kI], ay[kI];
#pragma unroll
    for (int ii = 0; ii < kI; ++ii) ax[ii] = ay[ii] = A(0);
    const bool live = r < R && !(skip && skip[ch.cfg * R + r] == skipval);
    if (live) {
        for (long long row = ch.row0 + ty; row < ch.row1; row += RY) {
            const V wv = w[row * R + r];
#pragma unroll
            for (int ii = 0; ii < kI; ++ii) {
                const int i = i0 + ii;
                if (i < nvv) {
                    const V vv = i < nv ? Vb[(long long)i * vstride + row * R + r] : wv;
                    ax[ii] = fma(vv.x, wv.x, fma(vv.y, wv.y, ax[ii]));  // conj(v) * w
                    ay[ii] = fma(vv.x, wv.y, fma(-vv.y, wv.x, ay[ii]));
                }
            }
        }
    }
    // lanes lane and lane ^ off (off >= RC) hold the same column: fold them
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int ii = 0; ii < kI; ++ii) {
        // within a warp in the storage precision (at most 32 terms), across
        // warps and chunks in FP64
        for (int off = 16; off >= RC; off >>= 1) {
            ax[ii] += __shfl_xor_sync(0xffffffffu, ax[ii], off);
            ay[ii] += __shfl_xor_sync(0xffffffffu, ay[ii], off);
        }
        if (lane < RC) red[warp][lane][ii] = make_double2((double)ax[ii], (double)ay[ii]);
    }
    __syncthreads();
    // one thread per (column lane, vector) adds the warps' partials
    for (int t = threadIdx.x; t < RC * kI; t += blockDim.x) {
        const int cl = t % RC, ii = t / RC;
        const int rr = blockIdx.y * RC + cl;
        if (rr >= R || i0 + ii >= nvv) continue;
        double2 s = make_double2(0.0, 0.0);
        for (int wv = 0; wv < kWarps; ++wv) {  // every warp carries all RC columns
            s.x += red[wv][cl][ii].x;
            s.y += red[wv][cl][ii].y;
        }
        part[((long long)blockIdx.x * nvv + (i0 + ii)) * R + rr] = s;
    }
}

// The same partial sums with one warp per vector i over the chunk's flat
// elements e = row * R + r (R divides 32, or R = 64): lane l reads elements
// e0 + l + 32 k, eight loads in flight, so a warp streams one contiguous
// stretch of its vector and of w.  The column of element e is e mod R, fixed
// per lane (Q = 1) or alternating between two columns (Q = 2, R = 64); lanes
// that hold the same column are folded by shuffles.  No block-level
// reduction: blocks are independent groups of eight vectors.
// Reduction of the chunk partials fused into the projection kernel (few
// systems): the last block of each group of vectors to finish sums that
// group's partials into out; with skip2 set, the last group to finish also
// takes the re-orthogonalisation decision (k_reorth_flags).  Counters start
// at zero and every last block puts its counter back to zero.
struct DotsFuse {
    int* cnt = nullptr;      // [gridDim.y] blocks finished per vector group (nullptr: no fusion)
    int* cnt_all = nullptr;  // vector groups finished
    const int* cfg_chunk_off = nullptr;
    int S = 0;
    double2* out = nullptr;
    int ostride = 0;
    // after the reduction, with wn2 set: wn2 = out[j + 1] - sum_{i <= j} |out[i]|^2
    // (||w - V h||^2 when out = V^H w with ||w||^2 at j + 1), and with skip2
    // also set the re-orthogonalisation flags (first projection)
    int j = 0;
    double2* wn2 = nullptr;
    const int* active = nullptr;
    int* skip2 = nullptr;
    double eta2 = 0.5;  // second pass when ||w'||^2 < eta2 ||w||^2
};

// ||w'||^2 = ||w||^2 - sum_{i <= j} |h_i|^2 and (skip2 != nullptr) the flag
// of one system, reduced over the CTA (every thread calls it).
__device__ void reorth_flag_cta(const double2* h, int j, double2* wn2, int act, int* skip2, double eta2) {
    double acc = 0.0;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) {
        const double2 v = __ldcg(h + i);
        acc += cabs2(v);
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    __shared__ double red[32];  // one slot per warp (blocks of up to 1024 threads)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double ss = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) ss += red[k];
        const double before = __ldcg(h + j + 1).x;  // ||w||^2 before the projection
        const double after = before - ss;
        *wn2 = make_double2(after, 0.0);
        if (skip2) *skip2 = !(act && after < eta2 * before);
    }
}

template <typename V, int Q>
__global__ void __launch_bounds__(kThreads, 4) k_dots_warp(const RowChunk* __restrict__ chunks, int R,
                                                        const V* __restrict__ Vb, long long vstride, int nv,
                                                        int self, const V* __restrict__ w,
                                                        const int* __restrict__ skip, int skipval,
                                                        double2* __restrict__ part, DotsFuse fz) {
    const RowChunk ch = chunks[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.y * (kThreads / 32) + warp;
    const int nvv = nv + self;
    const long long e0 = ch.row0 * R, e1 = ch.row1 * R;
    if (i < nvv) {  // a whole warp
        const V* u = i < nv ? Vb + (long long)i * vstride : w;
        // systems with skip set (no second projection) need no sums: a warp
        // whose columns are all skipped only writes its zeros
        bool live = true;
        if (skip) {
            live = false;
#pragma unroll
            for (int q = 0; q < Q; ++q) live |= skip[ch.cfg * R + (int)((e0 + lane + 32 * q) % R)] != skipval;
            live = __any_sync(0xffffffffu, live);
            if (!live) {
#pragma unroll
                for (int q = 0; q < Q; ++q)
                    if (Q == 2 || lane < R)
                        part[((long long)blockIdx.x * nvv + i) * R + (int)((e0 + lane + 32 * q) % R)] =
                            make_double2(0.0, 0.0);
            }
        }
        if (live) {
            typedef decltype(V{}.x) A;
            A ax[Q], ay[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) ax[q] = ay[q] = A(0);
            // loads in flight per lane: a multiple of Q (the column phase of k
            // survives the stride); 16 complex64 = the whole 512-row chunk of
            // one column in a single round trip
            constexpr int U = sizeof(V) == 8 ? 16 : 8;
            long long e = e0 + lane;
            for (; e + 32LL * (U - 1) < e1; e += 32LL * U) {
                V uv[U], wv[U];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    uv[k] = u[e + 32LL * k];
                    wv[k] = w[e + 32LL * k];
                }
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    const int q = k % Q;
                    ax[q] = fma(uv[k].x, wv[k].x, fma(uv[k].y, wv[k].y, ax[q]));  // conj(u) * w
                    ay[q] = fma(uv[k].x, wv[k].y, fma(-uv[k].y, wv[k].x, ay[q]));
                }
            }
            for (int k = 0; e < e1; e += 32, ++k) {
                const V uv = u[e], wv = w[e];
                if (Q == 2 && (k & 1)) {
                    ax[Q - 1] = fma(uv.x, wv.x, fma(uv.y, wv.y, ax[Q - 1]));
                    ay[Q - 1] = fma(uv.x, wv.y, fma(-uv.y, wv.x, ay[Q - 1]));
                } else {
                    ax[0] = fma(uv.x, wv.x, fma(uv.y, wv.y, ax[0]));
                    ay[0] = fma(uv.x, wv.y, fma(-uv.y, wv.x, ay[0]));
                }
            }
            if (Q == 1) {
                for (int off = 16; off >= R; off >>= 1) {
                    ax[0] += __shfl_xor_sync(0xffffffffu, ax[0], off);
                    ay[0] += __shfl_xor_sync(0xffffffffu, ay[0], off);
                }
            }
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                if (Q == 1 && lane >= R) break;
                const int r = (int)((e0 + lane + 32 * q) % R);
                const bool sk = skip && skip[ch.cfg * R + r] == skipval;
                part[((long long)blockIdx.x * nvv + i) * R + r] =
                    sk ? make_double2(0.0, 0.0) : make_double2((double)ax[q], (double)ay[q]);
            }
        }
    }
    if (!fz.cnt) return;
    // ---- fused reduction of this vector group (last block of the group)
    __shared__ int last;
    if (Q == 2 || lane < R) __threadfence();  // the lanes that wrote partial sums
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&fz.cnt[blockIdx.y], 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    constexpr int WPB = kThreads / 32;
    const int ib = blockIdx.y * WPB;
    for (int o = warp; o < fz.S * WPB; o += WPB) {
        const int sy = o / WPB, iv = ib + o % WPB;
        if (iv >= nvv) continue;  // a whole warp
        const int c = sy / R, r = sy % R;
        double2 acc = make_double2(0.0, 0.0);
        for (int k = fz.cfg_chunk_off[c] + lane; k < fz.cfg_chunk_off[c + 1]; k += 32) {
            const double2 v = __ldcg(part + ((long long)k * nvv + iv) * R + r);
            acc.x += v.x;
            acc.y += v.y;
        }
        for (int off = 16; off > 0; off >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        }
        if (lane == 0) fz.out[(long long)sy * fz.ostride + iv] = acc;
    }
    if (threadIdx.x == 0) fz.cnt[blockIdx.y] = 0;
    if (!fz.wn2) return;
    // ---- norm after the projection, re-orthogonalisation flags (last vector group to finish)
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(fz.cnt_all, 1) == (int)gridDim.y - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int sy = 0; sy < fz.S; ++sy)
        reorth_flag_cta(fz.out + (long long)sy * fz.ostride, fz.j, fz.wn2 + (long long)sy * fz.ostride,
                        fz.active ? fz.active[sy] : 1, fz.skip2 ? fz.skip2 + sy : nullptr, fz.eta2);
    if (threadIdx.x == 0) *fz.cnt_all = 0;
}

// out[s * ostride + i] = sum over the chunks of cfg(s) of part[chunk][i][r]
// (one warp per output: the lanes stride over the chunks, then shuffle-add)
// With tail.cnt set (few systems), the last block to finish also forms
// wn2[s] = out[s][j + 1] - sum_{i <= j} |out[s][i]|^2 and, with tail.skip2,
// the re-orthogonalisation flags (k_reorth_flags), and puts the counter back
// to zero.
struct FinTail {
    int* cnt = nullptr;
    int j = 0;
    double2* wn2 = nullptr;
    const int* active = nullptr;
    int* skip2 = nullptr;
    double eta2 = 0.5;  // second pass when ||w'||^2 < eta2 ||w||^2
};
__global__ void k_dots_fin(int C, int R, int nvv, const int* __restrict__ cfg_chunk_off,
                           const double2* __restrict__ part, double2* __restrict__ out, int ostride, FinTail tail) {
    const long long idx = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (idx < (long long)C * R * nvv) {  // uniform across the warp
        const int i = (int)(idx % nvv);
        const int s = (int)(idx / nvv);
        const int c = s / R, r = s % R;
        double2 acc = make_double2(0.0, 0.0);
        for (int k = cfg_chunk_off[c] + lane; k < cfg_chunk_off[c + 1]; k += 32) {
            const double2 v = part[((long long)k * nvv + i) * R + r];
            acc.x += v.x;
            acc.y += v.y;
        }
        for (int off = 16; off > 0; off >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
        }
        if (lane == 0) {
            out[(long long)s * ostride + i] = acc;
            if (tail.cnt) __threadfence();
        }
    }
    if (!tail.cnt) return;
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(tail.cnt, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int S = C * R;
    for (int sy = 0; sy < S; ++sy)
        reorth_flag_cta(out + (long long)sy * ostride, tail.j, tail.wn2 + (long long)sy * ostride,
                        tail.active ? tail.active[sy] : 1, tail.skip2 ? tail.skip2 + sy : nullptr, tail.eta2);
    if (threadIdx.x == 0) *tail.cnt = 0;
}

// w[row][r] += sign * sum_{i in block's group, i < nv} V_i[row][r] h[s][i].
// The block's slice of h (times sign) is staged in shared memory in the
// basis storage type and the sums run in that precision (FP32 for an FP32
// basis: the correction it builds only needs the accuracy of the FP32
// sweep).  With more than one vector group the groups meet in atomics;
// with one group the result is stored directly.
template <typename V, typename W>
__global__ void __launch_bounds__(kThreads, 4)
    k_update(const RowChunk* __restrict__ chunks, int R, const V* __restrict__ Vb, long long vstride,
                         int nv, const double2* __restrict__ h, int hstride, const int* __restrict__ skip,
                         int skipval, double sign, W* __restrict__ w) {
    typedef decltype(V{}.x) A;
    const RowChunk ch = chunks[blockIdx.x];
    const int RC = col_lanes(R);
    const int RY = blockDim.x / RC;
    const int tx = threadIdx.x % RC, ty = threadIdx.x / RC;
    const int r = blockIdx.y * RC + tx;
    const int i0 = blockIdx.z * kU;
    const int i1 = min(nv, i0 + kU);
    __shared__ V hsm[kU][32];
    for (int t = threadIdx.x; t < kU * RC; t += blockDim.x) {
        const int ii = t / RC, cl = t % RC;
        const int rr = blockIdx.y * RC + cl;
        double2 v = make_double2(0.0, 0.0);
        if (rr < R && i0 + ii < i1) v = h[(long long)(ch.cfg * R + rr) * hstride + i0 + ii];
        hsm[ii][cl] = V{(A)(sign * v.x), (A)(sign * v.y)};
    }
    __syncthreads();
    if (r >= R || i0 >= i1) return;
    if (skip && skip[ch.cfg * R + r] == skipval) return;
    const bool atomic = gridDim.z > 1;
    const int cnt = i1 - i0;
    for (long long row = ch.row0 + ty; row < ch.row1; row += RY) {
        A ax[4] = {A(0), A(0), A(0), A(0)}, ay[4] = {A(0), A(0), A(0), A(0)};
        const V* vp = Vb + (long long)i0 * vstride + row * R + r;
        // all kU loads of the row in flight before the multiply-adds
        V vv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) vv[u] = u < cnt ? vp[(long long)u * vstride] : V{A(0), A(0)};
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const V hh = hsm[u][tx];  // zero beyond cnt
            ax[u & 3] = fma(vv[u].x, hh.x, fma(-vv[u].y, hh.y, ax[u & 3]));
            ay[u & 3] = fma(vv[u].x, hh.y, fma(vv[u].y, hh.x, ay[u & 3]));
        }
        const double2 d = make_double2((double)((ax[0] + ax[1]) + (ax[2] + ax[3])),
                                       (double)((ay[0] + ay[1]) + (ay[2] + ay[3])));
        W* p = w + row * R + r;
        if (atomic) {
            atomic_add_v(p, d);
        } else {
            const double2 o = to_d2(*p);
            *p = W{(decltype(W{}.x))(o.x + d.x), (decltype(W{}.x))(o.y + d.y)};
        }
    }
}

// v = w * scale[s] for active systems, 0 otherwise; with xs (FP32 basis),
// also xs = rf .* v, the scaled columns the next product reads (the
// arithmetic of k_scale_cols on the stored v).
template <typename Vin, typename Vout>
__global__ void k_scale(const RowChunk* __restrict__ chunks, int R, const Vin* __restrict__ w,
                        const double* __restrict__ scale, const int* __restrict__ active,
                        Vout* __restrict__ v, const float* __restrict__ rf, float2* __restrict__ xs) {
    const RowChunk ch = chunks[blockIdx.x];
    const int RC = col_lanes(R);
    const int RY = blockDim.x / RC;
    const int tx = threadIdx.x % RC, ty = threadIdx.x / RC;
    const int r = blockIdx.y * RC + tx;
    if (ty >= RY || r >= R) return;
    const int s = ch.cfg * R + r;
    // arithmetic in the wider of the two storage types (FP32 for an FP32 basis)
    typedef decltype(Vin{}.x + Vout{}.x) A;
    const A f = (A)(active[s] ? scale[s] : 0.0);
    for (long long row = ch.row0 + ty; row < ch.row1; row += RY) {
        const Vin a = w[row * R + r];
        const Vout o = Vout{(decltype(Vout{}.x))((A)a.x * f), (decltype(Vout{}.x))((A)a.y * f)};
        v[row * R + r] = o;
        if (xs) {
            const float c = rf[row];
            xs[row * R + r] = make_float2(c * (float)o.x, c * (float)o.y);
        }
    }
}

// Selective re-orthogonalisation flags, one CTA per system: ||w'||^2 after
// the first projection is ||w||^2 - sum_i |h_i|^2 (Pythagoras, V orthonormal);
// need[s] = 1 for an active system where that is below ||w||^2 / 2.  The
// estimate is written to wn2 (the subdiagonal when no second pass runs);
// where cancellation makes it inaccurate the second pass runs and measures
// the norm itself.
__global__ void k_reorth_flags(int S, const double2* __restrict__ h1, int hstride, int j,
                               double2* __restrict__ wn2, const int* __restrict__ active,
                               int* __restrict__ skip2, double eta2) {
    const int s = blockIdx.x;
    const double2* h = h1 + (long long)s * hstride;
    double acc = 0.0;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) acc += cabs2(h[i]);
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    __shared__ double part[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double ss = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) ss += part[k];
    const double before = h[j + 1].x;  // ||w||^2 before the projection
    const double after = before - ss;
    wn2[(long long)s * hstride] = make_double2(after, 0.0);
    skip2[s] = !(active[s] && after < eta2 * before);
}

// Start of a cycle: beta = ||r||; systems whose residual already meets
// tol_abs are done.  g = [beta, 0, ...], scale = 1/beta.
__global__ void k_start(int S, int m, const double2* __restrict__ rr, int hstride,
                        const double* __restrict__ tol_abs, double* __restrict__ beta_out,
                        double* __restrict__ vscale, double2* __restrict__ g, int* __restrict__ active,
                        int* __restrict__ kconv, int* __restrict__ any_active) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const double beta = sqrt(fmax(rr[(long long)s * hstride].x, 0.0));
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

// affine map z -> A z + B (complex); compose(second, first) = second o first
struct Aff {
    double2 A, B;
};
__device__ __forceinline__ Aff compose(const Aff& second, const Aff& first) {
    return Aff{cmul(second.A, first.A), cadd(cmul(second.A, first.B), second.B)};
}
// the same maps in FP32 (z_j of the FP32 inner sweeps of a mixed solve)
struct AffF {
    float2 A, B;
};
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ AffF compose(const AffF& second, const AffF& first) {
    const float2 ab = cmulf(second.A, first.B);
    return AffF{cmulf(second.A, first.A), make_float2(ab.x + second.B.x, ab.y + second.B.y)};
}
template <typename M> struct AffOps;
template <> struct AffOps<Aff> {
    __device__ static Aff id() { return Aff{make_double2(1.0, 0.0), make_double2(0.0, 0.0)}; }
    __device__ static Aff step(double2 c, double2 sv, double2 hn1) {
        return Aff{cscale(cconj(sv), -1.0), cscale(hn1, c.x)};
    }
    __device__ static double2 apply(const Aff& f, double2 z) { return cadd(cmul(f.A, z), f.B); }
};
template <> struct AffOps<AffF> {
    __device__ static AffF id() { return AffF{make_float2(1.f, 0.f), make_float2(0.f, 0.f)}; }
    __device__ static AffF step(double2 c, double2 sv, double2 hn1) {
        return AffF{make_float2((float)-sv.x, (float)sv.y), make_float2((float)(hn1.x * c.x), (float)(hn1.y * c.x))};
    }
    __device__ static double2 apply(const AffF& f, double2 z) {
        const float2 r = cmulf(f.A, make_float2((float)z.x, (float)z.y));
        return make_double2((double)r.x + f.B.x, (double)r.y + f.B.y);
    }
};

// Arnoldi step j for one system per CTA: column h = h1 + h2 (h2 only where
// the second projection ran), h[j+1] = ||w||.  The step needs only the last
// entry z_j of the rotated column (for the new rotation and the residual
// estimate): z_j = A_{j-1}(...A_0(h_0)) with A_i(z) = c_i h_{i+1} -
// conj(s_i) z, an ordered reduction of affine maps over the CTA, in FP64
// (Map = Aff) or, for the FP32 inner sweeps of a mixed solve, in FP32 (Map =
// AffF: a warp-wide FP64 instruction costs ~64 cycles of an SM sub-partition
// on this GPU, and the chain made the step ~20 us).  The rotation itself is
// formed in FP64.  The raw column is stored; k_apply_rotations rotates all
// columns at the end of the cycle in FP64, in parallel across columns.
// Warp-shuffle transfer of the maps (lane + off -> lane).
__device__ __forceinline__ Aff shfl_down(const Aff& f, int off) {
    return Aff{make_double2(__shfl_down_sync(0xffffffffu, f.A.x, off), __shfl_down_sync(0xffffffffu, f.A.y, off)),
               make_double2(__shfl_down_sync(0xffffffffu, f.B.x, off), __shfl_down_sync(0xffffffffu, f.B.y, off))};
}
__device__ __forceinline__ AffF shfl_down(const AffF& f, int off) {
    return AffF{make_float2(__shfl_down_sync(0xffffffffu, f.A.x, off), __shfl_down_sync(0xffffffffu, f.A.y, off)),
                make_float2(__shfl_down_sync(0xffffffffu, f.B.x, off), __shfl_down_sync(0xffffffffu, f.B.y, off))};
}
// Ordered reduction over the 32 lanes of a warp: lane 0 receives
// f_31 o ... o f_1 o f_0 (later lanes compose onto earlier ones).
template <typename Map>
__device__ __forceinline__ Map warp_compose(Map f) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < 32; off *= 2) {
        const Map later = shfl_down(f, off);
        if ((lane & (2 * off - 1)) == 0) f = compose(later, f);
    }
    return f;
}

constexpr int kGivensThreads = 1024;

template <typename Map>
__global__ void __launch_bounds__(kGivensThreads) k_givens(int m, int j, const double2* __restrict__ h1,
                                                     const double2* __restrict__ h2, int hstride,
                                                     const double2* __restrict__ wn2a,
                                                     const double2* __restrict__ wn2b,
                                                     const int* __restrict__ skip2,
                                                     const double* __restrict__ tol_cycle,
                                                     double2* __restrict__ H, double2* __restrict__ cs,
                                                     double2* __restrict__ sn, double2* __restrict__ g,
                                                     double* __restrict__ vscale, int* __restrict__ active,
                                                     int* __restrict__ kconv, int* __restrict__ iters,
                                                     int* __restrict__ any_active, int* __restrict__ nonfinite,
                                                     double2* __restrict__ rdiag) {
    const int s = blockIdx.x;
    if (!active[s]) return;
    __shared__ Map red[kGivensThreads / 32];
    const int tid = threadIdx.x, T = blockDim.x;
    const bool second = !skip2[s];
    const double2* a = h1 + (long long)s * hstride;
    const double2* b = h2 + (long long)s * hstride;
    const double2* csj = cs + (long long)s * m;
    const double2* snj = sn + (long long)s * m;
    double2* Hc = H + ((long long)s * m + j) * (m + 1);  // column j, rows 0..j+1
    auto hval = [&](int i) {
        double2 v = a[i];
        if (second) v = cadd(v, b[i]);
        return v;
    };
    // operands of the tail, loaded before the reduction so that their
    // latency overlaps it (thread 0 finishes the step)
    double wn = 0.0, tol = 0.0;
    double2 h0 = make_double2(0.0, 0.0), gj = make_double2(0.0, 0.0);
    if (tid == 0) {
        wn = second ? wn2b[(long long)s * hstride].x : wn2a[(long long)s * hstride].x;
        tol = tol_cycle[s];
        h0 = hval(0);
        gj = g[(long long)s * (m + 1) + j];
    }
    for (int i = tid; i <= j; i += T) Hc[i] = hval(i);  // raw column
    // segment of rotations [lo, hi) owned by this thread
    const int per = (j + T - 1) / T;
    const int lo = min(j, tid * per), hi = min(j, lo + per);
    Map seg = AffOps<Map>::id();
    for (int i = lo; i < hi; ++i) seg = compose(AffOps<Map>::step(csj[i], snj[i], hval(i + 1)), seg);
    // ordered reduction: within each warp by shuffles, then over the warps
    seg = warp_compose(seg);
    const int nw = T >> 5;
    if ((tid & 31) == 0) red[tid >> 5] = seg;
    __syncthreads();
    if (tid >= 32) return;
    seg = tid < nw ? red[tid] : AffOps<Map>::id();
    seg = warp_compose(seg);
    if (tid != 0) return;
    const double2 hjj = AffOps<Map>::apply(seg, h0);
    // rotation c = |hjj| / den, s = (hjj / |hjj|) hn / den, den^2 = |hjj|^2 + hn^2,
    // from reciprocal square roots (the FP64 pipe of this GPU is narrow, and
    // this chain runs on one thread): 1/|hjj|, 1/den, 1/hn
    wn = fmax(wn, 0.0);
    const double a2 = cabs2(hjj);
    const double rw = wn > 0.0 ? rsqrt(wn) : 0.0;
    const double hn = wn * rw;
    double2 c, sv;
    if (a2 + wn == 0.0) {
        c = make_double2(1.0, 0.0);
        sv = make_double2(0.0, 0.0);
    } else if (a2 == 0.0) {
        c = make_double2(0.0, 0.0);
        sv = make_double2(1.0, 0.0);  // hn real and positive
    } else {
        const double ra = rsqrt(a2), rd = rsqrt(a2 + wn);
        c = make_double2(a2 * ra * rd, 0.0);
        sv = cscale(hjj, hn * ra * rd);  // ph * conj(hn) / den, hn real
    }
    cs[(long long)s * m + j] = c;
    sn[(long long)s * m + j] = sv;
    const double2 rjj = cadd(cscale(hjj, c.x), cscale(sv, hn));
    rdiag[(long long)s * m + j] = make_double2(hn, 0.0);  // R_jj is formed in FP64 at the end of the cycle
    double2* gs = g + (long long)s * (m + 1);
    const double2 gn = cscale(cmul(cconj(sv), gj), -1.0);
    gs[j + 1] = gn;
    gs[j] = cscale(gj, c.x);
    iters[s] += 1;
    const double res2 = cabs2(gn);  // squared residual estimate
    const bool bad = !isfinite(res2) || !isfinite(rjj.x) || !isfinite(rjj.y);
    if (bad) *nonfinite = 1;  // every writer stores the same value (the flag may live in host memory)
    if (bad || res2 <= tol * tol || hn == 0.0 || j + 1 == m) {
        active[s] = 0;
        kconv[s] = j + 1;
        vscale[s] = 0.0;
    } else {
        vscale[s] = rw;
        *any_active = 1;
    }
}

// End of a cycle: rotate every stored column j < kconv (raw h_0..h_j) by the
// rotations 0..j-1 into the triangle R, in FP64, and form R_jj from the
// rotated z_j with rotation j and the stored subdiagonal ||w_j||; one thread
// per column, all columns and systems in parallel.
__global__ void k_apply_rotations(int m, double2* __restrict__ H, const double2* __restrict__ cs,
                                  const double2* __restrict__ sn, const double2* __restrict__ rdiag,
                                  const int* __restrict__ kconv) {
    const int s = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kconv[s]) return;
    double2* Hc = H + ((long long)s * m + j) * (m + 1);
    const double2* csj = cs + (long long)s * m;
    const double2* snj = sn + (long long)s * m;
    double2 z = Hc[0];
    for (int i = 0; i < j; ++i) {
        const double2 c = csj[i], sv = snj[i], hn1 = Hc[i + 1];
        Hc[i] = cadd(cscale(z, c.x), cmul(sv, hn1));
        z = csub(cscale(hn1, c.x), cmul(cconj(sv), z));
    }
    // R_jj = c_j z_j + s_j ||w_j|| (the subdiagonal entry, real)
    Hc[j] = cadd(cscale(z, csj[j].x), cscale(snj[j], rdiag[(long long)s * m + j].x));
    Hc[j + 1] = make_double2(0.0, 0.0);
}

// Back substitution H y = g on the leading kconv x kconv triangle, one CTA
// per system: column-oriented, the CTA updates the remaining right-hand
// side in parallel after each pivot.
__global__ void __launch_bounds__(kThreads) k_lsq(int m, const double2* __restrict__ H,
                                                  const double2* __restrict__ g, const int* __restrict__ kconv,
                                                  double2* __restrict__ y, double2* __restrict__ work) {
    const int s = blockIdx.x;
    const int k = kconv[s];
    double2* ys = y + (long long)s * m;
    // the x update sweeps every column of the cycle: zero what this system did not use
    for (int i = k + threadIdx.x; i < m; i += blockDim.x) ys[i] = make_double2(0.0, 0.0);
    if (k == 0) return;
    const double2* Hs = H + (long long)s * m * (m + 1);
    double2* rhs = work + (long long)s * (m + 1);
    for (int i = threadIdx.x; i < k; i += blockDim.x) rhs[i] = g[(long long)s * (m + 1) + i];
    __shared__ double2 yi_sh;
    __syncthreads();
    for (int i = k - 1; i >= 0; --i) {
        if (threadIdx.x == 0) {
            const double2 d = Hs[(long long)i * (m + 1) + i];
            const double2 v = (d.x == 0.0 && d.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(rhs[i], d);
            ys[i] = v;
            yi_sh = v;
        }
        __syncthreads();
        const double2 v = yi_sh;
        const double2* col = Hs + (long long)i * (m + 1);
        for (int t = threadIdx.x; t < i; t += blockDim.x) rhs[t] = csub(rhs[t], cmul(col[t], v));
        __syncthreads();
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

inline unsigned blocks_for(long long n, int th) { return (unsigned)((n + th - 1) / th); }
inline unsigned rgroups(int R) { return (unsigned)((R + col_lanes(R) - 1) / col_lanes(R)); }

}  // namespace

// ---------------------------------------------------------------- host wrappers

template <typename V>
bool gm_dots(const GmresDims& d, const RowChunk* chunks, const int* cfg_chunk_off, const V* Vb, long long vstride,
             int nv, int self, const V* w, const int* skip, double2* part, double2* out, int ostride,
             cudaStream_t s, int skipval, const GmDotsFuse* fuse) {
    const int nvv = nv + self;
    constexpr int WPB = kThreads / 32;
    const bool warp_kernel = 32 % d.R == 0 || d.R == 64;
    // fused reduction inside the projection kernel: few systems and one
    // group of vectors (a fence and an atomic per block only pay off for
    // small grids); otherwise the reduction kernel takes the norm and the
    // flags in its last block
    const bool few = fuse && d.S <= kFuseMaxSystems;
    const bool fused = few && warp_kernel && (nvv + WPB - 1) / WPB == 1;
    DotsFuse fz;
    if (fused) {
        fz.cnt = fuse->cnt;
        fz.cnt_all = fuse->cnt + fuse->ncnt;
        fz.cfg_chunk_off = cfg_chunk_off;
        fz.S = d.S;
        fz.out = out;
        fz.ostride = ostride;
        if (fuse->wn2) {
            fz.j = fuse->j;
            fz.wn2 = fuse->wn2;
            fz.active = fuse->active;
            fz.skip2 = fuse->skip2;
            fz.eta2 = fuse->eta2;
        }
    }
    if (32 % d.R == 0) {
        k_dots_warp<V, 1><<<dim3(d.nchunk, (nvv + WPB - 1) / WPB), kThreads, 0, s>>>(chunks, d.R, Vb, vstride, nv,
                                                                                    self, w, skip, skipval, part, fz);
    } else if (d.R == 64) {
        k_dots_warp<V, 2><<<dim3(d.nchunk, (nvv + WPB - 1) / WPB), kThreads, 0, s>>>(chunks, d.R, Vb, vstride, nv,
                                                                                    self, w, skip, skipval, part, fz);
    } else {
        dim3 g(d.nchunk, rgroups(d.R), (nvv + kI - 1) / kI);
        k_dots_part<V><<<g, kThreads, 0, s>>>(chunks, d.R, Vb, vstride, nv, self, w, skip, skipval, part);
    }
    if (fused) {
        g_msd_launches += 1;
        return true;
    }
    const long long tot = (long long)d.S * nvv;
    FinTail tail;
    const bool tail_done = few && fuse->wn2;
    if (tail_done) {
        tail.cnt = fuse->cnt + fuse->ncnt;
        tail.j = fuse->j;
        tail.wn2 = fuse->wn2;
        tail.active = fuse->active;
        tail.skip2 = fuse->skip2;
        tail.eta2 = fuse->eta2;
    }
    k_dots_fin<<<blocks_for(tot * 32, 128), 128, 0, s>>>(d.C, d.R, nvv, cfg_chunk_off, part, out, ostride, tail);
    g_msd_launches += 2;
    return tail_done;
}

template <typename V, typename W>
void gm_update(const GmresDims& d, const RowChunk* chunks, const V* Vb, long long vstride, int nv, const double2* h,
               int hstride, const int* skip, double sign, W* w, cudaStream_t s, int skipval) {
    if (nv <= 0) return;
    dim3 g(d.nchunk, rgroups(d.R), (nv + kU - 1) / kU);
    k_update<V, W><<<g, kThreads, 0, s>>>(chunks, d.R, Vb, vstride, nv, h, hstride, skip, skipval, sign, w);
    g_msd_launches += 1;
}

template <typename Vin, typename Vout>
void gm_scale(const GmresDims& d, const RowChunk* chunks, const Vin* w, const double* scale, const int* active,
              Vout* v, cudaStream_t s, const float* rf, float2* xs) {
    k_scale<Vin, Vout><<<dim3(d.nchunk, rgroups(d.R)), kThreads, 0, s>>>(chunks, d.R, w, scale, active, v, rf, xs);
    g_msd_launches += 1;
}

void gm_reorth_flags(const GmresDims& d, const double2* h1, int hstride, int j, double2* wn2,
                     const int* active, int* skip2, cudaStream_t s, double eta2) {
    k_reorth_flags<<<d.S, 128, 0, s>>>(d.S, h1, hstride, j, wn2, active, skip2, eta2);
    g_msd_launches += 1;
}

void gm_start(const GmresDims& d, const double2* rr, int hstride, const double* tol_abs, double* beta,
              double* vscale, double2* g, int* active, int* kconv, int* any_active, cudaStream_t s) {
    k_start<<<blocks_for(d.S, 128), 128, 0, s>>>(d.S, d.m, rr, hstride, tol_abs, beta, vscale, g, active, kconv,
                                                 any_active);
    g_msd_launches += 1;
}

// Threads of the Givens step: about two rotations per thread, whole warps.
static int givens_threads(int j) {
    const int t = ((j + 1) / 2 + 31) / 32 * 32;
    return std::min(kGivensThreads, std::max(32, t));
}

void gm_givens(const GmresDims& d, int j, const double2* h1, const double2* h2, int hstride, const double2* wn2a,
               const double2* wn2b, const int* skip2, const double* tol_cycle, double2* H, double2* cs,
               double2* sn, double2* g, double* vscale, int* active, int* kconv, int* iters, int* any_active,
               int* nonfinite, double2* rdiag, bool fp32_maps, cudaStream_t s) {
    if (fp32_maps)
        k_givens<AffF><<<d.S, givens_threads(j), 0, s>>>(d.m, j, h1, h2, hstride, wn2a, wn2b, skip2, tol_cycle, H,
                                                         cs, sn, g, vscale, active, kconv, iters, any_active,
                                                         nonfinite, rdiag);
    else
        k_givens<Aff><<<d.S, givens_threads(j), 0, s>>>(d.m, j, h1, h2, hstride, wn2a, wn2b, skip2, tol_cycle, H,
                                                        cs, sn, g, vscale, active, kconv, iters, any_active,
                                                        nonfinite, rdiag);
    g_msd_launches += 1;
}

void gm_lsq(const GmresDims& d, double2* H, const double2* cs, const double2* sn, const double2* rdiag,
            const double2* g, const int* kconv, double2* y, double2* work, cudaStream_t s) {
    k_apply_rotations<<<dim3(blocks_for(d.m, 128), d.S), 128, 0, s>>>(d.m, H, cs, sn, rdiag, kconv);
    k_lsq<<<d.S, kThreads, 0, s>>>(d.m, H, g, kconv, y, work);
    g_msd_launches += 2;
}

void gm_residual(long long n, const double2* b, const double2* Ax, double2* r, cudaStream_t s) {
    k_residual<<<blocks_for(n, 256), 256, 0, s>>>(n, b, Ax, r);
    g_msd_launches += 1;
}

void gm_zero(long long n, double2* x, cudaStream_t s) {
    k_zero<<<blocks_for(n, 256), 256, 0, s>>>(n, x);
    g_msd_launches += 1;
}

template bool gm_dots<double2>(const GmresDims&, const RowChunk*, const int*, const double2*, long long, int, int,
                               const double2*, const int*, double2*, double2*, int, cudaStream_t, int,
                               const GmDotsFuse*);
template bool gm_dots<float2>(const GmresDims&, const RowChunk*, const int*, const float2*, long long, int, int,
                              const float2*, const int*, double2*, double2*, int, cudaStream_t, int,
                              const GmDotsFuse*);
template void gm_update<double2, double2>(const GmresDims&, const RowChunk*, const double2*, long long, int,
                                          const double2*, int, const int*, double, double2*, cudaStream_t, int);
template void gm_update<float2, float2>(const GmresDims&, const RowChunk*, const float2*, long long, int,
                                        const double2*, int, const int*, double, float2*, cudaStream_t, int);
template void gm_update<float2, double2>(const GmresDims&, const RowChunk*, const float2*, long long, int,
                                         const double2*, int, const int*, double, double2*, cudaStream_t, int);
template void gm_scale<double2, double2>(const GmresDims&, const RowChunk*, const double2*, const double*,
                                         const int*, double2*, cudaStream_t, const float*, float2*);
template void gm_scale<double2, float2>(const GmresDims&, const RowChunk*, const double2*, const double*,
                                        const int*, float2*, cudaStream_t, const float*, float2*);
template void gm_scale<float2, float2>(const GmresDims&, const RowChunk*, const float2*, const double*, const int*,
                                       float2*, cudaStream_t, const float*, float2*);
