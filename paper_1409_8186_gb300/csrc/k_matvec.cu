// K3: block-Toeplitz product of the single-scattering-preconditioned
// operator (section 5, built from the blocks of section 4.2):
//
//   y^p_m = x^p_m + l^p_m * s^p_m,   s^p_m = sum_{q != p} sum_n g^pq_{n-m} xs^q_n,
//   xs^q_n = r^q_n x^q_n,
//
// for R right-hand sides at once.  Each off-diagonal block is the Toeplitz
// matrix (S^pq)^T with generator g^pq (4N+1 values), scaled by the Bessel
// diagonals; the dense block (n^2 entries) is never formed.
//
// Work decomposition: a CTA owns a tile of 32 target disks (one per lane),
// a contiguous range of source disks q, and RT columns.  Warps split the
// target modes into blocks of KB consecutive m (and the columns into groups
// of RB).  Per source q the CTA stages, double-buffered, the 32 generator
// rows g^{p q}_{.} (contiguous in the [q][p][l] layout: one bulk copy on an
// mbarrier) and the RT-column slab of xs^q (cp.async) into shared memory.
// Each thread then sweeps n with a register window of KB generator values
// (one new value per n, since neighbouring m need neighbouring l = n - m)
// and accumulates KB x RB complex sums.  The rows keep their odd length
// L = 4N + 1, so the 32 lanes (32 different rows) hit 32 different banks;
// the xs slab is a broadcast.  KB is chosen per truncation order so that
// ceil(n / KB) * KB wastes as few padded modes as possible.  Raw sums go to a
// per-split partial buffer; a finalize kernel adds the splits, applies
// l^p_m and adds x.
#include "msd_internal.cuh"

namespace {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async(void* dst, const float2* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async(void* dst, const double2* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int n>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(n)); }

template <typename V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }

// Shared-memory footprint (elements) of one stage: the 32 generator rows
// contiguous (as in HBM) between kGFront zeros before and kGBack zeros after
// (the register window reaches up to KB - 1 <= 8 values past either end of a
// row; past a row's end it reads the next row, which only ever meets zero
// source values or padded target modes), then the source slab, rounded to
// 16 bytes.
constexpr int kGFront = 8, kGBack = 16;
__host__ __device__ inline int stage_g_elems(int L, int KB) { return MSD_TILE_P * L + kGFront + kGBack; }
__host__ __device__ inline int stage_x_elems(int n, int RT, int KB) {
    return (((n + KB - 1) / KB) * KB * RT + 1) & ~1;
}

__device__ int g_bt_status;  // bit 0: a wait for a bulk copy of generators expired
constexpr long long kBtWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ bool bt_mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kBtWaitCycles) return false;
    }
}

// Complex multiply-accumulate policies over a KB x RB register tile.
// Mac4: the textbook product, 4 real FMAs per complex MAC (FP32 path).
template <typename V, int KB, int RB>
struct Mac4 {
    struct G { V g; };
    struct X { V x; };
    V acc[KB][RB];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int b = 0; b < KB; ++b)
#pragma unroll
            for (int r = 0; r < RB; ++r) acc[b][r] = vzero<V>();
    }
    __device__ __forceinline__ static G gen(V v) { return G{v}; }
    __device__ __forceinline__ static X src(V v) { return X{v}; }
    __device__ __forceinline__ void mac(int b, int r, const G& g, const X& x) { cfma(acc[b][r], g.g, x.x); }
    __device__ __forceinline__ V result(int b, int r) const { return acc[b][r]; }
};

// Mac3: Gauss's three-multiplication form, accumulated in three real sums
// (FP64 path, where the FP64 pipe is the bound).  With g = c + i d and
// x = a + i b:  k1 += c (a + b),  k2 += a (d - c),  k3 += b (c + d);
// then Re = k1 - k3, Im = k1 + k2.  The sums c+d, d-c are formed once per
// generator value entering the register window and a+b once per source
// value, so a complex MAC costs 3 FMAs instead of 4.
template <typename V, int KB, int RB>
struct Mac3 {
    struct G { double c, u, v; };
    struct X { double a, b, s; };
    double k1[KB][RB], k2[KB][RB], k3[KB][RB];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int b = 0; b < KB; ++b)
#pragma unroll
            for (int r = 0; r < RB; ++r) k1[b][r] = k2[b][r] = k3[b][r] = 0.0;
    }
    __device__ __forceinline__ static G gen(V v) { return G{v.x, v.y - v.x, v.x + v.y}; }
    __device__ __forceinline__ static X src(V v) { return X{v.x, v.y, v.x + v.y}; }
    __device__ __forceinline__ void mac(int b, int r, const G& g, const X& x) {
        k1[b][r] = fma(g.c, x.s, k1[b][r]);
        k2[b][r] = fma(x.a, g.u, k2[b][r]);
        k3[b][r] = fma(x.b, g.v, k3[b][r]);
    }
    __device__ __forceinline__ V result(int b, int r) const {
        return V{k1[b][r] - k3[b][r], k1[b][r] + k2[b][r]};
    }
};

// Mac2: the FP32 complex multiply-add as two paired FMAs (fma.rn.f32x2, one
// instruction for the real and the imaginary part, IEEE round-to-nearest per
// lane): with g = gx + i gy and x = a + i b,
//   (re, im) += (gx, gy) * (a, a) + (-gy, gx) * (b, b).
// The pairs of g are formed once per generator value entering the register
// window and those of x once per source value, so the FP32 kernel, which is
// bound by instruction issue, issues half the FMA instructions of Mac4.
__device__ __forceinline__ unsigned long long pk2(float x, float y) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
template <int KB, int RB>
struct Mac2 {
    typedef unsigned long long P;
    struct G { P g1, g2; };
    struct X { P xa, xb; };
    P acc[KB][RB];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int b = 0; b < KB; ++b)
#pragma unroll
            for (int r = 0; r < RB; ++r) acc[b][r] = 0ull;  // (0.0f, 0.0f)
    }
    __device__ __forceinline__ static G gen(float2 v) { return G{pk2(v.x, v.y), pk2(-v.y, v.x)}; }
    __device__ __forceinline__ static X src(float2 v) { return X{pk2(v.x, v.x), pk2(v.y, v.y)}; }
    __device__ __forceinline__ void mac(int b, int r, const G& g, const X& x) {
        asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[b][r]) : "l"(g.g1), "l"(x.xa));
        asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[b][r]) : "l"(g.g2), "l"(x.xb));
    }
    __device__ __forceinline__ float2 result(int b, int r) const {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc[b][r]));
        return make_float2(lo, hi);
    }
};

template <typename V, int KB, int RB, int P> struct MacFor { typedef Mac4<V, KB, RB> type; };
template <int KB, int RB> struct MacFor<double2, KB, RB, 0> { typedef Mac3<double2, KB, RB> type; };
template <int KB, int RB> struct MacFor<float2, KB, RB, 1> { typedef Mac2<KB, RB> type; };

// S = 2: two shared-memory stages (the next source is staged while the
// current one is summed); S = 1: one stage, staged and then summed, for
// truncation orders whose two FP64 stages exceed the shared memory of a CTA.
template <typename V, int RT, int RB, int KB, int P, int S>
__global__ void __launch_bounds__(512, (RB == 1 && sizeof(V) == 8) ? 2 : 1) k_bt_matvec(const MsdConfig* __restrict__ cfgs,
                                                   const MatvecWork* __restrict__ works,
                                                   const V* __restrict__ G, const V* __restrict__ xs,
                                                   V* __restrict__ part, long long Ntot, int R, int rtiles,
                                                   const int* __restrict__ live) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* smem = reinterpret_cast<V*>(smem_raw);
    __shared__ __align__(8) uint64_t gfull[2];  // generator bulk copy of stage s landed

    const int wi = blockIdx.x / rtiles;
    const int rt = blockIdx.x % rtiles;
    const MatvecWork w = works[wi];
    const MsdConfig c = cfgs[w.cfg];
    const int N = c.N, n = c.n, L = c.L;
    const int I = (n + KB - 1) / KB;
    const int npad = I * KB;
    const int gsz = stage_g_elems(L, KB), xsz = stage_x_elems(n, RT, KB);
    V* gbuf[2] = {smem, smem + (S == 2 ? gsz + xsz : 0)};
    V* xbuf[2] = {smem + gsz, smem + (S == 2 ? 2 * gsz + xsz : gsz)};

    const int lane = threadIdx.x;  // target p0 + lane
    const int warp = threadIdx.y;
    const int nthreads = blockDim.x * blockDim.y;
    const int tid = warp * 32 + lane;
    // the launch sizes warps for the largest N of the batch: blocks beyond
    // this configuration's I m-blocks only help with staging
    const int Imax = blockDim.y / (RT / RB);
    const int mblk = warp % Imax;
    const int rgrp = warp / Imax;
    const bool mact = mblk < I;
    const int m0 = mblk * KB;
    const int c0 = rgrp * RB;  // first column of this thread within the tile
    const int col0 = rt * RT;  // first column of the tile

    // no active column in this tile (converged Krylov systems): zero raw
    // sums, no other work
    if (live) {
        bool any = false;
        for (int r = 0; r < RT; ++r) any |= live[w.cfg * R + col0 + r] != 0;
        if (!any) {
            const int p = w.p0 + lane;
            if (!w.pad && mact && p < c.M) {
                V* out = part + (long long)w.split * Ntot * R;
                for (int b = 0; b < KB; ++b)
                    if (m0 + b < n)
                        for (int r = 0; r < RB; ++r)
                            out[(c.row_off + (long long)p * n + m0 + b) * R + col0 + c0 + r] = vzero<V>();
            }
            return;
        }
    }

    // zero the padding of the stages once (staging never writes it)
    for (int s = 0; s < S; ++s) {
        for (int t = tid; t < kGFront + kGBack; t += nthreads)
            gbuf[s][t < kGFront ? t : MSD_TILE_P * L + t] = vzero<V>();
        for (int t = n * RT + tid; t < npad * RT; t += nthreads) xbuf[s][t] = vzero<V>();
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&gfull[s])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();

    // The 32 generator rows of a source are contiguous in HBM (32 L values):
    // one thread moves them with a single bulk copy that completes on the
    // stage's mbarrier.  Tiles that do not start on 16 bytes (never for the
    // layouts the library builds, whose offsets are even) are staged by
    // every thread with cp.async instead; alignment is the same for every
    // source of a CTA, so the choice is made once.
    const V* gsrc_cfg = G + c.gen_off + (long long)w.p0 * L;
    const unsigned gbytes = (unsigned)(MSD_TILE_P * L * sizeof(V));
    const bool bulk = (((uintptr_t)gsrc_cfg) & 15) == 0 && (((long long)c.Mp * L * sizeof(V)) & 15) == 0;
    auto stage = [&](int q, int s) {
        const V* src = gsrc_cfg + (long long)q * c.Mp * L;
        V* dst = gbuf[s] + kGFront;
        if (bulk) {
            if (tid == 0) {
                const uint32_t bar = smem_u32(&gfull[s]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(gbytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(dst)),
                    "l"(src), "r"(gbytes), "r"(bar)
                    : "memory");
            }
        } else {
            for (int t = tid; t < MSD_TILE_P * L; t += nthreads) cp_async(dst + t, src + t);
        }
        const V* xsrc = xs + (c.row_off + (long long)q * n) * R + col0;
        V* xd = xbuf[s];
        for (int t = tid; t < n * RT; t += nthreads) {
            const int rr = t / RT, cc = t - rr * RT;
            cp_async(xd + t, xsrc + (long long)rr * R + cc);
        }
    };

    typedef typename MacFor<V, KB, RB, P>::type Mac;
    Mac acc;
    acc.init();

    if (S == 2 && w.q0 < w.q1) stage(w.q0, 0);
    cp_commit();
    const int base = kGFront + 2 * N - m0;  // smem position of l' = n - m0 + 2N at n = 0 (row 0)
    bool waits_ok = true;
    for (int it = 0, q = w.q0; q < w.q1; ++it, ++q) {
        if (S == 2) {
            if (q + 1 < w.q1) stage(q + 1, (it + 1) & 1);
            cp_commit();
            cp_wait<1>();
        } else {
            stage(q, 0);
            cp_commit();
            cp_wait<0>();
        }
        const int sb = S == 2 ? (it & 1) : 0;
        // use number of stage sb: it / 2 (two stages) or it (one stage)
        if (bulk && waits_ok)
            waits_ok = bt_mbar_wait(smem_u32(&gfull[sb]), (uint32_t)((S == 2 ? (it >> 1) : it) & 1));
        __syncthreads();
        if (mact) {
            const V* gs = gbuf[sb] + lane * L + base;
            const V* xsl = xbuf[sb] + c0;
            typename Mac::G win[KB];
#pragma unroll
            for (int j = 1; j < KB; ++j) win[KB - j] = Mac::gen(gs[-j]);
            for (int nb = 0; nb < npad; nb += KB) {
#pragma unroll
                for (int u = 0; u < KB; ++u) {
                    win[u] = Mac::gen(gs[nb + u]);
                    typename Mac::X xv[RB];
#pragma unroll
                    for (int r = 0; r < RB; ++r) xv[r] = Mac::src(xsl[(nb + u) * RT + r]);
#pragma unroll
                    for (int b = 0; b < KB; ++b) {
#pragma unroll
                        for (int r = 0; r < RB; ++r) acc.mac(b, r, win[(u - b + KB) % KB], xv[r]);
                    }
                }
            }
        }
        __syncthreads();
    }
    cp_wait<0>();
    // an expired wait: the partial sums are not valid; the host reports it
    if (!waits_ok) atomicOr(&g_bt_status, 1);

    const int p = w.p0 + lane;
    if (mact && p < c.M) {
        V* out = part + (long long)w.split * Ntot * R;
#pragma unroll
        for (int b = 0; b < KB; ++b) {
            const int mi = m0 + b;
            if (mi < n) {
                const long long row = c.row_off + (long long)p * n + mi;
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const long long o = row * R + col0 + c0 + r;
                    const V v = acc.result(b, r);
                    if (w.pad) {  // a later source block of a recomputed product: accumulate
                        const V u = out[o];
                        out[o] = V{u.x + v.x, u.y + v.y};
                    } else {
                        out[o] = v;
                    }
                }
            }
        }
    }
}

// The single-column FP32 product without CTA barriers in the source loop:
// the generator stages are filled by bulk copies (full mbarriers) and
// released by every warp once it has swept them (empty mbarriers, one
// arrival per warp), and each thread reads the source values xs^q_n straight
// from global memory (one address for the whole warp: a broadcast from L1),
// zero for the padded modes n >= 2N+1.  Warps therefore drift apart by up to
// a stage instead of meeting twice per source.  Same window, sums and output
// as k_bt_matvec<float2, 1, 1, KB, P, 2>.
template <int KB, int P>
__global__ void __launch_bounds__(512, P ? 1 : 2) k_bt_matvec1(const MsdConfig* __restrict__ cfgs,
                                                       const MatvecWork* __restrict__ works,
                                                       const float2* __restrict__ G,
                                                       const float2* __restrict__ xs, float2* __restrict__ part,
                                                       long long Ntot, int R, int rtiles,
                                                       const int* __restrict__ live) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* smem = reinterpret_cast<float2*>(smem_raw);
    __shared__ __align__(8) uint64_t gfull[2], gempty[2];

    const int wi = blockIdx.x / rtiles;
    const int rt = blockIdx.x % rtiles;
    const MatvecWork w = works[wi];
    const MsdConfig c = cfgs[w.cfg];
    const int N = c.N, n = c.n, L = c.L;
    const int I = (n + KB - 1) / KB;
    const int npad = I * KB;
    const int gsz = stage_g_elems(L, KB);
    const int lane = threadIdx.x, warp = threadIdx.y;
    const int nwarps = blockDim.y;
    const int tid = warp * 32 + lane;
    const bool mact = warp < I;
    const int m0 = warp * KB;
    const int col0 = rt;

    if (live && live[w.cfg * R + col0] == 0) {
        const int p = w.p0 + lane;
        if (!w.pad && mact && p < c.M) {
            float2* out = part + (long long)w.split * Ntot * R;
            for (int b = 0; b < KB; ++b)
                if (m0 + b < n) out[(c.row_off + (long long)p * n + m0 + b) * R + col0] = make_float2(0.f, 0.f);
        }
        return;
    }
    float2* gbuf[2] = {smem, smem + gsz};
    for (int s = 0; s < 2; ++s)
        for (int t = tid; t < kGFront + kGBack; t += nwarps * 32)
            gbuf[s][t < kGFront ? t : MSD_TILE_P * L + t] = make_float2(0.f, 0.f);
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&gfull[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&gempty[s])), "r"(nwarps));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();

    const float2* gsrc_cfg = G + c.gen_off + (long long)w.p0 * L;
    const unsigned gbytes = (unsigned)(MSD_TILE_P * L * sizeof(float2));
    // alignment is the same for every source of a CTA (the plan builder only
    // offers this kernel where it holds; an unaligned tile is not staged and
    // the expired wait below reports the failure)
    const bool aligned = (((uintptr_t)gsrc_cfg) & 15) == 0 && (((long long)c.Mp * L * sizeof(float2)) & 15) == 0;
    auto issue = [&](int q, int s) {
        const uint32_t bar = smem_u32(&gfull[s]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(gbytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(gbuf[s] + kGFront)),
                     "l"(gsrc_cfg + (long long)q * c.Mp * L), "r"(gbytes), "r"(bar)
                     : "memory");
    };

    typedef typename MacFor<float2, KB, 1, P>::type Mac;
    Mac acc;
    acc.init();
    bool ok = aligned;
    int pending = -1;  // (thread 0) the last iteration whose stage was issued
    if (tid == 0 && ok && w.q0 < w.q1) {
        issue(w.q0, 0);
        pending = 0;
    }
    const int base = kGFront + 2 * N - m0;
    for (int it = 0, q = w.q0; q < w.q1; ++it, ++q) {
        const int sb = it & 1;
        // producer: the next source into the other stage once every warp has
        // released it (its use at it - 1)
        if (tid == 0 && ok && q + 1 < w.q1) {
            if (it >= 1) ok = bt_mbar_wait(smem_u32(&gempty[sb ^ 1]), (uint32_t)(((it - 1) >> 1) & 1));
            if (ok) {
                issue(q + 1, sb ^ 1);
                pending = it + 1;
            }
        }
        __syncwarp();
        bool here = ok;
        if (here) here = bt_mbar_wait(smem_u32(&gfull[sb]), (uint32_t)((it >> 1) & 1));
        here = __all_sync(0xffffffffu, here);
        if (!here) ok = false;
        if (ok && mact) {
            const float2* gs = gbuf[sb] + lane * L + base;
            const float2* xq = xs + (c.row_off + (long long)q * n) * R + col0;
            typename Mac::G win[KB];
#pragma unroll
            for (int j = 1; j < KB; ++j) win[KB - j] = Mac::gen(gs[-j]);
            for (int nb = 0; nb < npad; nb += KB) {
                float2 xr[KB];
#pragma unroll
                for (int u = 0; u < KB; ++u) xr[u] = nb + u < n ? __ldg(xq + (long long)(nb + u) * R) : make_float2(0.f, 0.f);
#pragma unroll
                for (int u = 0; u < KB; ++u) {
                    win[u] = Mac::gen(gs[nb + u]);
                    const typename Mac::X xv = Mac::src(xr[u]);
#pragma unroll
                    for (int b = 0; b < KB; ++b) acc.mac(b, 0, win[(u - b + KB) % KB], xv);
                }
            }
        }
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&gempty[sb])) : "memory");
        if (!ok) break;
    }
    if (!ok && w.q0 < w.q1) {
        atomicOr(&g_bt_status, 1);
        // a copy issued for a stage nobody waited for: let it land (bounded)
        // before the CTA's shared memory is given up
        if (tid == 0 && pending >= 0)
            bt_mbar_wait(smem_u32(&gfull[pending & 1]), (uint32_t)((pending >> 1) & 1));
    }

    const int p = w.p0 + lane;
    if (mact && p < c.M) {
        float2* out = part + (long long)w.split * Ntot * R;
#pragma unroll
        for (int b = 0; b < KB; ++b) {
            const int mi = m0 + b;
            if (mi < n) {
                const long long o = (c.row_off + (long long)p * n + mi) * R + col0;
                const float2 v = acc.result(b, 0);
                if (w.pad) {
                    const float2 u = out[o];
                    out[o] = make_float2(u.x + v.x, u.y + v.y);
                } else {
                    out[o] = v;
                }
            }
        }
    }
}

// xs = rf .* x   (columns scaled by the column factor r^q_n of their row)
template <typename V, typename S>
__global__ void k_scale_cols(long long Ntot, int R, const S* __restrict__ rf, const V* __restrict__ x,
                             V* __restrict__ xs) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Ntot * R) return;
    const S f = rf[i / R];
    const V v = x[i];
    xs[i] = V{v.x * f, v.y * f};
}

// y = x + lf .* sum_s part[s]
// (kFinLanes threads per element split the partial slots, then shuffle-add)
constexpr int kFinLanes = 8;
template <typename V>
__global__ void k_finalize(long long Ntot, int R, int nsplit, const V* __restrict__ lf,
                           const V* __restrict__ x, const V* __restrict__ part, V* __restrict__ y) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long i = t / kFinLanes;
    const int sub = (int)(t % kFinLanes);
    const long long tot = Ntot * R;
    V s = vzero<V>();
    if (i < tot) {
        for (int k = sub; k < nsplit; k += kFinLanes) {
            const V v = part[(long long)k * tot + i];
            s.x += v.x;
            s.y += v.y;
        }
    }
#pragma unroll
    for (int off = kFinLanes / 2; off > 0; off >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
    }
    if (i >= tot || sub != 0) return;
    const V l = lf[i / R];
    const V v = x[i];
    y[i] = V{v.x + (l.x * s.x - l.y * s.y), v.y + (l.x * s.y + l.y * s.x)};
}

// ---------------------------------------------------------------- kernel selection

// Candidate window lengths: FP64 keeps the three-sum accumulators and the
// converted window in <= 128 registers up to KB = 7; FP32 up to KB = 9.
constexpr int kKbMin = 4;
constexpr int kKbMax64 = 7;
constexpr int kKbMax32 = 9;

using Choice = MatvecChoice;

// Two FP64 stages of the CUDA-core kernel (32 generator rows of L values
// with their guards, and the padded source column, complex128) exceed the
// shared memory of a CTA.
bool f64_one_stage(int Nmax, int KB) {
    const int n = 2 * Nmax + 1, L = 4 * Nmax + 1;
    return 2 * (size_t)(stage_g_elems(L, KB) + stage_x_elems(n, 1, KB)) * 16 > kMatvecSmemCap;
}

Choice choose(int R, int Nmax, bool fp64) {
    const int n = 2 * Nmax + 1;
    Choice best{8, 1, 1, 0};
    double best_cost = 1e300;
    for (int KB = kKbMin; KB <= (fp64 ? kKbMax64 : kKbMax32); ++KB) {
        const int I = (n + KB - 1) / KB;
        if (I > 16) continue;
        const double pad = (double)I * KB;
        // padded MACs times the per-MAC instruction overhead of the window
        // (3 extra FP64 adds per KB x 3 FMAs, or ~3 extra instructions per
        // KB x 4 FFMAs)
        const double cost = pad * pad * (fp64 ? (1.0 + 1.0 / KB) : (1.0 + 0.75 / KB));
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = Choice{KB, 1, 1, I};
        }
    }
    if (fp64) best.ONE = f64_one_stage(Nmax, best.KB) ? 1 : 0;
    if (!fp64) {
        const int rb_max = 4;
        for (int rt = 2; rt <= 16; rt *= 2) {
            if (R % rt) break;
            const int rb = rt < rb_max ? rt : rb_max;
            if (best.I * (rt / rb) <= 16) {
                best.RT = rt;
                best.RB = rb;
            }
        }
    }
    return best;
}

template <typename V, int RT, int RB, int KB, int P = 0, int S = 2>
struct Bt {
    static void attr() {
        static bool done = false;
        if (!done) {
            cudaFuncSetAttribute(k_bt_matvec<V, RT, RB, KB, P, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMatvecSmemCap);
            done = true;
        }
    }
    static size_t smem(int Nmax) {
        const int n = 2 * Nmax + 1, L = 4 * Nmax + 1;
        return S * (size_t)(stage_g_elems(L, KB) + stage_x_elems(n, RT, KB)) * sizeof(V);
    }
    static dim3 block(int Nmax) {
        const int n = 2 * Nmax + 1;
        return dim3(32, ((n + KB - 1) / KB) * (RT / RB));
    }
    static void launch(const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, int Nmax, const V* G,
                       const V* xs, V* part, long long Ntot, int R, cudaStream_t s, const int* live = nullptr) {
        attr();
        const int rtiles = R / RT;
        k_bt_matvec<V, RT, RB, KB, P, S><<<(unsigned)(nwork * rtiles), block(Nmax), smem(Nmax), s>>>(
            d_cfg, d_work, G, xs, part, Ntot, R, rtiles, live);
    }
    static int occupancy(int Nmax) {
        attr();
        const dim3 b = block(Nmax);
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bt_matvec<V, RT, RB, KB, P, S>, b.x * b.y,
                                                          smem(Nmax)) != cudaSuccess) {
            cudaGetLastError();
            nb = 1;
        }
        return nb < 1 ? 1 : nb;
    }
};

template <int KB, int P>
struct Bt1 {
    static void attr() {
        static bool done = false;
        if (!done) {
            cudaFuncSetAttribute(k_bt_matvec1<KB, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMatvecSmemCap);
            done = true;
        }
    }
    static size_t smem(int Nmax) { return 2 * (size_t)stage_g_elems(4 * Nmax + 1, KB) * sizeof(float2); }
    static dim3 block(int Nmax) { return dim3(32, (2 * Nmax + 1 + KB - 1) / KB); }
    static void launch(const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, int Nmax, const float2* G,
                       const float2* xs, float2* part, long long Ntot, int R, cudaStream_t s,
                       const int* live = nullptr) {
        attr();
        k_bt_matvec1<KB, P><<<(unsigned)(nwork * R), block(Nmax), smem(Nmax), s>>>(d_cfg, d_work, G, xs, part, Ntot,
                                                                                   R, R, live);
    }
    static int occupancy(int Nmax) {
        attr();
        const dim3 b = block(Nmax);
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_bt_matvec1<KB, P>, b.x * b.y, smem(Nmax)) !=
            cudaSuccess) {
            cudaGetLastError();
            nb = 1;
        }
        return nb < 1 ? 1 : nb;
    }
};

// Dispatch on (RT, RB) for a fixed KB (FP32), or KB alone (FP64).
template <int KB, int P, typename F>
void with_f32_p(const Choice& c, F&& f) {
    switch (c.RT) {
        case 1: f(Bt<float2, 1, 1, KB, P>()); break;
        case 2: f(Bt<float2, 2, 2, KB, P>()); break;
        case 4: f(Bt<float2, 4, 4, KB, P>()); break;
        case 8: f(Bt<float2, 8, 4, KB, P>()); break;
        default: f(Bt<float2, 16, 4, KB, P>()); break;
    }
}
// P2 bit 0: paired FMAs; bit 1: the barrier-free single-column kernel
template <int KB, typename F>
void with_f32(const Choice& c, F&& f) {
    if (c.P2 & 2) {
        if (c.P2 & 1) f(Bt1<KB, 1>());
        else f(Bt1<KB, 0>());
    } else if (c.P2) {
        with_f32_p<KB, 1>(c, f);
    } else {
        with_f32_p<KB, 0>(c, f);
    }
}

// FP64: two stages when they fit in the shared memory of a CTA, else one
// (choice field I holds ceil(n / KB); c.ONE selects the one-stage kernel).
template <int KB, typename F>
void with_f64(const Choice& c, F&& f) {
    if (c.ONE) f(Bt<double2, 1, 1, KB, 0, 1>());
    else f(Bt<double2, 1, 1, KB, 0, 2>());
}
template <typename F>
void dispatch64(const Choice& c, F&& f) {
    switch (c.KB) {
        case 4: with_f64<4>(c, f); break;
        case 5: with_f64<5>(c, f); break;
        case 6: with_f64<6>(c, f); break;
        default: with_f64<7>(c, f); break;
    }
}

template <typename F>
void dispatch32(const Choice& c, F&& f) {
    switch (c.KB) {
        case 4: with_f32<4>(c, f); break;
        case 5: with_f32<5>(c, f); break;
        case 6: with_f32<6>(c, f); break;
        case 7: with_f32<7>(c, f); break;
        case 8: with_f32<8>(c, f); break;
        default: with_f32<9>(c, f); break;
    }
}

template <typename F>
void dispatch(const Choice& c, bool fp64, F&& f) {
    if (fp64) dispatch64(c, f);
    else dispatch32(c, f);
}

}  // namespace

MatvecChoice matvec_default_choice(int R, int Nmax, bool fp64) { return choose(R, Nmax, fp64); }

int bt_status_and_clear() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_bt_status, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_bt_status, &z, sizeof(int));
    }
    return v;
}

// Every instantiated tile shape that fits this (R, N): FP64 KB = 4..7 with
// RT = 1; FP32 KB = 4..9 with each column tile RT in {1, 2, 4, 8, 16} that
// divides R and keeps I * RT / RB <= 16 warps per CTA, four-FFMA and
// paired-FMA forms, for RT = 1 also in the barrier-free kernel, and the
// tensor-core kernel with TC in {16, 32, 64} columns dividing R (n <= 128).
int matvec_candidates(int R, int Nmax, bool fp64, MatvecChoice* out, int cap, bool allow_sh) {
    const int n = 2 * Nmax + 1;
    int cnt = 0;
    for (int KB = kKbMin; KB <= (fp64 ? kKbMax64 : kKbMax32); ++KB) {
        const int I = (n + KB - 1) / KB;
        if (I > 16) continue;
        for (int rt = 1; rt <= (fp64 ? 1 : 16); rt *= 2) {
            if (R % rt) break;
            const int rb = rt < 4 ? rt : 4;
            if (I * (rt / rb) > 16) continue;
            for (int p2 = 0; p2 <= (fp64 ? 0 : (rt == 1 ? 3 : 1)); ++p2) {
                Choice c{KB, rt, rb, I, 0, p2};
                if (fp64) c.ONE = f64_one_stage(Nmax, KB) ? 1 : 0;
                size_t b = 0;
                dispatch(c, fp64, [&](auto k) { b = decltype(k)::smem(Nmax); });
                if (b > kMatvecSmemCap) continue;
                if (cnt < cap) out[cnt] = c;
                ++cnt;
            }
        }
    }
    if (!fp64)
        for (int rc = 16; rc <= 64; rc *= 2)
            if (tc_supported(R, Nmax, rc)) {
                if (cnt < cap) out[cnt] = Choice{0, rc, 0, 0, rc};
                ++cnt;
            }
    if (!fp64 && allow_sh && tcs_supported(R, Nmax))
        for (int sh = 1; sh <= 2; ++sh) {  // KB = sh - 1 in the encoding of msd_set_tile
            if (cnt < cap) out[cnt] = Choice{sh - 1, MSD_TCS_COLS, 0, 0, 0, 0, sh};
            ++cnt;
        }
    return cnt < cap ? cnt : cap;
}

size_t matvec_smem_bytes(const MatvecChoice& c, int Nmax, bool fp64) {
    if (c.SH) return tcs_smem_bytes(Nmax);
    if (c.TC) return tc_smem_bytes(c.TC);
    size_t b = 0;
    dispatch(c, fp64, [&](auto k) { b = decltype(k)::smem(Nmax); });
    return b;
}

// Resident CTAs per SM of one product kernel instance.
int matvec_blocks_per_sm(const MatvecChoice& c, int Nmax, bool fp64) {
    if (c.TC || c.SH) return 1;
    int nb = 1;
    dispatch(c, fp64, [&](auto k) { nb = decltype(k)::occupancy(Nmax); });
    return nb;
}

void launch_scale_cols(bool fp64, long long Ntot, int R, const void* rf, const void* x, void* xs, cudaStream_t s) {
    const long long tot = Ntot * R;
    const int th = 256;
    const unsigned blocks = (unsigned)((tot + th - 1) / th);
    if (fp64) k_scale_cols<double2, double><<<blocks, th, 0, s>>>(Ntot, R, (const double*)rf, (const double2*)x,
                                                                   (double2*)xs);
    else k_scale_cols<float2, float><<<blocks, th, 0, s>>>(Ntot, R, (const float*)rf, (const float2*)x, (float2*)xs);
    g_msd_launches += 1;
}

void launch_finalize(bool fp64, long long Ntot, int R, int nsplit, const void* lf, const void* x, const void* part,
                     void* y, cudaStream_t s) {
    const long long tot = Ntot * R;
    const int th = 256;
    const unsigned blocks = (unsigned)((tot * kFinLanes + th - 1) / th);
    if (fp64) k_finalize<double2><<<blocks, th, 0, s>>>(Ntot, R, nsplit, (const double2*)lf, (const double2*)x,
                                                         (const double2*)part, (double2*)y);
    else k_finalize<float2><<<blocks, th, 0, s>>>(Ntot, R, nsplit, (const float2*)lf, (const float2*)x,
                                                  (const float2*)part, (float2*)y);
    g_msd_launches += 1;
}

void launch_bt_only(const MatvecChoice& c, bool fp64, const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork,
                    int Nmax, const void* G, const void* xs, void* part, long long Ntot, int R, cudaStream_t s) {
    if (fp64)
        dispatch64(c, [&](auto k) {
            decltype(k)::launch(d_cfg, d_work, nwork, Nmax, (const double2*)G, (const double2*)xs, (double2*)part,
                                Ntot, R, s);
        });
    else if (c.TC) {
        launch_bt_tc(c.TC, d_cfg, d_work, nwork, (const float2*)G, (const float2*)xs, (float2*)part, Ntot, R, s);
        return;  // counted by launch_bt_tc
    } else
        dispatch32(c, [&](auto k) {
            decltype(k)::launch(d_cfg, d_work, nwork, Nmax, (const float2*)G, (const float2*)xs, (float2*)part,
                                Ntot, R, s);
        });
    g_msd_launches += 1;
}

void launch_matvec_f64(const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, int Nmax,
                       const double2* G, const double* rf, const double2* lf, long long Ntot, int R,
                       const double2* x, double2* xs, double2* part, int nsplit, double2* y, cudaStream_t s,
                       cudaEvent_t ev0, cudaEvent_t ev1, const MatvecChoice* ch, const int* live) {
    const long long tot = Ntot * R;
    const int th = 256;
    const unsigned blocks = (unsigned)((tot + th - 1) / th);
    k_scale_cols<double2, double><<<blocks, th, 0, s>>>(Ntot, R, rf, x, xs);
    if (ev0) cudaEventRecord(ev0, s);
    dispatch64(ch ? *ch : choose(R, Nmax, true), [&](auto k) {
        decltype(k)::launch(d_cfg, d_work, nwork, Nmax, G, xs, part, Ntot, R, s, live);
    });
    if (ev1) cudaEventRecord(ev1, s);
    k_finalize<double2><<<(unsigned)((tot * kFinLanes + th - 1) / th), th, 0, s>>>(Ntot, R, nsplit, lf, x, part, y);
    g_msd_launches += 3;
}

void launch_matvec_f32(const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, int Nmax,
                       const float2* G, const float* rf, const float2* lf, long long Ntot, int R,
                       const float2* x, float2* xs, float2* part, int nsplit, float2* y, cudaStream_t s,
                       cudaEvent_t ev0, cudaEvent_t ev1, const MatvecChoice* ch, const int* live,
                       bool xs_ready) {
    const long long tot = Ntot * R;
    const int th = 256;
    const unsigned blocks = (unsigned)((tot + th - 1) / th);
    if (!xs_ready) k_scale_cols<float2, float><<<blocks, th, 0, s>>>(Ntot, R, rf, x, xs);
    else g_msd_launches -= 1;  // counted below with the product and the reduction
    if (ev0) cudaEventRecord(ev0, s);
    const Choice c = ch ? *ch : choose(R, Nmax, false);
    if (c.TC) {
        launch_bt_tc(c.TC, d_cfg, d_work, nwork, G, xs, part, Ntot, R, s, live);
        g_msd_launches -= 1;  // counted below with the scaling and the reduction
    } else {
        dispatch32(c, [&](auto k) {
            decltype(k)::launch(d_cfg, d_work, nwork, Nmax, G, xs, part, Ntot, R, s, live);
        });
    }
    if (ev1) cudaEventRecord(ev1, s);
    k_finalize<float2><<<(unsigned)((tot * kFinLanes + th - 1) / th), th, 0, s>>>(Ntot, R, nsplit, lf, x, part, y);
    g_msd_launches += 3;
}

// ---------------------------------------------------------------- general scalings
// The same Toeplitz sums with other diagonal scalings, for the adjoint
// operator (P^-1 A)^H z = z + r .* T^H (conj(l) .* z) and for the raw sums
// the gradient needs.  Column scaling: real (r) or complex (conj l); row
// scaling: none (raw sums), real or complex; optional + x.

namespace {

template <typename V>
__global__ void k_scale_cols_c(long long Ntot, int R, const V* __restrict__ cf, const V* __restrict__ x,
                               V* __restrict__ xs) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Ntot * R) return;
    const V f = cf[i / R];
    const V v = x[i];
    xs[i] = V{f.x * v.x - f.y * v.y, f.x * v.y + f.y * v.x};
}

// y = (add_x ? x : 0) + row .* sum_s part[s];  row: rr (real), rc (complex) or none
template <typename V, typename S>
__global__ void k_finalize_gen(long long Ntot, int R, int nsplit, const S* __restrict__ rr,
                               const V* __restrict__ rc, int add_x, const V* __restrict__ x,
                               const V* __restrict__ part, V* __restrict__ y) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long i = t / kFinLanes;
    const int sub = (int)(t % kFinLanes);
    const long long tot = Ntot * R;
    V s = vzero<V>();
    if (i < tot) {
        for (int k = sub; k < nsplit; k += kFinLanes) {
            const V v = part[(long long)k * tot + i];
            s.x += v.x;
            s.y += v.y;
        }
    }
#pragma unroll
    for (int off = kFinLanes / 2; off > 0; off >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
    }
    if (i >= tot || sub != 0) return;
    V o = s;
    if (rr) {
        const S f = rr[i / R];
        o = V{f * s.x, f * s.y};
    } else if (rc) {
        const V l = rc[i / R];
        o = V{l.x * s.x - l.y * s.y, l.x * s.y + l.y * s.x};
    }
    if (add_x) {
        const V v = x[i];
        o.x += v.x;
        o.y += v.y;
    }
    y[i] = o;
}

template <typename V, typename S, typename D>
void product_general(D&& dispatch_fn, const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, int Nmax,
                     const V* G, const S* col_r, const V* col_c, const S* row_r, const V* row_c, int add_x,
                     long long Ntot, int R, const V* x, V* xs, V* part, int nsplit, V* y, cudaStream_t s) {
    const long long tot = Ntot * R;
    const int th = 256;
    const unsigned blocks = (unsigned)((tot + th - 1) / th);
    if (col_c) k_scale_cols_c<V><<<blocks, th, 0, s>>>(Ntot, R, col_c, x, xs);
    else k_scale_cols<V, S><<<blocks, th, 0, s>>>(Ntot, R, col_r, x, xs);
    dispatch_fn([&](auto k) { decltype(k)::launch(d_cfg, d_work, nwork, Nmax, G, xs, part, Ntot, R, s); });
    k_finalize_gen<V, S><<<(unsigned)((tot * kFinLanes + th - 1) / th), th, 0, s>>>(Ntot, R, nsplit, row_r, row_c,
                                                                                   add_x, x, part, y);
    g_msd_launches += 3;
}

}  // namespace

void launch_product_f64(const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, int Nmax, const double2* G,
                        const double* col_r, const double2* col_c, const double* row_r, const double2* row_c,
                        int add_x, long long Ntot, int R, const double2* x, double2* xs, double2* part, int nsplit,
                        double2* y, cudaStream_t s, const MatvecChoice* ch) {
    const Choice c = ch ? *ch : choose(R, Nmax, true);
    product_general<double2, double>([&](auto f) { dispatch64(c, f); }, d_cfg, d_work, nwork, Nmax, G, col_r,
                                     col_c, row_r, row_c, add_x, Ntot, R, x, xs, part, nsplit, y, s);
}

void launch_product_f32(const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, int Nmax, const float2* G,
                        const float* col_r, const float2* col_c, const float* row_r, const float2* row_c,
                        int add_x, long long Ntot, int R, const float2* x, float2* xs, float2* part, int nsplit,
                        float2* y, cudaStream_t s, const MatvecChoice* ch) {
    const Choice c = ch ? *ch : choose(R, Nmax, false);
    if (c.TC) {
        // the same scalings around the tensor-core kernel
        struct TcLaunch {
            int RC;
            void launch(const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, int, const float2* G,
                        const float2* xs, float2* part, long long Ntot, int R, cudaStream_t s) const {
                launch_bt_tc(RC, d_cfg, d_work, nwork, G, xs, part, Ntot, R, s);
                g_msd_launches -= 1;
            }
        };
        const TcLaunch tl{c.TC};
        product_general<float2, float>(
            [&](auto f) {
                (void)f;
                tl.launch(d_cfg, d_work, nwork, Nmax, G, xs, part, Ntot, R, s);
            },
            d_cfg, d_work, nwork, Nmax, G, col_r, col_c, row_r, row_c, add_x, Ntot, R, x, xs, part, nsplit, y, s);
        return;
    }
    product_general<float2, float>([&](auto f) { dispatch32(c, f); }, d_cfg, d_work, nwork, Nmax, G, col_r, col_c,
                                   row_r, row_c, add_x, Ntot, R, x, xs, part, nsplit, y, s);
}
