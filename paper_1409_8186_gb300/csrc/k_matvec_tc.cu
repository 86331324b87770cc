// Tensor-core form of the block-Toeplitz product (kernel K3, FP32 products
// with many right-hand sides).  With R >= 16 columns the sum
//     Y^p[m][r] = sum_q sum_n g^pq_{n-m} Xs^q[n][r]        (section 4.2 blocks)
// is a dense contraction over the source modes (q, n), so it runs on the
// fifth-generation tensor cores (tcgen05.mma, accumulators in TMEM):
//
//  * A (M = 128 rows): the Toeplitz blocks of up to TP = floor(128 / n)
//    target disks, expanded in shared memory from the generators, one source
//    q and 16 modes n per pipeline stage;
//  * B (N = 2 RC rows, K-major): the scaled columns of source q, as
//    B1 = [Re X | Im X] and B2 = [-Im X | Re X], so that
//    D = Re(A) B1 + Im(A) B2 = [Re Y | Im Y] (complex product as two real
//    GEMMs into one FP32 accumulator of 2 RC columns);
//  * precision: every operand is split into two TF32 parts (x = hi + lo,
//    hi = tf32(x), lo = tf32(x - hi)) and the products hi*hi + hi*lo + lo*hi
//    are accumulated ("3xTF32"); each source's sum stays in TMEM only
//    until it is added to FP32 registers (round-to-nearest), which keeps the
//    FP32 accuracy of the CUDA-core kernel over thousands of sources.
//
// Shared-memory operand layout: K-major without swizzle, 8-row x 16-byte core
// matrices, 128 bytes between K-adjacent core matrices (LBO), 512 bytes
// between 8-row groups (SBO).  One thread issues the MMAs of a stage and
// commits them to the stage's mbarrier; the other threads expand the next
// stages meanwhile.  Every wait has a clock limit: on expiry the kernel sets
// an error bit, waits (again bounded) for its issued MMAs, frees its TMEM
// and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "msd_internal.cuh"

__device__ int g_tc_status;  // bit 0: a pipeline wait expired

namespace {

constexpr int kTcM = 128;       // rows of one MMA
constexpr int kTcThreads = 288;   // 8 expansion / accumulator warps + 1 MMA warp
constexpr int kExpThreads = 256;
constexpr int kTcStages = 3;
constexpr int kKc = 16;         // modes per stage (two K-steps of 8)
constexpr int kLbo = 128;
constexpr int kSbo = 512;
constexpr int kABytes = kTcM * kKc * 4;  // one A array of a stage (8 KB)
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz
constexpr long long kTestWaitCycles = 20000;     // msd_test_expire_waits

template <int RC>
struct TcLayout {
    static constexpr int kBBytes = 2 * RC * kKc * 4;
    static constexpr int kStageBytes = 4 * kABytes + 4 * kBBytes;
    static constexpr int kSmem = kTcStages * kStageBytes + 1024;  // + alignment slack
    static constexpr int kTmemCols = 4 * RC;  // two accumulators of 2 RC columns: 64, 128 or 256
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(kLbo >> 4) << 16) | ((uint64_t)(kSbo >> 4) << 32) |
           (1ull << 46);  // descriptor version; base offset 0; no swizzle
}

// kind::tf32 instruction descriptor: D F32, A and B TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// byte offset of the 16-byte chunk (row, modes 4kq..4kq+3) of a 128 x 16 or
// 2RC x 16 operand
__device__ __forceinline__ int quad_off(int row, int kq) { return (row & 7) * 16 + (row >> 3) * kSbo + kq * kLbo; }

__device__ __forceinline__ void split4(const float v[4], float4& hi, float4& lo) {
    float h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        h[j] = tf32_rna(v[j]);
        l[j] = tf32_rna(v[j] - h[j]);
    }
    hi = make_float4(h[0], h[1], h[2], h[3]);
    lo = make_float4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
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
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

// Test hook (msd_test_expire_waits): a wait on a flag that nothing sets,
// with a short limit, so that the expiry path runs without any fault.
__device__ __forceinline__ bool wait_unset_flag(const volatile int* flag) {
    const long long t0 = clock64();
    while (!*flag)
        if (clock64() - t0 > kTestWaitCycles) return false;
    return true;
}

template <int NC>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* v);

template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// y[0..NC) <- TMEM columns taddr..taddr+NC-1 of this thread's lane, in groups of 8
template <int NC>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float* v) {
#pragma unroll
    for (int j = 0; j < NC; j += 8) tmem_ld<8>(taddr + j, v + j);
}

template <int RC>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_bt_tc(const MsdConfig* __restrict__ cfgs, const MatvecWork* __restrict__ works, const float2* __restrict__ G,
            const float2* __restrict__ xs, float2* __restrict__ part, long long Ntot, int R, int rtiles,
            int expire_test, const int* __restrict__ live) {
    typedef TcLayout<RC> Lay;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint32_t tmem_sh;
    __shared__ __align__(8) uint64_t mbar[kTcStages];
    __shared__ __align__(8) uint64_t accbar[2];  // the MMAs of a source into accumulator 0 / 1 are done
    __shared__ int abort_sh;                      // a pipeline wait ran out
    __shared__ int never_sh;                      // stays 0 (test hook)

    const int wi = blockIdx.x / rtiles;
    const int rt = blockIdx.x - wi * rtiles;
    const MatvecWork w = works[wi];
    const MsdConfig c = cfgs[w.cfg];
    const int N = c.N, n = c.n, L = c.L;
    const int TP = kTcM / n;
    const int np = min(min(TP, 32 - (w.p0 & 31)), c.M - w.p0);  // target disks of this tile
    const int nk = (n + kKc - 1) / kKc;                          // stages per source
    const int col0 = rt * RC;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // no active column in this tile (converged Krylov systems): zero raw
    // sums, no other work
    if (live) {
        bool any = false;
        for (int r = 0; r < RC; ++r) any |= live[w.cfg * R + col0 + r] != 0;
        if (!any) {
            if (!w.pad) {
                float2* out = part + (long long)w.split * Ntot * R + col0;
                for (int t = tid; t < np * n * RC; t += kTcThreads) {
                    const int i = t / RC, j = t - i * RC;
                    out[(c.row_off + (long long)w.p0 * n + i) * R + j] = make_float2(0.f, 0.f);
                }
            }
            return;
        }
    }

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(Lay::kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        abort_sh = 0;
        never_sh = 0;
        for (int s = 0; s < kTcStages; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])));
        for (int s = 0; s < 2; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accbar[s])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_sh;

    // A expansion role: row ai = (target pl, mode m), modes 8*akh .. 8*akh+7 of the stage
    // warp 8 only issues the MMAs; warps 0-7 expand the operands and hold the
    // accumulator sums (warp & 3 = TMEM lane quarter, warp >> 2 = half of the columns)
    const bool mma_warp = warp == kExpThreads / 32;
    const int ai = tid & (kTcM - 1), akh = (tid >> 7) & 1;
    const int apl = ai / n, am = ai - apl * n;
    const bool arow = !mma_warp && apl < np;
    const float2* grow = G + c.gen_off + (long long)(w.p0 + (arow ? apl : 0)) * L + 2 * N - am;
    // B expansion role: column cb, mode quad bq (4 RC items)
    const float2* xq0 = xs + c.row_off * R + col0;

    // Each source is accumulated in TMEM alone (accumulator qi & 1), then
    // added in FP32 registers with round-to-nearest: the tensor pipe's own
    // accumulation is not round-to-nearest, and its error over thousands of
    // sources would exceed the FP32 kernel's.  Register sums: warp -> TMEM
    // lane quarter (warp & 3) and half of the columns (warp >> 2).
    constexpr int HC = RC / 2;
    const int quarter = warp & 3, half = warp >> 2;
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    float sr[HC], si[HC];
#pragma unroll
    for (int j = 0; j < HC; ++j) sr[j] = si[j] = 0.f;
    auto fold = [&](int acc) {
        float t[HC];
        const uint32_t a = lane_addr + acc * 2 * RC + half * HC;
        tmem_ld<HC>(a, t);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int j = 0; j < HC; ++j) sr[j] += t[j];
        tmem_ld<HC>(a + RC, t);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int j = 0; j < HC; ++j) si[j] += t[j];
    };

    // raw values of a stage, loaded one stage ahead into registers so that the
    // global-memory latency overlaps the expansion and MMAs of the stage before
    const int bitem = tid < 4 * RC ? tid : -1;  // B item (column cb, mode quad kq); 4 RC <= 256 items
                                                // (so the MMA warp has none)
    const int bcb = bitem % RC, bkq = bitem / RC;
    auto load_stage = [&](int st_it, float2* ga, float2* xv) {
        const int sq = w.q0 + st_it / nk;
        const int sk0 = (st_it % nk) * kKc;
        const float2* gq = grow + (long long)sq * c.Mp * L;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = sk0 + akh * 8 + j;
            ga[j] = (arow && k < n) ? __ldg(gq + k) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = sk0 + bkq * 4 + j;
            xv[j] = (bitem >= 0 && k < n) ? __ldg(xq0 + ((long long)sq * n + k) * R + bcb) : make_float2(0.f, 0.f);
        }
    };
    float2 ga[8], xv[4], gn[8], xn[4];

    const int nst = (w.q1 - w.q0) * nk;
    if (nst > 0) load_stage(0, ga, xv);
    bool ok = true;
    int issued = 0;  // stages whose MMAs were committed
    for (int it = 0; it < nst; ++it) {
        const int b = it % kTcStages;
        const int qi = it / nk, kc = it - qi * nk;
        if (it + 1 < nst) load_stage(it + 1, gn, xn);  // in flight during the waits and the expansion
        // One CTA barrier per stage (after the expansion).  A wait that runs
        // out records the failure and the thread carries on through the same
        // barriers (no thread leaves them), so the results are discarded at
        // the end; warp-collective TMEM loads only run for whole warps.
        bool mine = true;  // the MMAs that last read buffer b are done
        if (it >= kTcStages) mine = mbar_wait(smem_u32(&mbar[b]), (uint32_t)((it / kTcStages - 1) & 1));
        if (expire_test && it == kTcStages) mine = wait_unset_flag(&never_sh) && mine;
        // the accumulator of this source last held source qi - 2: fold it first
        if (kc == 0 && qi >= 2 && !mma_warp) {
            bool acc_ready = mine && mbar_wait(smem_u32(&accbar[qi & 1]), (uint32_t)(((qi - 2) >> 1) & 1));
            acc_ready = __all_sync(0xffffffffu, acc_ready);
            if (acc_ready) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                fold(qi & 1);
                asm volatile("tcgen05.fence::before_thread_sync;");
            }
            mine = mine && acc_ready;
        }
        if (!mine) abort_sh = 1;
        const int k0 = kc * kKc;
        unsigned char* st = sm + b * Lay::kStageBytes;
        unsigned char* Arh = st;
        unsigned char* Arl = st + kABytes;
        unsigned char* Aih = st + 2 * kABytes;
        unsigned char* Ail = st + 3 * kABytes;
        unsigned char* Bb = st + 4 * kABytes;  // B1h, B1l, B2h, B2l
        // ---- A: Toeplitz rows g_{k-m}, k = k0 + 8 akh + j
        if (!mma_warp) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int kq = akh * 2 + h;
                float re[4], im[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    re[j] = ga[h * 4 + j].x;
                    im[j] = ga[h * 4 + j].y;
                }
                float4 hi, lo;
                const int off = quad_off(ai, kq);
                split4(re, hi, lo);
                *(float4*)(Arh + off) = hi;
                *(float4*)(Arl + off) = lo;
                split4(im, hi, lo);
                *(float4*)(Aih + off) = hi;
                *(float4*)(Ail + off) = lo;
            }
        }
        // ---- B: [Re X | Im X] and [-Im X | Re X] of source q, modes k0 .. k0+15
        if (bitem >= 0) {
            const int cb = bcb, kq = bkq;
            float xr[4], xi[4], nxi[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                xr[j] = xv[j].x;
                xi[j] = xv[j].y;
                nxi[j] = -xv[j].y;
            }
            float4 hi, lo;
            split4(xr, hi, lo);  // Re X: B1 row cb, B2 row RC + cb
            *(float4*)(Bb + quad_off(cb, kq)) = hi;
            *(float4*)(Bb + Lay::kBBytes + quad_off(cb, kq)) = lo;
            *(float4*)(Bb + 2 * Lay::kBBytes + quad_off(RC + cb, kq)) = hi;
            *(float4*)(Bb + 3 * Lay::kBBytes + quad_off(RC + cb, kq)) = lo;
            split4(xi, hi, lo);  // Im X: B1 row RC + cb
            *(float4*)(Bb + quad_off(RC + cb, kq)) = hi;
            *(float4*)(Bb + Lay::kBBytes + quad_off(RC + cb, kq)) = lo;
            split4(nxi, hi, lo);  // -Im X: B2 row cb
            *(float4*)(Bb + 2 * Lay::kBBytes + quad_off(cb, kq)) = hi;
            *(float4*)(Bb + 3 * Lay::kBBytes + quad_off(cb, kq)) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        if (tid == kExpThreads) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            constexpr uint32_t id = idesc_tf32(kTcM, 2 * RC);
            const uint32_t a_addr[6] = {smem_u32(Arh), smem_u32(Arh), smem_u32(Arl),
                                        smem_u32(Aih), smem_u32(Aih), smem_u32(Ail)};
            const uint32_t b_addr[6] = {smem_u32(Bb), smem_u32(Bb + Lay::kBBytes), smem_u32(Bb),
                                        smem_u32(Bb + 2 * Lay::kBBytes), smem_u32(Bb + 3 * Lay::kBBytes),
                                        smem_u32(Bb + 2 * Lay::kBBytes)};
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                if (k0 + ks * 8 >= n) break;  // an all-zero K-step at the end of a source
#pragma unroll
                for (int t = 0; t < 6; ++t) {
                    const uint64_t da = umma_desc(a_addr[t] + ks * 2 * kLbo);
                    const uint64_t db = umma_desc(b_addr[t] + ks * 2 * kLbo);
                    const uint32_t acc = (kc > 0 || ks > 0 || t > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                            tmem + (uint32_t)((qi & 1) * 2 * RC)),
                        "l"(da), "l"(db), "r"(id), "r"(acc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar[b])));
            if (kc == nk - 1)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&accbar[qi & 1])));
        }
        issued = it + 1;
#pragma unroll
        for (int j = 0; j < 8; ++j) ga[j] = gn[j];
#pragma unroll
        for (int j = 0; j < 4; ++j) xv[j] = xn[j];
    }
    // wait for the last committed stage (a commit covers all earlier MMAs)
    bool drained = true;
    if (issued > 0) {
        const int last = issued - 1;
        drained = mbar_wait(smem_u32(&mbar[last % kTcStages]), (uint32_t)((last / kTcStages) & 1));
    }
    drained = __syncthreads_and(drained);
    ok = abort_sh == 0;  // read after the barrier above
    if ((!ok || !drained) && tid == 0) atomicOr(&g_tc_status, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");

    if (ok && drained && !mma_warp) {
        // fold the last one or two sources (every MMA is complete here)
        const int nsrc = w.q1 - w.q0;
        for (int s2 = nsrc >= 2 ? nsrc - 2 : 0; s2 < nsrc; ++s2) fold(s2 & 1);
        const int i = quarter * 32 + lane;
        const int pl = i / n, m = i - pl * n;
        if (pl < np) {
            const long long row = c.row_off + (long long)(w.p0 + pl) * n + m;
            float2* out = part + (long long)w.split * Ntot * R + row * R + col0 + half * HC;
#pragma unroll
            for (int j = 0; j < HC; ++j) {
                float2 v = make_float2(sr[j], si[j]);
                if (w.pad) {
                    const float2 u = out[j];
                    v.x += u.x;
                    v.y += u.y;
                }
                out[j] = v;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Lay::kTmemCols));
}

template <int RC>
void launch_rc(const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, const float2* G, const float2* xs,
               float2* part, long long Ntot, int R, cudaStream_t s, const int* live) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_bt_tc<RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcLayout<RC>::kSmem);
        attr = true;
    }
    const int rtiles = R / RC;
    k_bt_tc<RC><<<(unsigned)(nwork * rtiles), kTcThreads, TcLayout<RC>::kSmem, s>>>(d_cfg, d_work, G, xs, part, Ntot,
                                                                                    R, rtiles,
                                                                                    g_msd_expire_waits.load(), live);
}

}  // namespace

bool tc_supported(int R, int Nmax, int RC) {
    return (RC == 16 || RC == 32 || RC == 64) && R % RC == 0 && 2 * Nmax + 1 <= kTcM;
}

// Target tiles of the tensor-core product: TP = floor(128 / n) disks, never
// crossing a 32-disk boundary (so that a tile lies inside one block of the
// generator layouts, stored or recomputed).
int tc_tile_disks(int n) { return kTcM / n; }

size_t tc_smem_bytes(int RC) {
    return RC == 16 ? TcLayout<16>::kSmem : RC == 32 ? TcLayout<32>::kSmem : TcLayout<64>::kSmem;
}

void launch_bt_tc(int RC, const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, const float2* G,
                  const float2* xs, float2* part, long long Ntot, int R, cudaStream_t s, const int* live) {
    if (nwork <= 0) return;
    switch (RC) {
        case 16: launch_rc<16>(d_cfg, d_work, nwork, G, xs, part, Ntot, R, s, live); break;
        case 32: launch_rc<32>(d_cfg, d_work, nwork, G, xs, part, Ntot, R, s, live); break;
        default: launch_rc<64>(d_cfg, d_work, nwork, G, xs, part, Ntot, R, s, live); break;
    }
    g_msd_launches += 1;
}

int tc_status_and_clear() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_tc_status, &z, sizeof(int));
    }
    return v;
}
