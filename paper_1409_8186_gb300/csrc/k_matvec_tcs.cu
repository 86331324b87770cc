// Shift-GEMM form of the block-Toeplitz product on the tensor cores (kernel
// K3, FP32 products with R a multiple of 8 columns).
//
// With d = n - m the Toeplitz sum of section 4.2 reads
//     S^p[m][r] = sum_d sum_q g^pq_d Xs^q[m + d][r],   Xs^q[j] = 0 outside 0 <= j < n,
// so for every shift d it is a dense product over the source disks q: the
// generator matrix G_d = (g^pq_d)_{p,q} times the source columns moved down by
// d modes.  Nothing has to be expanded: the operands are streamed as they
// are stored.
//
//  * A (M = 128 rows): G_d for 128 target disks and 8 sources (one K-step
//    of kind::tf32), its real and imaginary parts each as two TF32 numbers
//    (hi = tf32(g), lo = tf32(g - hi)).  The generators are kept in HBM in
//    exactly this order (k_tcs_build_gt), so one stage is one 16 KB bulk
//    copy.
//  * B (N = 16 mb rows for a block of mb modes): the 8 columns of Xs for
//    modes j = m + d, real and imaginary rows, hi and lo.  The sources of one
//    K-step are staged once as a "slab" of all n modes (plus 15 zero modes on
//    either side, which give the zeros outside 0 <= j < n); the B operand of
//    shift d is the slab seen from mode m0 + d, i.e. the same bytes with a
//    start address 256 bytes further per shift.
//  * D1 = Re(G_d) B and D2 = Im(G_d) B accumulate in TMEM (FP32); the
//    complex sum is Re S = D1[Re x] - D2[Im x], Im S = D1[Im x] + D2[Re x].
//  * 3xTF32: hi*hi + hi*lo + lo*hi for both real products (6 MMAs per
//    stage and mode block), which keeps FP32 accuracy.  The tensor pipe's
//    accumulation does not round to nearest, so after every kFoldQc K-steps
//    (32 sources) the accumulators are added to FP32 registers (round to
//    nearest) and restarted.
//
// Roles: warp 0 issues the bulk copies (one thread), warp 1 allocates TMEM
// and issues the MMAs (one thread), warps 2-9 fold the accumulators and
// write the CTA's raw sums (warp w covers TMEM lanes 32 (w mod 4) ..
// and mode block (w - 2) / 4).  Shared-memory operand layout: K-major
// without swizzle, 8-row x 16-byte core matrices, 128 bytes between 8-row
// groups.  Every wait has a clock limit; after an expired wait the CTA
// records it, waits no more except (bounded) for its own copies and MMAs,
// writes nothing, frees TMEM and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "msd_internal.cuh"

__device__ int g_tcs_status;  // bit 0: a wait of the shift-GEMM kernel expired

namespace {

constexpr int kRC = MSD_TCS_COLS;  // columns per CTA (8)
constexpr int kPad = 15;            // zero modes on either side of the slab: a B operand of a block
                                    // of mb <= 16 modes starts at most mb - 1 modes outside 0..n-1
constexpr int kStagesMax = 8;       // A ring: as many 16 KB stages as fit next to the slab, 3..8
constexpr int kAStage = 16384;      // bytes of one A stage (Gr hi/lo, Gi hi/lo, 2 x 4 sources)
constexpr int kThreads = 320;
constexpr int kFoldQc = 4;          // K-steps of 8 sources between folds into registers
constexpr int kMbMax = 8;           // modes per block (N = 16 mb <= 128)
// Wide blocks: at most 13 modes (MMA N = 16 mb <= 208).  An autotuner run
// whose wide blocks had 16 modes (N = 256) on the lattice ended in an
// illegal-instruction fault; N <= 208 ran correctly, so wider is not offered.
constexpr int kMbWide = 13;
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz
constexpr long long kTestWaitCycles = 20000;     // msd_test_expire_waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle, given strides
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// kind::tf32 instruction descriptor: D F32, A and B TF32, both K-major.
__device__ __forceinline__ uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

__device__ __forceinline__ bool wait_unset_flag(const volatile int* flag) {
    const long long t0 = clock64();
    while (!*flag)
        if (clock64() - t0 > kTestWaitCycles) return false;
    return true;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// global -> shared bulk copy completing on an mbarrier (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
}

// 16 consecutive TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// One work item: configuration w.cfg, targets [p0, p0 + 128), modes
// [m0, m0 + nmb mb) in nmb blocks of mb modes (packed in w.pad), sources
// [q0, q1) (multiples of 8 except at the end), partial slot w.split.
__global__ void __launch_bounds__(kThreads, 1)
    k_bt_tcs(const MsdConfig* __restrict__ cfgs, const MatvecWork* __restrict__ works, const float* __restrict__ GT,
             const float* __restrict__ XT, float2* __restrict__ part, long long Ntot, int R, int rtiles,
             int kStages, int expire_test, const int* __restrict__ live) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint32_t tmem_sh;
    __shared__ __align__(8) uint64_t a_full[kStagesMax], a_empty[kStagesMax];
    __shared__ __align__(8) uint64_t s_full[2], s_empty[2];
    __shared__ __align__(8) uint64_t acc_full, acc_empty, mma_done;
    __shared__ int abort_sh, never_sh;

    const int wi = blockIdx.x / rtiles;
    const int rt = blockIdx.x - wi * rtiles;
    const MatvecWork w = works[wi];
    const MsdConfig c = cfgs[w.cfg];
    const int N = c.N, n = c.n, L = c.L;
    const int m0 = w.pad & 0xFF, mb = (w.pad >> 8) & 0xF, nmb = (w.pad >> 12) & 0xF;
    const int qc0 = w.q0 >> 3, qc1 = (w.q1 + 7) >> 3;
    const int nqc = qc1 - qc0;
    const int ptile = w.p0 >> 7;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // no active column in this tile (converged Krylov systems): zero raw
    // sums, no other work
    if (live) {
        bool any = false;
        for (int r = 0; r < kRC; ++r) any |= live[w.cfg * R + rt * kRC + r] != 0;
        if (!any) {
            const int mend0 = min(n, m0 + nmb * mb), nm = mend0 - m0;
            float2* out = part + (long long)w.split * Ntot * R + rt * kRC;
            for (int t = threadIdx.x; t < 128 * nm; t += kThreads) {
                const int p = w.p0 + t / nm, m = m0 + t % nm;
                if (p < c.M) {
                    float4* o = (float4*)(out + (c.row_off + (long long)p * n + m) * R);
#pragma unroll
                    for (int r = 0; r < kRC / 2; ++r) o[r] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            return;
        }
    }
    unsigned char* A = sm;                                   // [kStages][16 KB]
    unsigned char* slab = sm + kStages * kAStage;            // [2][4][(n + 14) * 256]
    const int blk = (n + 2 * kPad) * 256;                    // bytes of one slab block
    const int buf = 4 * blk;

    // modes covered: [m0, mend); shifts d in [-(mend - 1), n - 1 - m0]
    const int mend = min(n, m0 + nmb * mb);
    const int dlo = -(mend - 1), dhi = n - 1 - m0;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        abort_sh = 0;
        never_sh = 0;
        for (int s = 0; s < kStagesMax; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&a_full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&a_empty[s])));
        }
        for (int s = 0; s < 2; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_full)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_u32(&acc_empty)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_done)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // zero modes of both slab buffers (the bulk copies never write them)
    for (int i = tid; i < 2 * 4 * 2 * kPad * 16; i += kThreads) {
        const int b = i / (2 * kPad * 16), rem = i - b * (2 * kPad * 16);
        const int side = rem / (kPad * 16), o = rem - side * (kPad * 16);
        unsigned char* base = slab + b * blk + (side ? (kPad + n) * 256 : 0);
        *(float4*)(base + o * 16) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_sh;
    volatile int* abort_v = &abort_sh;
    const int nd = dhi - dlo + 1;
    const int ngroups = (nqc + kFoldQc - 1) / kFoldQc;
    int issued_mma = 0;

    if (warp == 0 && lane == 0) {
        // ---------------- producer
        const float* gt = GT + c.gt_off + (long long)ptile * L * (c.Mq / 4) * 2048;
        const float* xt = XT + c.xrow_off * 4 * R + (long long)rt * c.Mq * n * 32;
        long long ait = 0;
        // slab of K-step qi; issued one K-step ahead, once the MMAs of K-step
        // qi - 2 (the previous user of its buffer) have certainly completed
        auto issue_slab = [&](int qi) {
            const int qc = qc0 + qi, sb = qi & 1;
            if (qi >= 2) {
                if (!*abort_v && !mbar_wait(smem_u32(&s_empty[sb]), ((qi >> 1) - 1) & 1)) *abort_v = 1;
                // own previous copy into this buffer is complete before re-arming
                mbar_wait(smem_u32(&s_full[sb]), ((qi >> 1) - 1) & 1);
            }
            const uint32_t sbar = smem_u32(&s_full[sb]);
            mbar_expect_tx(sbar, 4u * n * 256u);
            for (int h = 0; h < 2; ++h)
                for (int hl = 0; hl < 2; ++hl)
                    bulk_g2s(smem_u32(slab + sb * buf + (h * 2 + hl) * blk + kPad * 256),
                             xt + ((long long)(2 * qc + h) * 2 + hl) * n * 64, (uint32_t)n * 256u, sbar);
        };
        if (nqc > 0) issue_slab(0);
        const int next_at = min(nd - 1, kStages);
        // ring position of the next A stage and the parity of its previous use
        int s = 0;
        uint32_t ph = 1;  // parity of the phase to wait for before reuse (first lap: none)
        bool lap1 = true;
        const float* gq = gt + (long long)(dlo + 2 * N) * (c.Mq / 4) * 2048;
        const long long dstep = (long long)(c.Mq / 4) * 2048;
        for (int qi = 0; qi < nqc; ++qi) {
            const float* gd = gq + (long long)(2 * (qc0 + qi)) * 2048;
            for (int t = 0; t < nd; ++t, gd += dstep) {
                // the next slab once kStages A stages of this K-step are issued:
                // the MMAs of K-step qi - 1 are then complete
                if (t == next_at && qi + 1 < nqc) issue_slab(qi + 1);
                if (!lap1) {
                    if (!*abort_v && !mbar_wait(smem_u32(&a_empty[s]), ph)) *abort_v = 1;
                    mbar_wait(smem_u32(&a_full[s]), ph);
                }
                const uint32_t abar = smem_u32(&a_full[s]);
                mbar_expect_tx(abar, kAStage);
                bulk_g2s(smem_u32(A + s * kAStage), gd, kAStage, abar);
                ++ait;
                if (++s == kStages) {
                    s = 0;
                    ph ^= 1;
                    if (lap1) {
                        lap1 = false;
                        ph = 0;
                    }
                }
            }
        }
        // every copy of this CTA has landed before it exits
        for (int s2 = 0; s2 < kStages; ++s2)
            if (ait > s2) mbar_wait(smem_u32(&a_full[s2]), (uint32_t)(((ait - 1 - s2) / kStages) & 1));
        for (int sb = 0; sb < 2; ++sb)
            if (nqc > sb) mbar_wait(smem_u32(&s_full[sb]), (uint32_t)(((nqc - 1 - sb) >> 1) & 1));
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issue
        // Descriptors are linear in the start address (field = address / 16),
        // so the per-stage and per-shift ones are base descriptors plus
        // offsets; stage and phase advance incrementally.
        const uint32_t id = idesc_tf32(128, 16 * mb);
        const uint32_t d2off = mb > kMbMax ? 256u : 128u;  // D2 after D1 (N = 16 mb columns each)
        const uint32_t sbo = 128;
        const uint64_t adesc0 = sdesc(smem_u32(A), 8192, sbo);
        const uint64_t bdesc0[2] = {sdesc(smem_u32(slab), 2 * blk, sbo), sdesc(smem_u32(slab + buf), 2 * blk, sbo)};
        const uint64_t blo = (uint64_t)(blk >> 4);
        int group = 0;
        int fresh = 3;  // bit b: the next MMA into block b's accumulators overwrites them
        bool first_wait = true;
        int s = 0;
        uint32_t ph = 0;  // parity of the stage's current fill
        for (int qi = 0; qi < nqc; ++qi) {
            const int sb = qi & 1;
            if (!*abort_v && !mbar_wait(smem_u32(&s_full[sb]), (qi >> 1) & 1)) *abort_v = 1;
            const uint64_t bd = bdesc0[sb];
            const bool fold_wait = qi % kFoldQc == 0 && group > 0;
            for (int d = dlo; d <= dhi; ++d) {
                bool ok = *abort_v ? true : mbar_wait(smem_u32(&a_full[s]), ph);
                if (expire_test && first_wait) ok = wait_unset_flag(&never_sh) && ok;
                first_wait = false;
                if (!ok) *abort_v = 1;
                if (fold_wait && d == dlo && !*abort_v && !mbar_wait(smem_u32(&acc_empty), (uint32_t)((group - 1) & 1)))
                    *abort_v = 1;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint64_t grh = adesc0 + (uint64_t)(s * (kAStage >> 4));
                const uint64_t grl = grh + 128, gih = grh + 256, gil = grh + 384;  // + 2, 4, 6 KB
                for (int b = 0; b < nmb; ++b) {
                    const int mb0 = m0 + b * mb;
                    const int mb1 = min(n, mb0 + mb) - 1;
                    if (d < -mb1 || d > n - 1 - mb0) continue;  // no mode of the block meets a source mode
                    const int jb = mb0 + d + kPad;  // first slab mode of the B operand
                    if (jb < 0 || jb + mb > n + 2 * kPad) {  // outside the slab block: never by construction
                        *abort_v = 1;
                        continue;
                    }
                    const uint64_t bh = bd + (uint64_t)(jb * 16), bl = bh + blo;  // jb * 256 bytes
                    const uint32_t d1 = tmem + (uint32_t)(b * 256), d2 = d1 + d2off;
                    const uint32_t acc = ((fresh >> b) & 1) ? 0u : 1u;
                    mma_tf32(d1, grh, bh, id, acc);
                    mma_tf32(d1, grh, bl, id, 1u);
                    mma_tf32(d1, grl, bh, id, 1u);
                    mma_tf32(d2, gih, bh, id, acc);
                    mma_tf32(d2, gih, bl, id, 1u);
                    mma_tf32(d2, gil, bh, id, 1u);
                    fresh &= ~(1 << b);
                    issued_mma = 1;
                }
                mma_commit(smem_u32(&a_empty[s]));
                if (++s == kStages) {
                    s = 0;
                    ph ^= 1;
                }
            }
            mma_commit(smem_u32(&s_empty[sb]));
            if ((qi + 1) % kFoldQc == 0 || qi == nqc - 1) {
                mma_commit(smem_u32(&acc_full));
                fresh = 3;
                ++group;
            }
        }
        if (issued_mma) mma_commit(smem_u32(&mma_done));
    } else if (warp >= 2) {
        // ---------------- fold the accumulators into FP32 registers (round to nearest)
        // warp group g = (warp - 2) / 4 folds block g (two blocks of <= 8
        // modes), or modes 8 g .. 8 g + 7 of the single block (<= 16 modes)
        const int quarter = warp & 3, g4 = (warp - 2) >> 2;
        const bool wide = mb > kMbMax;
        const int b = wide ? 0 : g4;
        const int u0 = wide ? kMbMax * g4 : 0;
        const int ucnt = wide ? min(kMbMax, mb - u0) : mb;
        const uint32_t d2off = wide ? 256u : 128u;
        const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256);
        float sr[kMbMax][kRC], si[kMbMax][kRC];
#pragma unroll
        for (int u = 0; u < kMbMax; ++u)
#pragma unroll
            for (int r = 0; r < kRC; ++r) sr[u][r] = si[u][r] = 0.f;
        for (int g = 0; g < ngroups; ++g) {
            bool ok = *abort_v ? false : mbar_wait(smem_u32(&acc_full), (uint32_t)(g & 1));
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) *abort_v = 1;
            if (ok && b < nmb) {
                asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
                for (int u = 0; u < kMbMax; ++u) {
                    if (u < ucnt) {
                        float v1[16], v2[16];
                        tmem_ld16(lane_addr + (u0 + u) * 16, v1);
                        tmem_ld16(lane_addr + d2off + (u0 + u) * 16, v2);
                        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                        for (int r = 0; r < kRC; ++r) {
                            sr[u][r] += v1[r] - v2[kRC + r];
                            si[u][r] += v1[kRC + r] + v2[r];
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&acc_empty));
        }
        if (!*abort_v && b < nmb) {
            const int p = w.p0 + quarter * 32 + lane;
            if (p < c.M) {
                float2* out = part + (long long)w.split * Ntot * R + rt * kRC;
#pragma unroll
                for (int u = 0; u < kMbMax; ++u) {
                    const int m = m0 + b * mb + u0 + u;
                    if (u < ucnt && m < n) {
                        float2* o = out + (c.row_off + (long long)p * n + m) * R;
#pragma unroll
                        for (int r = 0; r < kRC; r += 2)
                            *(float4*)(o + r) = make_float4(sr[u][r], si[u][r], sr[u][r + 1], si[u][r + 1]);
                    }
                }
            }
        }
    }
    // every MMA has completed before TMEM is freed
    __syncthreads();
    bool drained = true;
    if (tid == 32 && issued_mma) drained = mbar_wait(smem_u32(&mma_done), 0);
    drained = __syncthreads_and(drained);
    if (tid == 0 && (abort_sh || !drained)) atomicOr(&g_tcs_status, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// GT: generators of configuration c in the A-operand order of k_bt_tcs,
//   GT[c][ptile][d + 2N][q4][{Re hi, Re lo, Im hi, Im lo}][row 0..127][q 0..3]
// (q4 = group of 4 sources, sources padded to Mq = a multiple of 8 with
// zeros, targets padded to 128 with zeros), from the complex64 generators
// G[q][p][l] (l = d + 2N).  One CTA per (configuration, target tile, q4):
// 8 shifts at a time are staged through shared memory.
constexpr int kGtD = 8;
__global__ void __launch_bounds__(128) k_tcs_build_gt(const MsdConfig* __restrict__ cfgs, int C,
                                                      const long long* __restrict__ blk_off, const float2* __restrict__ G,
                                                      float* __restrict__ GT) {
    __shared__ float2 tile[4][128][kGtD + 1];
    // configuration of this block: blk_off[c] <= blockIdx.x < blk_off[c + 1]
    int lo = 0, hi = C - 1;
    const long long bid = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk_off[mid] <= bid) lo = mid;
        else hi = mid - 1;
    }
    const MsdConfig c = cfgs[lo];
    const long long local = bid - blk_off[lo];
    const int nq4 = c.Mq / 4;
    const int ptile = (int)(local / nq4), q4 = (int)(local % nq4);
    const int t = threadIdx.x;
    for (int d0 = 0; d0 < c.L; d0 += kGtD) {
        __syncthreads();
        // stage G[q][p][d0 .. d0 + 15] for the 4 sources and the 128 targets
        for (int i = t; i < 4 * 128 * kGtD; i += 128) {
            const int qq = i / (128 * kGtD), rem = i - qq * (128 * kGtD);
            const int pr = rem / kGtD, dd = rem - pr * kGtD;
            const int q = q4 * 4 + qq, pp = ptile * 128 + pr, l = d0 + dd;
            float2 v = make_float2(0.f, 0.f);
            if (q < c.M && pp < c.M && l < c.L) v = G[c.gen_off + ((long long)q * c.Mp + pp) * c.L + l];
            tile[qq][pr][dd] = v;
        }
        __syncthreads();
        for (int dd = 0; dd < kGtD && d0 + dd < c.L; ++dd) {
            float4 rh, rl, ih, il;
            float* prh = &rh.x;
            float* prl = &rl.x;
            float* pih = &ih.x;
            float* pil = &il.x;
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
                const float2 g = tile[qq][t][dd];
                const float gr = tf32_rna(g.x), gi = tf32_rna(g.y);
                prh[qq] = gr;
                prl[qq] = tf32_rna(g.x - gr);
                pih[qq] = gi;
                pil[qq] = tf32_rna(g.y - gi);
            }
            float* out = GT + c.gt_off + (((long long)ptile * c.L + d0 + dd) * nq4 + q4) * 2048 + t * 4;
            *(float4*)(out) = rh;
            *(float4*)(out + 512) = rl;
            *(float4*)(out + 1024) = ih;
            *(float4*)(out + 1536) = il;
        }
    }
}

// XT: the scaled columns xs = rf .* x in the slab order of k_bt_tcs,
//   XT[c][rtile][q4][{hi, lo}][j 0..n-1][{Re, Im}][r 0..7][q 0..3],
// sources padded to Mq with zeros.  One thread per (configuration rows of
// 4 sources, mode j, column r): reads the four source rows, writes one
// float4 (the 4 sources) per (hi/lo, Re/Im).
__global__ void k_tcs_prep_x(const MsdConfig* __restrict__ cfgs, int C, long long rows4, int R,
                             const float* __restrict__ rf, const float2* __restrict__ x, float* __restrict__ XT) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows4 * R) return;
    const long long row4 = i / R;  // index over (configuration, q4, j)
    const int r = (int)(i - row4 * R);
    // configuration: xrow_off[c] / 4 <= row4 (xrow_off counts rows of single sources)
    int lo = 0, hi = C - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cfgs[mid].xrow_off / 4 <= row4) lo = mid;
        else hi = mid - 1;
    }
    const MsdConfig c = cfgs[lo];
    const long long local = row4 - c.xrow_off / 4;
    const int q4 = (int)(local / c.n), j = (int)(local - (long long)q4 * c.n);
    float re[4], im[4];
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
        const int q = q4 * 4 + qq;
        re[qq] = im[qq] = 0.f;
        if (q < c.M) {
            const long long row = c.row_off + (long long)q * c.n + j;
            const float2 v = x[row * R + r];
            const float f = rf[row];
            re[qq] = v.x * f;
            im[qq] = v.y * f;
        }
    }
    float4 rh, rl, ih, il;
    float* prh = &rh.x;
    float* prl = &rl.x;
    float* pih = &ih.x;
    float* pil = &il.x;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
        prh[qq] = tf32_rna(re[qq]);
        prl[qq] = tf32_rna(re[qq] - prh[qq]);
        pih[qq] = tf32_rna(im[qq]);
        pil[qq] = tf32_rna(im[qq] - pih[qq]);
    }
    const int rt = r / kRC, rr = r - rt * kRC;
    float* base = XT + c.xrow_off * 4 * R + (long long)rt * c.Mq * c.n * 32 + (long long)q4 * c.n * 128 +
                  (long long)j * 64 + rr * 4;
    *(float4*)(base) = rh;                 // hi, Re
    *(float4*)(base + 32) = ih;            // hi, Im
    *(float4*)(base + c.n * 64) = rl;      // lo, Re
    *(float4*)(base + c.n * 64 + 32) = il;  // lo, Im
}

}  // namespace

// dynamic shared memory limit of the kernel: 227 KB less its static part
constexpr size_t kSmemCap = 226 * 1024;

size_t tcs_slab_bytes(int Nmax) { return 2 * 4 * (size_t)(2 * Nmax + 1 + 2 * kPad) * 256; }

// A stages that fit next to the two slab buffers (at most kStagesMax)
int tcs_stages(int Nmax) {
    const long long room = (long long)kSmemCap - 1024 - (long long)tcs_slab_bytes(Nmax);
    return (int)std::min<long long>(kStagesMax, std::max<long long>(0, room / kAStage));
}

size_t tcs_smem_bytes(int Nmax) { return (size_t)tcs_stages(Nmax) * kAStage + tcs_slab_bytes(Nmax) + 1024; }

bool tcs_supported(int R, int Nmax) { return R % kRC == 0 && tcs_stages(Nmax) >= 3; }

// Mode blocks of one configuration: block length mb (4..8), blocks grouped
// two per CTA (TMEM holds 2 blocks x (D1, D2) x 128 columns).  The choice
// minimises the streamed A stages per CTA group, n + span - 1 each, with
// the MMA work of padded modes as a tie-break.
void tcs_mode_blocks(int n, int* mb_out, int* nblocks_out, bool wide) {
    if (wide) {  // single blocks of at most kMbWide modes, balanced
        const int nb = (n + kMbWide - 1) / kMbWide;
        *mb_out = (n + nb - 1) / nb;
        *nblocks_out = nb;
        return;
    }
    double best = 1e300;
    for (int mb = 4; mb <= kMbMax; ++mb) {
        const int nb = (n + mb - 1) / mb;
        const int groups = (nb + 1) / 2;
        double cost = 0;
        for (int g = 0; g < groups; ++g) {
            const int blocks = std::min(2, nb - 2 * g);
            const int span = std::min(n, (2 * g + blocks) * mb) - 2 * g * mb;
            cost += (double)(n + span - 1) * (1.0 + 0.02 * blocks * mb);
        }
        if (cost < best - 1e-9) {
            best = cost;
            *mb_out = mb;
            *nblocks_out = nb;
        }
    }
}

void launch_bt_tcs(const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, int Nmax, const float* GT,
                   const float* XT, float2* part, long long Ntot, int R, cudaStream_t s, const int* live) {
    if (nwork <= 0) return;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_bt_tcs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
        attr = true;
    }
    const int rtiles = R / kRC;
    k_bt_tcs<<<(unsigned)((long long)nwork * rtiles), kThreads, tcs_smem_bytes(Nmax), s>>>(
        d_cfg, d_work, GT, XT, part, Ntot, R, rtiles, tcs_stages(Nmax), g_msd_expire_waits.load(), live);
    g_msd_launches += 1;
}

void launch_tcs_build_gt(const MsdConfig* d_cfg, int C, const long long* d_blk_off, long long nblocks,
                         const float2* G32, float* GT, cudaStream_t s) {
    if (nblocks <= 0) return;
    k_tcs_build_gt<<<(unsigned)nblocks, 128, 0, s>>>(d_cfg, C, d_blk_off, G32, GT);
    g_msd_launches += 1;
}

void launch_tcs_prep_x(const MsdConfig* d_cfg, int C, long long rows4, int R, const float* rf, const float2* x,
                       float* XT, cudaStream_t s) {
    const long long tot = rows4 * R;
    if (tot <= 0) return;
    k_tcs_prep_x<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d_cfg, C, rows4, R, rf, x, XT);
    g_msd_launches += 1;
}

int tcs_status_and_clear() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tcs_status, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_tcs_status, &z, sizeof(int));
    }
    return v;
}
