// C ABI of libmsd (declared in include/msd.h) and the host-side runtime:
// problem plans (row/generator offsets, matvec work lists, reduction
// chunks), device work buffers, and the restarted-GMRES driver that chains
// the kernels of K3/K4 on the problem's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "msd_internal.cuh"

// ---------------------------------------------------------------- errors

std::atomic<long long> g_msd_launches{0};
std::atomic<int> g_msd_expire_waits{0};

namespace {
thread_local std::string g_err;

struct MsdError {
    msd_status st;
};

void fail(msd_status st, const std::string& msg) {
    g_err = msg;
    throw MsdError{st};
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            cudaGetLastError();                                                                   \
            fail(e_ == cudaErrorMemoryAllocation ? MSD_ERR_OOM : MSD_ERR_CUDA,                    \
                 std::string(#call) + ": " + cudaGetErrorString(e_));                             \
        }                                                                                         \
    } while (0)

#define CK_LAUNCH() CK(cudaGetLastError())

template <typename F>
msd_status guarded(F&& f) {
    try {
        g_err.clear();
        return f();
    } catch (const MsdError& e) {
        return e.st;
    } catch (const std::bad_alloc&) {
        g_err = "host allocation failed";
        return MSD_ERR_OOM;
    } catch (...) {
        g_err = "unexpected internal error";
        return MSD_ERR_CUDA;
    }
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// True when the byte ranges [x, x + bytes) and [y, y + bytes) intersect.
bool ranges_overlap(const void* x, const void* y, size_t bytes) {
    const uintptr_t a = (uintptr_t)x, b = (uintptr_t)y;
    return a < b + bytes && b < a + bytes;
}

// Growable device buffer owned by the library.
struct DBuf {
    void* p = nullptr;
    size_t cap = 0;
    void* get(size_t bytes) {
        if (bytes > cap) {
            if (p) cudaFree(p);
            p = nullptr;
            cap = 0;
            CK(cudaMalloc(&p, bytes ? bytes : 16));
            cap = bytes;
        }
        return p;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

template <typename T>
T* dalloc_copy(const T* h, size_t n) {
    T* d = nullptr;
    CK(cudaMalloc(&d, std::max<size_t>(n, 1) * sizeof(T)));
    if (n) CK(cudaMemcpy(d, h, n * sizeof(T), cudaMemcpyHostToDevice));
    return d;
}
template <typename T>
T* dalloc(size_t n) {
    T* d = nullptr;
    CK(cudaMalloc(&d, std::max<size_t>(n, 1) * sizeof(T)));
    return d;
}

}  // namespace

// ---------------------------------------------------------------- problem

struct MatvecPlan {
    std::vector<MatvecWork> work;
    MatvecWork* d_work = nullptr;
    int nsplit = 1;
    MatvecChoice ch{0, 1, 1, 0};  // tile shape of the product kernel
    int ns_div = 1;               // split count = the wave model's / ns_div
    int candidates = 0;           // shapes the autotuner timed (0: model choice)
    double tuned_ms = 0;          // kernel time of the chosen shape in the tuning run
};

// Product plan with recomputed generators: chunks of generator blocks
// (configuration x target range x source range) small enough to stay in L2;
// per chunk the generator kernel fills the chunk buffer and the product
// kernel reads it through a configuration array whose generator offset and
// target stride address that buffer.
struct RecomputeChunk {
    MsdConfig* d_cfg = nullptr;  // [C] copies with gen_off/Mp of this chunk
    GenBlock* d_blocks = nullptr;
    int nblocks = 0;
    long long nitems = 0;
    MatvecWork* d_work = nullptr;
    int nwork = 0;
};

struct RecomputePlan {
    std::vector<RecomputeChunk> chunks;
    size_t buf_elems = 0;  // largest chunk buffer (complex elements)
    int nsplit = 1;
    MatvecChoice ch{0, 1, 1, 0};
};

struct msd_problem {
    cudaStream_t stream = nullptr;
    int C = 0, Mtot = 0, Nmax = 0, Mmax = 0;
    long long Ntot = 0;
    std::vector<MsdConfig> cfg;
    MsdConfig* d_cfg = nullptr;
    double2* d_centre = nullptr;
    double* d_radius = nullptr;
    int8_t* d_bc = nullptr;
    int* d_disk_cfg = nullptr;
    double2 *d_J = nullptr, *d_dJ = nullptr, *d_H = nullptr, *d_dH = nullptr;
    double2 *d_lf64 = nullptr, *d_rhs_scale = nullptr;
    double* d_rf64 = nullptr;
    float2* d_lf32 = nullptr;
    float* d_rf32 = nullptr;
    int* d_flags = nullptr;
    long long gen_elems = 0;
    double2* d_G64 = nullptr;
    float2* d_G32 = nullptr;
    // adjoint operator data: GA[p][q][l] = conj(g^pq_{-l}), conj(l); rebuilt
    // when the geometry version moves on
    double2* d_GA64 = nullptr;
    float2* d_GA32 = nullptr;
    double2* d_clf64 = nullptr;
    float2* d_clf32 = nullptr;
    long long geom_version = 0, adj64_version = -1, adj32_version = -1, adj_rows_version = -1;
    std::map<long long, MatvecPlan> plans;  // key: R*4 + precision
    std::map<long long, MatvecChoice> pinned;  // shapes fixed by msd_set_tile
    // generator mode of the forward products (msd_set_generator_mode)
    int gen_mode = MSD_GEN_STREAMED;
    size_t gen_chunk_bytes = 64ull << 20;
    std::vector<GenBlock> gen_full;  // one block per configuration: the stored array
    GenBlock* d_gen_full = nullptr;
    std::map<long long, RecomputePlan> rplans;  // key: R*4 + precision
    DBuf genbuf;
    long long rc_checked = -1;  // geometry version whose complex64 range was checked
    std::vector<RowChunk> chunks;
    RowChunk* d_chunks = nullptr;
    int* d_cfg_chunk_off = nullptr;
    // coarse reduction chunks (>= 4096 rows): projections onto many basis
    // vectors give each thread enough rows to amortise its reductions
    std::vector<RowChunk> chunks_coarse;
    RowChunk* d_chunks_coarse = nullptr;
    int* d_cfg_chunk_off_coarse = nullptr;
    // medium chunks (>= 1024 rows) for the warp-per-vector projections onto
    // many basis vectors: each warp streams twice the rows of a fine chunk
    std::vector<RowChunk> chunks_mid;
    RowChunk* d_chunks_mid = nullptr;
    int* d_cfg_chunk_off_mid = nullptr;
    int* h_pinned = nullptr;  // small pinned host flags: [0..1] sync reads, [2..9] ring of step flags, [10] DORT barrier
    int* d_hpinned = nullptr;  // the same flags as the device addresses them (mapped host memory)
    cudaEvent_t ring_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    DBuf xs, part, sbuf[24];
    DBuf gbuf[9];   // gradient work buffers
    DBuf nfbuf[4];  // near-field buffers: rho, points, weights, output stage
    DBuf dortbuf[6];  // time reversal: rho, angles, F, T, eigenvalues, eigen work
    // integral-equation formulation (msd_set_formulation); form == false: the
    // default rows (L on sound-soft disks, -I/2 + N on sound-hard ones, u = L rho)
    bool form = false;
    MsdFormulation fw{};
    DBuf fbuf;  // the per-row factors below, in one allocation
    double2 *d_fl1_64 = nullptr, *d_fl2_64 = nullptr, *d_frs = nullptr, *d_fff = nullptr, *d_fdiag = nullptr;
    float2 *d_fl1_32 = nullptr, *d_fl2_32 = nullptr;
    double* d_frf2_64 = nullptr;
    float* d_frf2_32 = nullptr;
    // penetrable obstacles (msd_set_penetrable): the same geometry at the
    // interior wavenumber k- (its Bessel diagonals and generators), and the
    // problem whose 2 M disk slots per configuration give the Krylov solver
    // the row layout of (rho+, rho-); pen_parent is set on the latter
    msd_problem* pen_minus = nullptr;
    msd_problem* pen_shadow = nullptr;
    msd_problem* pen_parent = nullptr;
    DBuf penbuf;     // A64 [Ntot][4], A32 [Ntot][4], S64 [2][Ntot], mu [Mtot]
    DBuf penio[4];   // transmission-layout vectors and right-hand sides
    double2* d_penA64 = nullptr;
    float2* d_penA32 = nullptr;
    double2* d_penS = nullptr;
    double* d_pen_mu = nullptr;
    // shift-GEMM tensor-core product: the complex64 generators in its
    // A-operand order (TF32 hi/lo), built for geometry version gt_version;
    // xrows = sum over configurations of Mq * n (its source rows per column)
    // active flags [C*R] of the Krylov systems while an Arnoldi step runs its
    // product (nullptr otherwise): forward products of the default rows skip
    // the tiles none of whose columns are active (converged systems, whose
    // columns of the step are never read) and leave zero sums there
    const int* live = nullptr;
    // the product input whose scaled columns rf .* x the last Arnoldi step
    // already wrote into xs (FP32 products of the default rows only; nullptr
    // otherwise); consumed by the next product
    const void* xs_src = nullptr;
    // per-disk truncation orders (msd_set_truncation); d_Np == nullptr: N of
    // the configuration on every disk
    std::vector<int> Np;
    int* d_Np = nullptr;
    float* d_GT = nullptr;
    long long gt_floats = 0, gt_blocks = 0, xrows = 0, gt_version = -1;
    long long* d_gt_blk = nullptr;
    DBuf xt;
    // algorithmic size of one product with one column (section 5 storage):
    // sum over ordered pairs of the generator length, and of n^2
    double offdiag_L = 0, offdiag_n2 = 0;
    // optional timing of the block-Toeplitz kernel (msd_matvec_timing)
    bool timing = false;
    std::vector<cudaEvent_t> events;
    size_t ev_used = 0;
    double timed_ms = 0, timed_flops = 0, timed_bytes = 0;
    long long timed_launches = 0;
};

namespace {

// Fold the recorded kernel-event pairs into the running totals.
void flush_timing(msd_problem* pb) {
    if (pb->ev_used == 0) return;
    CK(cudaEventSynchronize(pb->events[pb->ev_used - 1]));
    for (size_t i = 0; i + 1 < pb->ev_used; i += 2) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, pb->events[i], pb->events[i + 1]));
        pb->timed_ms += ms;
        pb->timed_launches += 1;
    }
    pb->ev_used = 0;
}

// A pipeline wait of the tensor-core product expired (results invalid).
void check_tc(const char* where) {
    const int t = tc_status_and_clear();
    const int u = tcs_status_and_clear();
    if (t > 0 || u > 0) fail(MSD_ERR_CUDA, std::string(where) + ": a tensor-core pipeline wait expired");
    if (bt_status_and_clear() > 0) fail(MSD_ERR_CUDA, std::string(where) + ": a generator bulk-copy wait expired");
}

void check_flags(msd_problem* pb, const char* where) {
    int f = 0;
    CK(cudaMemcpyAsync(&f, pb->d_flags, sizeof(int), cudaMemcpyDeviceToHost, pb->stream));
    CK(cudaStreamSynchronize(pb->stream));
    check_tc(where);
    if (f & 1) fail(MSD_ERR_NONFINITE, std::string(where) + ": non-finite Bessel factor (k a_p at a zero of J_m for a Neumann disk?)");
    if (f & 2) fail(MSD_ERR_RANGE, std::string(where) + ": a Hankel generator exceeds the complex64 range; use MSD_FP64");
}

// Right-hand-side scale and field factor of the current formulation.
const double2* rhs_scale_of(const msd_problem* pb) { return pb->form ? pb->d_frs : pb->d_rhs_scale; }
const double2* field_factor_of(const msd_problem* pb) { return pb->form ? pb->d_fff : pb->d_J; }

// Per-row factors of the formulation pb->fw (after the Bessel diagonals).
void form_rows(msd_problem* pb) {
    const size_t n = (size_t)pb->Ntot;
    char* b = (char*)pb->fbuf.get(n * (5 * 16 + 2 * 8 + 8 + 4));
    pb->d_fl1_64 = (double2*)b;
    pb->d_fl2_64 = pb->d_fl1_64 + n;
    pb->d_frs = pb->d_fl2_64 + n;
    pb->d_fff = pb->d_frs + n;
    pb->d_fdiag = pb->d_fff + n;
    pb->d_fl1_32 = (float2*)(pb->d_fdiag + n);
    pb->d_fl2_32 = pb->d_fl1_32 + n;
    pb->d_frf2_64 = (double*)(pb->d_fl2_32 + n);
    pb->d_frf2_32 = (float*)(pb->d_frf2_64 + n);
    CK(cudaMemsetAsync(pb->d_flags, 0, sizeof(int), pb->stream));
    launch_form_rows(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_radius, pb->d_bc, pb->d_J, pb->d_dJ, pb->d_H,
                     pb->d_dH, pb->fw, pb->d_fl1_64, pb->d_fl2_64, pb->d_fl1_32, pb->d_fl2_32, pb->d_frf2_64,
                     pb->d_frf2_32, pb->d_frs, pb->d_fff, pb->d_fdiag, pb->d_flags, pb->stream);
    CK_LAUNCH();
    int f = 0;
    CK(cudaMemcpyAsync(&f, pb->d_flags, sizeof(int), cudaMemcpyDeviceToHost, pb->stream));
    CK(cudaStreamSynchronize(pb->stream));
    if (f & 1)
        fail(MSD_ERR_NONFINITE,
             "msd_set_formulation: the self block of the combination vanishes for some mode (a resonance of this "
             "formulation at k a_p)");
}

// Per-disk truncation: mask the default rows' factors (after every K1).
void apply_truncation(msd_problem* pb) {
    if (!pb->d_Np) return;
    launch_mask_rows(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_Np, pb->d_lf64, pb->d_lf32, pb->d_rf64, pb->d_rf32,
                     pb->d_rhs_scale, pb->stream);
    CK_LAUNCH();
}

// Algorithmic size of one product (generator values and multiply-adds of
// the off-diagonal blocks) with the truncation orders in force.
void count_offdiag(msd_problem* pb) {
    pb->offdiag_L = pb->offdiag_n2 = 0;
    for (const MsdConfig& c : pb->cfg) {
        double sN = 0, sn = 0, sn2 = 0;
        for (int d = c.disk_off; d < c.disk_off + c.M; ++d) {
            const int np = pb->Np.empty() ? c.N : pb->Np[d];
            sN += np;
            sn += 2.0 * np + 1;
            sn2 += (2.0 * np + 1) * (2.0 * np + 1);
        }
        pb->offdiag_L += 4.0 * (c.M - 1) * sN + (double)c.M * (c.M - 1);
        pb->offdiag_n2 += sn * sn - sn2;
    }
}

// Per-row transmission factors from the Bessel diagonals at k+ and k-.
void pen_rows(msd_problem* pb) {
    CK(cudaMemsetAsync(pb->d_flags, 0, sizeof(int), pb->stream));
    msd_problem* pm = pb->pen_minus;
    launch_pen_rows(pb->d_cfg, pm->d_cfg, pb->Mtot, pb->Ntot, pb->d_disk_cfg, pb->d_radius, pb->d_pen_mu, pb->d_J,
                    pb->d_dJ, pb->d_H, pb->d_dH, pm->d_J, pm->d_dJ, pm->d_H, pm->d_dH, pb->d_penA64, pb->d_penA32,
                    pb->d_penS, pb->d_flags, pb->stream);
    CK_LAUNCH();
    int f = 0;
    CK(cudaMemcpyAsync(&f, pb->d_flags, sizeof(int), cudaMemcpyDeviceToHost, pb->stream));
    CK(cudaStreamSynchronize(pb->stream));
    if (f & 1) fail(MSD_ERR_NONFINITE, "msd_set_penetrable: a 2 x 2 self block of the transmission system is singular");
}

void pen_release(msd_problem* pb) {
    if (pb->pen_minus) msd_destroy(pb->pen_minus);
    if (pb->pen_shadow) msd_destroy(pb->pen_shadow);
    pb->pen_minus = pb->pen_shadow = nullptr;
}

// K2 over the whole problem: the stored generator array(s).
void launch_full_generators(msd_problem* pb, double2* G64, float2* G32) {
    if (!pb->d_gen_full) {
        pb->gen_full.clear();
        long long items = 0;
        for (int ci = 0; ci < pb->C; ++ci) {
            const MsdConfig& c = pb->cfg[ci];
            GenBlock g{ci, 0, c.Mp, 0, c.M, 0, items, c.gen_off};
            pb->gen_full.push_back(g);
            items += (long long)c.M * c.Mp;
        }
        pb->d_gen_full = dalloc_copy(pb->gen_full.data(), pb->gen_full.size());
    }
    const GenBlock& last = pb->gen_full.back();
    launch_generator_blocks(pb->d_cfg, pb->d_gen_full, pb->C, last.item_off + (long long)last.Qb * last.Pc,
                            pb->d_centre, G64, G32, pb->d_flags, pb->stream);
}

void ensure_generators(msd_problem* pb, bool fp64) {
    if (fp64 && pb->d_G64) return;
    if (!fp64 && pb->d_G32) return;
    if (fp64) pb->d_G64 = dalloc<double2>(pb->gen_elems);
    else pb->d_G32 = dalloc<float2>(pb->gen_elems);
    launch_full_generators(pb, fp64 ? pb->d_G64 : nullptr, fp64 ? nullptr : pb->d_G32);
    CK_LAUNCH();
    check_flags(pb, "pair generators");
}

// Generators of the shift-GEMM tensor-core product (A-operand order, TF32
// hi/lo), rebuilt after a geometry update.  Returns false when they would
// take more than 60 % of the free device memory (the kernel is then not
// offered).
bool ensure_gt(msd_problem* pb) {
    ensure_generators(pb, false);
    if (!pb->d_GT) {
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        if ((double)pb->gt_floats * 4.0 > 0.6 * (double)free_b) return false;
        pb->d_GT = dalloc<float>(pb->gt_floats);
        pb->gt_version = -1;
    }
    if (pb->gt_version != pb->geom_version) {
        launch_tcs_build_gt(pb->d_cfg, pb->C, pb->d_gt_blk, pb->gt_blocks, pb->d_G32, pb->d_GT, pb->stream);
        CK_LAUNCH();
        pb->gt_version = pb->geom_version;
    }
    return true;
}

// Target tiles of a product kernel within [P0, P1) (multiples of 32): 32
// disks for the CUDA-core kernel; for the tensor-core kernel floor(128 / n)
// disks, restarted at every 32-disk boundary and cut at M.
void tile_starts(const MsdConfig& c, int P0, int P1, const MatvecChoice& ch, std::vector<int>& out) {
    out.clear();
    if (!ch.TC) {
        for (int p0 = P0; p0 < P1; p0 += MSD_TILE_P) out.push_back(p0);
        return;
    }
    const int tp = tc_tile_disks(c.n);
    for (int b = P0; b < P1; b += MSD_TILE_P)
        for (int p0 = b; p0 < b + MSD_TILE_P && p0 < c.M; p0 += tp) out.push_back(p0);
}

// Work list of a plan: every target tile of every configuration, its
// sources split into ns ranges.  ns is chosen so that the CTAs fill whole
// waves of the resident slots: efficiency(ns) = (work items / slots) /
// ceil(...) times the balance of the largest source range against the mean.
void build_work_tcs(msd_problem* pb, MatvecPlan& plan, int R) {
    const int rtiles = R / MSD_TCS_COLS;
    const bool wide = plan.ch.SH == 2;
    const int per_cta = wide ? 1 : 2;  // mode blocks per CTA
    long long units = 0;
    for (auto& c : pb->cfg) {
        int mb = 8, nb = 1;
        tcs_mode_blocks(c.n, &mb, &nb, wide);
        units += (long long)((c.M + 127) / 128) * ((nb + per_cta - 1) / per_cta) * rtiles;
    }
    int sms = 0, dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long slots = sms;
    int ns = 1;
    double best = -1;
    const int qc_max = (pb->Mmax + 7) / 8;
    for (int t = 1; t <= std::min(64, qc_max); ++t) {
        if (t > 1 && (size_t)t * pb->Ntot * R * 8 > (2ull << 30)) break;  // partial sums <= 2 GB
        const double waves = (double)(units * t) / slots;
        const double fill = waves / std::ceil(waves);
        const double per = (double)qc_max / t;
        const double bal = per / std::ceil(per);
        const double eff = fill * bal;
        if (eff > best + 1e-9) {
            best = eff;
            ns = t;
        }
    }
    ns = std::max(1, ns / plan.ns_div);
    plan.nsplit = ns;
    plan.work.clear();
    for (int ci = 0; ci < pb->C; ++ci) {
        const MsdConfig& c = pb->cfg[ci];
        int mb = 8, nb = 1;
        tcs_mode_blocks(c.n, &mb, &nb, wide);
        if (16 * mb > 208 || mb < 1 || (!wide && mb > 8))
            fail(MSD_ERR_ARG, "shift-GEMM product: mode block outside the validated MMA shapes");
        const int nqc = c.Mq / 8;
        for (int p0 = 0; p0 < c.M; p0 += 128)
            for (int b0 = 0; b0 < nb; b0 += per_cta) {
                const int nmb = std::min(per_cta, nb - b0);
                for (int sp = 0; sp < ns; ++sp) {
                    const int qc0 = (int)((long long)nqc * sp / ns), qc1 = (int)((long long)nqc * (sp + 1) / ns);
                    MatvecWork w;
                    w.cfg = ci;
                    w.p0 = p0;
                    w.q0 = qc0 * 8;
                    w.q1 = std::min(c.M, qc1 * 8);
                    w.split = sp;
                    w.pad = (b0 * mb) | (mb << 8) | (nmb << 12);
                    plan.work.push_back(w);
                }
            }
    }
}

void build_work(msd_problem* pb, MatvecPlan& plan, int R, bool fp64) {
    if (plan.ch.SH) {
        build_work_tcs(pb, plan, R);
        return;
    }
    const int rtiles = R / plan.ch.RT;
    std::vector<int> starts;
    long long tiles = 0;
    for (auto& c : pb->cfg) {
        tile_starts(c, 0, c.Mp, plan.ch, starts);
        tiles += (long long)starts.size();
    }
    int sms = 0, dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long slots = (long long)sms * matvec_blocks_per_sm(plan.ch, pb->Nmax, fp64);
    const long long units = tiles * rtiles;
    const size_t elem = fp64 ? 16 : 8;
    int ns = 1;
    double best = -1;
    for (int t = 1; t <= std::min(64, std::max(1, pb->Mmax / 2)); ++t) {
        if (t > 1 && (size_t)t * pb->Ntot * R * elem > (2ull << 30)) break;  // partial sums <= 2 GB
        const double waves = (double)(units * t) / slots;
        const double fill = waves / std::ceil(waves);
        const double per = (double)pb->Mmax / t;
        const double bal = per / std::ceil(per);
        const double eff = fill * bal;
        if (eff > best + 1e-9) {
            best = eff;
            ns = t;
        }
    }
    ns = std::max(1, ns / plan.ns_div);
    plan.nsplit = ns;
    plan.work.clear();
    for (int ci = 0; ci < pb->C; ++ci) {
        const MsdConfig& c = pb->cfg[ci];
        tile_starts(c, 0, c.Mp, plan.ch, starts);
        for (int p0 : starts)
            for (int s = 0; s < ns; ++s) {
                MatvecWork w;
                w.cfg = ci;
                w.p0 = p0;
                w.q0 = (int)((long long)c.M * s / ns);
                w.q1 = (int)((long long)c.M * (s + 1) / ns);
                w.split = s;
                w.pad = 0;
                plan.work.push_back(w);
            }
    }
}

// Autotuner: time the product kernel of every candidate tile shape (with its
// own split count) on the problem's generators and keep the fastest.  Large
// products are timed on a prefix of the work list of about 20 ms, scaled to
// the whole list.  Results are cached per process by problem shape.  The
// tuning run synchronises the stream; MSD_AUTOTUNE=0 keeps the model choice.
bool autotune_enabled() {
    const char* e = std::getenv("MSD_AUTOTUNE");
    return !(e && e[0] == '0');
}

typedef std::tuple<int, int, int, int, long long, int, int> TuneKey;  // Nmax R fp64 C Ntot Mmax device
struct TuneResult {
    MatvecChoice ch;
    int ns_div;
    double ms;
};

void autotune(msd_problem* pb, MatvecPlan& plan, int R, bool fp64, bool allow_sh) {
    static std::mutex mu;
    static std::map<TuneKey, TuneResult> cache;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    const TuneKey key{pb->Nmax, R, (fp64 ? 1 : 0) + (allow_sh ? 2 : 0), pb->C, pb->Ntot, pb->Mmax, dev};
    MatvecChoice cand[128];
    const int nc = matvec_candidates(R, pb->Nmax, fp64, cand, 128, allow_sh);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            plan.ch = it->second.ch;
            plan.ns_div = it->second.ns_div;
            plan.tuned_ms = it->second.ms;
            plan.candidates = nc;
            return;
        }
    }
    if (nc <= 1) return;
    const size_t elem = fp64 ? 16 : 8;
    const size_t vec = (size_t)pb->Ntot * R * elem;
    void* xs = pb->xs.get(vec);
    CK(cudaMemsetAsync(xs, 0, vec, pb->stream));
    const void* G = fp64 ? (const void*)pb->d_G64 : (const void*)pb->d_G32;
    // estimated full time (FP64 ~1.2 TFLOP/s, FP32 ~40 TFLOP/s) -> prefix fraction
    const double est_ms = 8.0 * R * pb->offdiag_n2 / (fp64 ? 1.2e9 : 4.0e10);
    const double frac = est_ms > 20.0 ? 20.0 / est_ms : 1.0;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    DBuf dwork;
    double best_ms = 1e300;
    MatvecChoice best = plan.ch;
    int best_div = 1;
    // every shape at the wave model's split count and at a half, a quarter
    // and an eighth of it (fewer, longer source ranges: less partial-sum
    // traffic and per-CTA set-up, at some cost in wave fill)
    constexpr int kDivs[4] = {1, 2, 4, 8};
    int model_ns = 1;
    for (int i = 0; i < 4 * nc; ++i) {
        const int dv = kDivs[i & 3];
        if (dv > 1 && model_ns / (dv / 2) <= 1) continue;  // the same plan as a smaller divisor
        MatvecPlan trial;
        trial.ch = cand[i / 4];
        trial.ns_div = dv;
        float* XT = nullptr;
        if (trial.ch.SH) {
            if (!ensure_gt(pb)) continue;
            XT = (float*)pb->xt.get((size_t)pb->xrows * 4 * R * sizeof(float));
            CK(cudaMemsetAsync(XT, 0, (size_t)pb->xrows * 4 * R * sizeof(float), pb->stream));
        }
        build_work(pb, trial, R, fp64);
        if (dv == 1) model_ns = trial.nsplit;
        const int nfull = (int)trial.work.size();
        const int nw = std::max(1, std::min(nfull, (int)std::ceil(frac * nfull)));
        MatvecWork* dw = (MatvecWork*)dwork.get(nfull * sizeof(MatvecWork));
        CK(cudaMemcpyAsync(dw, trial.work.data(), nw * sizeof(MatvecWork), cudaMemcpyHostToDevice, pb->stream));
        void* part = pb->part.get((size_t)trial.nsplit * vec);
        double t = 1e300;
        for (int rep = 0; rep < 3; ++rep) {  // first run warms caches and the module
            CK(cudaEventRecord(e0, pb->stream));
            if (trial.ch.SH)
                launch_bt_tcs(pb->d_cfg, dw, nw, pb->Nmax, pb->d_GT, XT, (float2*)part, pb->Ntot, R, pb->stream);
            else
                launch_bt_only(cand[i / 4], fp64, pb->d_cfg, dw, nw, pb->Nmax, G, xs, part, pb->Ntot, R, pb->stream);
            CK_LAUNCH();
            CK(cudaEventRecord(e1, pb->stream));
            CK(cudaEventSynchronize(e1));
            check_tc("autotune");
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) t = std::min(t, (double)ms * nfull / nw);
        }
        if (t < best_ms) {
            best_ms = t;
            best = cand[i / 4];
            best_div = trial.ns_div;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dwork.release();
    plan.ch = best;
    plan.ns_div = best_div;
    plan.tuned_ms = best_ms;
    plan.candidates = nc;
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = TuneResult{best, best_div, best_ms};
}

// Plans are kept per (R, precision) and per use: allow_sh = the forward
// product of the default rows with stored generators (matvec_dev), the only
// one that may run the shift-GEMM kernel; every other product (formulations,
// penetrable, adjoint, raw, recomputed) uses a plan without it.
long long plan_key(int R, bool fp64, bool allow_sh) {
    return ((long long)R * 4 + (fp64 ? 0 : 1)) * 2 + (allow_sh ? 1 : 0);
}

MatvecPlan& get_plan(msd_problem* pb, int R, bool fp64, bool allow_sh = false) {
    allow_sh = allow_sh && !fp64;
    const long long key = plan_key(R, fp64, allow_sh);
    auto it = pb->plans.find(key);
    if (it != pb->plans.end()) return it->second;
    MatvecPlan plan;
    auto pin = pb->pinned.find((long long)R * 4 + (fp64 ? 0 : 1));
    if (pin != pb->pinned.end()) {
        plan.ch = pin->second;
        if (plan.ch.SH && !(allow_sh && ensure_gt(pb))) plan.ch = matvec_default_choice(R, pb->Nmax, fp64);
    } else {
        plan.ch = matvec_default_choice(R, pb->Nmax, fp64);
        if (autotune_enabled()) autotune(pb, plan, R, fp64, allow_sh);
    }
    build_work(pb, plan, R, fp64);
    plan.d_work = dalloc_copy(plan.work.data(), plan.work.size());
    return pb->plans.emplace(key, std::move(plan)).first->second;
}

// Chunks of a recomputed product.  A configuration whose M x Mp pairs fit
// the budget is one block (several such share a chunk); a larger one is cut
// into blocks of Qb >= 32 sources by Pc targets (multiples of 32), one
// chunk each.  Work items split each block's sources into ns ranges; the
// items of blocks with Q0 > 0 add to the partial sums (pad = 1).
RecomputePlan build_recompute_plan(msd_problem* pb, int R, bool fp64, const MatvecChoice& choice) {
    RecomputePlan rp;
    rp.ch = choice;
    const size_t elem = fp64 ? 16 : 8;
    const long long budget = std::max<long long>(1, (long long)(pb->gen_chunk_bytes / (elem * (4 * pb->Nmax + 1))));
    // blocks grouped into chunks
    std::vector<std::vector<GenBlock>> groups;
    std::vector<GenBlock> cur;
    long long cur_rows = 0;
    auto flush = [&]() {
        if (!cur.empty()) groups.push_back(cur);
        cur.clear();
        cur_rows = 0;
    };
    for (int ci = 0; ci < pb->C; ++ci) {
        const MsdConfig& c = pb->cfg[ci];
        const long long rows = (long long)c.M * c.Mp;
        if (rows <= budget) {
            if (cur_rows + rows > budget) flush();
            cur.push_back(GenBlock{ci, 0, c.Mp, 0, c.M, 0, 0, 0});
            cur_rows += rows;
            continue;
        }
        flush();
        const int Qb = std::min<long long>(c.M, std::max<long long>(32, budget / c.Mp));
        const int Pc = (int)std::min<long long>(c.Mp, MSD_TILE_P * std::max<long long>(1, budget / (MSD_TILE_P * (long long)Qb)));
        for (int P0 = 0; P0 < c.Mp; P0 += Pc)
            for (int Q0 = 0; Q0 < c.M; Q0 += Qb) {
                groups.push_back({GenBlock{ci, P0, std::min(Pc, c.Mp - P0), Q0, std::min(Qb, c.M - Q0), 0, 0, 0}});
            }
    }
    flush();
    // splits: enough CTAs in the largest chunk to fill the resident slots
    int sms = 0, dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long slots = (long long)sms * matvec_blocks_per_sm(rp.ch, pb->Nmax, fp64);
    long long max_units = 1;
    int min_q = 1 << 30;
    std::vector<int> starts;
    for (auto& g : groups) {
        long long u = 0;
        for (auto& b : g) {
            tile_starts(pb->cfg[b.cfg], b.P0, b.P0 + b.Pc, rp.ch, starts);
            u += (long long)starts.size() * (R / rp.ch.RT);
            min_q = std::min(min_q, b.Qb);
        }
        max_units = std::max(max_units, u);
    }
    int ns = (int)std::min<long long>(64, std::max<long long>(1, (slots + max_units - 1) / max_units));
    ns = std::max(1, std::min(ns, std::max(1, min_q / 2)));
    while (ns > 1 && (size_t)ns * pb->Ntot * R * elem > (2ull << 30)) --ns;
    rp.nsplit = ns;
    for (auto& g : groups) {
        RecomputeChunk ch;
        std::vector<MsdConfig> ccfg = pb->cfg;
        std::vector<MatvecWork> work;
        long long items = 0, out = 0;
        for (auto& b : g) {
            const MsdConfig& c = pb->cfg[b.cfg];
            b.item_off = items;
            b.out_off = out;
            ccfg[b.cfg].Mp = b.Pc;
            ccfg[b.cfg].gen_off = out - ((long long)b.Q0 * b.Pc + b.P0) * c.L;
            items += (long long)b.Qb * b.Pc;
            out += (long long)b.Qb * b.Pc * c.L;
            tile_starts(c, b.P0, b.P0 + b.Pc, rp.ch, starts);
            for (int p0 : starts)
                for (int sp = 0; sp < ns; ++sp) {
                    MatvecWork w;
                    w.cfg = b.cfg;
                    w.p0 = p0;
                    w.q0 = b.Q0 + (int)((long long)b.Qb * sp / ns);
                    w.q1 = b.Q0 + (int)((long long)b.Qb * (sp + 1) / ns);
                    w.split = sp;
                    w.pad = b.Q0 > 0 ? 1 : 0;
                    work.push_back(w);
                }
        }
        ch.d_cfg = dalloc_copy(ccfg.data(), ccfg.size());
        ch.d_blocks = dalloc_copy(g.data(), g.size());
        ch.nblocks = (int)g.size();
        ch.nitems = items;
        ch.d_work = dalloc_copy(work.data(), work.size());
        ch.nwork = (int)work.size();
        rp.buf_elems = std::max(rp.buf_elems, (size_t)out);
        rp.chunks.push_back(ch);
    }
    return rp;
}

void free_recompute_plan(RecomputePlan& rp) {
    for (auto& ch : rp.chunks) {
        cudaFree(ch.d_cfg);
        cudaFree(ch.d_blocks);
        cudaFree(ch.d_work);
    }
    rp.chunks.clear();
}

// Time the product kernel of a recompute plan on its first chunk (whose
// generators are evaluated once beforehand).
double time_first_chunk(msd_problem* pb, RecomputePlan& rp, int R, bool fp64) {
    const size_t elem = fp64 ? 16 : 8;
    void* gbuf = pb->genbuf.get(rp.buf_elems * elem);
    void* xs = pb->xs.get((size_t)pb->Ntot * R * elem);
    void* part = pb->part.get((size_t)rp.nsplit * pb->Ntot * R * elem);
    CK(cudaMemsetAsync(xs, 0, (size_t)pb->Ntot * R * elem, pb->stream));
    const RecomputeChunk& ch = rp.chunks[0];
    launch_generator_blocks(pb->d_cfg, ch.d_blocks, ch.nblocks, ch.nitems, pb->d_centre,
                            fp64 ? (double2*)gbuf : nullptr, fp64 ? nullptr : (float2*)gbuf, pb->d_flags, pb->stream,
                            !fp64);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double t = 1e300;
    for (int rep = 0; rep < 3; ++rep) {
        CK(cudaEventRecord(e0, pb->stream));
        launch_bt_only(rp.ch, fp64, ch.d_cfg, ch.d_work, ch.nwork, pb->Nmax, gbuf, xs, part, pb->Ntot, R, pb->stream);
        CK_LAUNCH();
        CK(cudaEventRecord(e1, pb->stream));
        CK(cudaEventSynchronize(e1));
        check_tc("recompute autotune");
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) t = std::min(t, (double)ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return t;
}

// The recompute plan of (R, precision): a pinned shape, else the faster on
// the first chunk of the cost-model CUDA-core shape and (FP32, R divisible
// by 16) the widest tensor-core shape.
RecomputePlan& get_recompute_plan(msd_problem* pb, int R, bool fp64) {
    const long long key = (long long)R * 4 + (fp64 ? 0 : 1);
    auto it = pb->rplans.find(key);
    if (it != pb->rplans.end()) return it->second;
    auto pin = pb->pinned.find(key);
    if (pin != pb->pinned.end() && !pin->second.SH)
        return pb->rplans.emplace(key, build_recompute_plan(pb, R, fp64, pin->second)).first->second;
    RecomputePlan rp = build_recompute_plan(pb, R, fp64, matvec_default_choice(R, pb->Nmax, fp64));
    int rc = 0;
    for (int c = 64; c >= 16 && !fp64; c /= 2)
        if (tc_supported(R, pb->Nmax, c)) {
            rc = c;
            break;
        }
    if (rc && autotune_enabled() && !rp.chunks.empty()) {
        RecomputePlan rt = build_recompute_plan(pb, R, fp64, MatvecChoice{0, rc, 0, 0, rc});
        const double ta = time_first_chunk(pb, rp, R, fp64);
        const double tb = time_first_chunk(pb, rt, R, fp64);
        if (tb < ta) std::swap(rp, rt);
        free_recompute_plan(rt);
    }
    return pb->rplans.emplace(key, std::move(rp)).first->second;
}

void free_recompute_plans(msd_problem* pb) {
    for (auto& kv : pb->rplans) free_recompute_plan(kv.second);
    pb->rplans.clear();
}

// y = P^-1 A x with the generators recomputed chunk by chunk (no stored array).
void matvec_recompute_dev(msd_problem* pb, int R, bool fp64, const void* x, void* y) {
    RecomputePlan& rp = get_recompute_plan(pb, R, fp64);
    const size_t elem = fp64 ? 16 : 8;
    void* gbuf = pb->genbuf.get(rp.buf_elems * elem);
    if (!fp64 && pb->rc_checked != pb->geom_version) {
        // complex64 range of every generator, once per geometry
        CK(cudaMemsetAsync(pb->d_flags, 0, sizeof(int), pb->stream));
        for (auto& ch : rp.chunks)
            launch_generator_blocks(pb->d_cfg, ch.d_blocks, ch.nblocks, ch.nitems, pb->d_centre, nullptr,
                                    (float2*)gbuf, pb->d_flags, pb->stream, true);
        CK_LAUNCH();
        check_flags(pb, "recomputed generators");
        pb->rc_checked = pb->geom_version;
    }
    void* xs = pb->xs.get((size_t)pb->Ntot * R * elem);
    void* part = pb->part.get((size_t)rp.nsplit * pb->Ntot * R * elem);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (pb->timing) {
        while (pb->events.size() < 256) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            pb->events.push_back(e);
        }
        if (pb->ev_used + 2 > pb->events.size()) flush_timing(pb);
        e0 = pb->events[pb->ev_used++];
        e1 = pb->events[pb->ev_used++];
        pb->timed_flops += 8.0 * (double)R * pb->offdiag_n2;
        pb->timed_bytes += (double)elem * 2.0 * (double)pb->Ntot * R;  // no stored generators
    }
    launch_scale_cols(fp64, pb->Ntot, R, fp64 ? (const void*)pb->d_rf64 : (const void*)pb->d_rf32, x, xs,
                      pb->stream);
    if (e0) CK(cudaEventRecord(e0, pb->stream));
    for (auto& ch : rp.chunks) {
        launch_generator_blocks(pb->d_cfg, ch.d_blocks, ch.nblocks, ch.nitems, pb->d_centre,
                                fp64 ? (double2*)gbuf : nullptr, fp64 ? nullptr : (float2*)gbuf, pb->d_flags,
                                pb->stream, !fp64);
        launch_bt_only(rp.ch, fp64, ch.d_cfg, ch.d_work, ch.nwork, pb->Nmax, gbuf, xs, part, pb->Ntot, R,
                       pb->stream);
    }
    if (e1) CK(cudaEventRecord(e1, pb->stream));
    launch_finalize(fp64, pb->Ntot, R, rp.nsplit, fp64 ? (const void*)pb->d_lf64 : (const void*)pb->d_lf32, x, part,
                    y, pb->stream);
    CK_LAUNCH();
}

// y = P^-1 A x on the problem's stream (device pointers).
// The product of a formulation (msd_set_formulation): one block-Toeplitz
// product over 2R columns (sqrt(a) J x | sqrt(a) J' x) with the stored
// generators, then y = x + l1 z1 + l2 z2.
void matvec_form_dev(msd_problem* pb, int R, bool fp64, const void* x, void* y) {
    if (matvec_smem_bytes(matvec_default_choice(2 * R, pb->Nmax, fp64), pb->Nmax, fp64) > kMatvecSmemCap)
        fail(MSD_ERR_ARG, "truncation order too large for the shared-memory tile of this precision");
    ensure_generators(pb, fp64);
    MatvecPlan& plan = get_plan(pb, 2 * R, fp64);
    const size_t elem = fp64 ? 16 : 8;
    void* xs = pb->xs.get((size_t)pb->Ntot * 2 * R * elem);
    void* part = pb->part.get((size_t)plan.nsplit * pb->Ntot * 2 * R * elem);
    launch_form_scale(fp64, pb->Ntot, R, fp64 ? (const void*)pb->d_rf64 : (const void*)pb->d_rf32,
                      fp64 ? (const void*)pb->d_frf2_64 : (const void*)pb->d_frf2_32, x, xs, pb->stream);
    launch_bt_only(plan.ch, fp64, pb->d_cfg, plan.d_work, (int)plan.work.size(), pb->Nmax,
                   fp64 ? (const void*)pb->d_G64 : (const void*)pb->d_G32, xs, part, pb->Ntot, 2 * R, pb->stream);
    launch_form_finalize(fp64, pb->Ntot, R, plan.nsplit, fp64 ? (const void*)pb->d_fl1_64 : (const void*)pb->d_fl1_32,
                         fp64 ? (const void*)pb->d_fl2_64 : (const void*)pb->d_fl2_32, x, part, y, pb->stream);
    CK_LAUNCH();
}

// The transmission product (penetrable obstacles) of the parent problem pb
// on vectors in the transmission layout: one block-Toeplitz product with
// the generators at k+ (pb) and one at k- (pb->pen_minus), then
// y = x + A [z+; z-].
void pen_matvec(msd_problem* pb, int R, bool fp64, const void* x, void* y) {
    msd_problem* pm = pb->pen_minus;
    if (matvec_smem_bytes(matvec_default_choice(R, pb->Nmax, fp64), pb->Nmax, fp64) > kMatvecSmemCap)
        fail(MSD_ERR_ARG, "truncation order too large for the shared-memory tile of this precision");
    ensure_generators(pb, fp64);
    ensure_generators(pm, fp64);
    MatvecPlan& pp = get_plan(pb, R, fp64);
    MatvecPlan& pq = get_plan(pm, R, fp64);
    const size_t elem = fp64 ? 16 : 8;
    const size_t nv = (size_t)pb->Ntot * R;
    void* xsp = pb->xs.get(nv * elem);
    void* xsm = pm->xs.get(nv * elem);
    void* partp = pb->part.get((size_t)pp.nsplit * nv * elem);
    void* partm = pm->part.get((size_t)pq.nsplit * nv * elem);
    launch_pen_scale(fp64, pb->d_cfg, pb->C, pb->Ntot, R, fp64 ? (const void*)pb->d_rf64 : (const void*)pb->d_rf32,
                     fp64 ? (const void*)pm->d_rf64 : (const void*)pm->d_rf32, x, xsp, xsm, pb->stream);
    launch_bt_only(pp.ch, fp64, pb->d_cfg, pp.d_work, (int)pp.work.size(), pb->Nmax,
                   fp64 ? (const void*)pb->d_G64 : (const void*)pb->d_G32, xsp, partp, pb->Ntot, R, pb->stream);
    launch_bt_only(pq.ch, fp64, pm->d_cfg, pq.d_work, (int)pq.work.size(), pm->Nmax,
                   fp64 ? (const void*)pm->d_G64 : (const void*)pm->d_G32, xsm, partm, pm->Ntot, R, pb->stream);
    launch_pen_finalize(fp64, pb->d_cfg, pb->C, pb->Ntot, R,
                        fp64 ? (const void*)pb->d_penA64 : (const void*)pb->d_penA32, x, partp, pp.nsplit, partm,
                        pq.nsplit, y, pb->stream);
    CK_LAUNCH();
}

void matvec_dev(msd_problem* pb, int R, bool fp64, const void* x, void* y) {
    if (pb->pen_parent) {
        pen_matvec(pb->pen_parent, R, fp64, x, y);
        return;
    }
    if (pb->form) {
        matvec_form_dev(pb, R, fp64, x, y);
        return;
    }
    if (matvec_smem_bytes(matvec_default_choice(R, pb->Nmax, fp64), pb->Nmax, fp64) > kMatvecSmemCap)
        fail(MSD_ERR_ARG, "truncation order too large for the shared-memory tile of this precision");
    if (pb->gen_mode == MSD_GEN_RECOMPUTE) {
        matvec_recompute_dev(pb, R, fp64, x, y);
        return;
    }
    ensure_generators(pb, fp64);
    MatvecPlan& plan = get_plan(pb, R, fp64, true);
    if (plan.ch.SH && !ensure_gt(pb)) fail(MSD_ERR_OOM, "shift-GEMM generators do not fit in device memory");
    const size_t elem = fp64 ? 16 : 8;
    void* xs = plan.ch.SH ? nullptr : pb->xs.get((size_t)pb->Ntot * R * elem);
    const bool xs_ready = !fp64 && !plan.ch.SH && x == pb->xs_src;
    pb->xs_src = nullptr;
    void* part = pb->part.get((size_t)plan.nsplit * pb->Ntot * R * elem);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (pb->timing) {
        // events bracket the block-Toeplitz kernel alone (not the scaling or
        // the split reduction around it)
        while (pb->events.size() < 256) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            pb->events.push_back(e);
        }
        if (pb->ev_used + 2 > pb->events.size()) flush_timing(pb);  // waits, then reuses the pool
        e0 = pb->events[pb->ev_used++];
        e1 = pb->events[pb->ev_used++];
        const double sc = fp64 ? 16.0 : 8.0;
        pb->timed_flops += 8.0 * (double)R * pb->offdiag_n2;
        pb->timed_bytes += sc * ((double)pb->offdiag_L + 2.0 * (double)pb->Ntot * R);
    }
    if (plan.ch.SH) {
        // shift-GEMM tensor-core product: columns scaled and split into the
        // slab order, the kernel, then y = x + l .* (sum of the splits)
        float* XT = (float*)pb->xt.get((size_t)pb->xrows * 4 * R * sizeof(float));
        launch_tcs_prep_x(pb->d_cfg, pb->C, pb->xrows / 4, R, pb->d_rf32, (const float2*)x, XT, pb->stream);
        if (e0) CK(cudaEventRecord(e0, pb->stream));
        launch_bt_tcs(pb->d_cfg, plan.d_work, (int)plan.work.size(), pb->Nmax, pb->d_GT, XT, (float2*)part, pb->Ntot,
                      R, pb->stream, pb->live);
        if (e1) CK(cudaEventRecord(e1, pb->stream));
        launch_finalize(false, pb->Ntot, R, plan.nsplit, pb->d_lf32, x, part, y, pb->stream);
    } else if (fp64)
        launch_matvec_f64(pb->d_cfg, plan.d_work, (int)plan.work.size(), pb->Nmax, pb->d_G64, pb->d_rf64,
                          pb->d_lf64, pb->Ntot, R, (const double2*)x, (double2*)xs, (double2*)part,
                          plan.nsplit, (double2*)y, pb->stream, e0, e1, &plan.ch, pb->live);
    else
        launch_matvec_f32(pb->d_cfg, plan.d_work, (int)plan.work.size(), pb->Nmax, pb->d_G32, pb->d_rf32,
                          pb->d_lf32, pb->Ntot, R, (const float2*)x, (float2*)xs, (float2*)part,
                          plan.nsplit, (float2*)y, pb->stream, e0, e1, &plan.ch, pb->live, xs_ready);
    CK_LAUNCH();
}

// Adjoint generators GA[p][q][l] = conj(g^pq_{-l}) and conj(l) of the current
// geometry (rebuilt after msd_update_geometry).
void ensure_adjoint(msd_problem* pb, bool fp64) {
    ensure_generators(pb, fp64);
    if (!pb->d_clf64 || pb->adj_rows_version != pb->geom_version) {
        if (!pb->d_clf64) {
            pb->d_clf64 = dalloc<double2>(pb->Ntot);
            pb->d_clf32 = dalloc<float2>(pb->Ntot);
        }
        launch_conj_rows(pb->Ntot, pb->d_lf64, pb->d_clf64, pb->d_clf32, pb->stream);
        CK_LAUNCH();
        pb->adj_rows_version = pb->geom_version;
    }
    if (fp64) {
        if (!pb->d_GA64 || pb->adj64_version != pb->geom_version) {
            if (!pb->d_GA64) pb->d_GA64 = dalloc<double2>(pb->gen_elems);
            launch_adjoint_generators_f64(pb->d_cfg, pb->C, pb->cfg.data(), pb->d_G64, pb->d_GA64, pb->stream);
            CK_LAUNCH();
            pb->adj64_version = pb->geom_version;
        }
    } else {
        if (!pb->d_GA32 || pb->adj32_version != pb->geom_version) {
            if (!pb->d_GA32) pb->d_GA32 = dalloc<float2>(pb->gen_elems);
            launch_adjoint_generators_f32(pb->d_cfg, pb->C, pb->cfg.data(), pb->d_G32, pb->d_GA32, pb->stream);
            CK_LAUNCH();
            pb->adj32_version = pb->geom_version;
        }
    }
}

// Products with other scalings on the problem's stream (device pointers):
//   adjoint: y = x + r .* T^H(conj(l) .* x)       ((P^-1 A)^H x)
//   raw forward: y = T(r .* x)    raw adjoint: y = T^H(conj(l) .* x)
void product_dev(msd_problem* pb, int R, bool fp64, bool adjoint, bool raw, const void* x, void* y) {
    if (pb->form) fail(MSD_ERR_ARG, "adjoint and raw products need the default formulation");
    if (matvec_smem_bytes(matvec_default_choice(R, pb->Nmax, fp64), pb->Nmax, fp64) > kMatvecSmemCap)
        fail(MSD_ERR_ARG, "truncation order too large for the shared-memory tile of this precision");
    if (adjoint) ensure_adjoint(pb, fp64);
    else ensure_generators(pb, fp64);
    MatvecPlan& plan = get_plan(pb, R, fp64);
    const size_t elem = fp64 ? 16 : 8;
    void* xs = pb->xs.get((size_t)pb->Ntot * R * elem);
    void* part = pb->part.get((size_t)plan.nsplit * pb->Ntot * R * elem);
    const int nwork = (int)plan.work.size();
    if (fp64) {
        const double2* G = adjoint ? pb->d_GA64 : pb->d_G64;
        launch_product_f64(pb->d_cfg, plan.d_work, nwork, pb->Nmax, G, adjoint ? nullptr : pb->d_rf64,
                           adjoint ? pb->d_clf64 : nullptr, (adjoint && !raw) ? pb->d_rf64 : nullptr,
                           (!adjoint && !raw) ? pb->d_lf64 : nullptr, raw ? 0 : 1, pb->Ntot, R,
                           (const double2*)x, (double2*)xs, (double2*)part, plan.nsplit, (double2*)y, pb->stream,
                           &plan.ch);
    } else {
        const float2* G = adjoint ? pb->d_GA32 : pb->d_G32;
        launch_product_f32(pb->d_cfg, plan.d_work, nwork, pb->Nmax, G, adjoint ? nullptr : pb->d_rf32,
                           adjoint ? pb->d_clf32 : nullptr, (adjoint && !raw) ? pb->d_rf32 : nullptr,
                           (!adjoint && !raw) ? pb->d_lf32 : nullptr, raw ? 0 : 1, pb->Ntot, R,
                           (const float2*)x, (float2*)xs, (float2*)part, plan.nsplit, (float2*)y, pb->stream,
                           &plan.ch);
    }
    CK_LAUNCH();
}

// The operator of a solve: P^-1 A, or its adjoint.
void operator_dev(msd_problem* pb, int R, bool fp64, bool adjoint, const void* x, void* y) {
    if (adjoint) product_dev(pb, R, fp64, true, false, x, y);
    else matvec_dev(pb, R, fp64, x, y);
}

// Stage a caller buffer that may live on the host: returns a device pointer
// (the caller's if it is device memory, else a library buffer filled from it).
const void* stage_in(msd_problem* pb, DBuf& buf, const void* p, size_t bytes) {
    if (is_device_ptr(p)) return p;
    void* d = buf.get(bytes);
    CK(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, pb->stream));
    return d;
}

struct OutStage {
    msd_problem* pb;
    void* user;
    void* dev;
    size_t bytes;
    bool host;
    OutStage(msd_problem* pb_, DBuf& buf, void* p, size_t n) : pb(pb_), user(p), bytes(n) {
        host = !is_device_ptr(p);
        dev = host ? buf.get(n) : p;
    }
    void finish() {
        if (host) {
            CK(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, pb->stream));
            CK(cudaStreamSynchronize(pb->stream));
        }
    }
};

}  // namespace

// ---------------------------------------------------------------- GMRES driver

namespace {

struct SolveCtx {
    msd_problem* pb;
    GmresDims d;
    int m;
    // FP64 vectors [Ntot][R]
    double2 *b, *x, *r, *Ax;
    // per-system arrays ([S][hstride] for projections and norms)
    double2 *h1, *h2, *wn2, *wn2b, *H, *cs, *sn, *g, *y, *lsq_work, *rdiag;
    double *beta, *vscale, *tol_abs, *tol_cycle;
    int *active, *kconv, *iters, *skip2, *flags;  // flags[0] any_active, flags[1] nonfinite
    int* cnt = nullptr;  // ncnt + 1 counters of the fused projection reductions (zero between launches)
    int ncnt = 0;
    double eta2 = 0.5;  // second Gram-Schmidt pass when ||w'||^2 < eta2 ||w||^2
    int hstride;
    double2* part;  // [nchunk][m + 2][R] reduction partials
    bool adjoint = false;  // solve with (P^-1 A)^H
};

// ||u||^2 per system into out[s * hstride] (FP64 vectors)
void norm2_f64(SolveCtx& cx, const double2* u, double2* out) {
    gm_dots<double2>(cx.d, cx.pb->d_chunks, cx.pb->d_cfg_chunk_off, nullptr, 0, 0, 1, u, nullptr, cx.part, out,
                     cx.hstride, cx.pb->stream);
}

// Counters of the fused projection reductions: one per group of eight
// basis vectors (bases of up to 4000 vectors plus w), and one more.
constexpr int kDotsCounters = 512;

// Basis size from which projections run over the coarse row chunks.
constexpr int kCoarseFrom = 64;

// Hands the active flags of the Krylov systems to the products of one
// Arnoldi step, and takes them back however the step ends.
struct LiveScope {
    msd_problem* pb;
    LiveScope(msd_problem* p, const int* active) : pb(p) { pb->live = active; }
    ~LiveScope() { pb->live = nullptr; }
};

// One restart cycle of GMRES on P^-1 A d = r (x += d), basis type V.
template <typename V>
void arnoldi_cycle(SolveCtx& cx, V* Vb, V* w, bool fp64, int maxit_left, int* steps_taken) {
    msd_problem* pb = cx.pb;
    // scaled columns prepared by a step are for that step's successor only
    struct XsReset {
        msd_problem* pb;
        ~XsReset() { pb->xs_src = nullptr; }
    } xs_reset{pb};
    pb->xs_src = nullptr;
    cudaStream_t s = pb->stream;
    const GmresDims& d = cx.d;
    const long long vstride = pb->Ntot * d.R;
    const RowChunk* ch = pb->d_chunks;
    const int* co = pb->d_cfg_chunk_off;
    norm2_f64(cx, cx.r, cx.wn2);
    CK(cudaMemsetAsync(cx.flags, 0, 2 * sizeof(int), s));
    gm_start(d, cx.wn2, cx.hstride, cx.tol_abs, cx.beta, cx.vscale, cx.g, cx.active, cx.kconv, cx.flags, s);
    gm_scale<double2, V>(d, ch, cx.r, cx.vscale, cx.active, Vb, s);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(pb->h_pinned, cx.flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int any = pb->h_pinned[0];
    // The host reads the convergence flags of step j - kLag while step j is
    // queued, so the GPU never waits for the host; the (at most kLag) steps
    // queued after the last system converged run on zero vectors and change
    // nothing.
    constexpr int kLag = 2, kRing = 4;
    int j = 0;
    for (; any && j < cx.m && j < maxit_left; ++j) {
        if (j >= kLag) {
            const int slot = (j - kLag) % kRing;
            CK(cudaEventSynchronize(pb->ring_ev[slot]));
            if (pb->h_pinned[2 + 2 * slot + 1]) {
                check_tc("GMRES");
                fail(MSD_ERR_NONFINITE, "GMRES: non-finite Arnoldi coefficient");
            }
            if (!pb->h_pinned[2 + 2 * slot]) break;
        }
        V* vj = Vb + (long long)j * vstride;
        {
            // the product may skip configurations with no active column
            LiveScope live(pb, cx.active);
            operator_dev(pb, d.R, fp64, cx.adjoint, vj, w);
        }
        // projections onto many basis vectors: the coarse row chunks when the
        // block-reduction kernel serves this column count, the medium ones for
        // the warp-per-vector kernels (no block reduction; longer-lived warps)
        const bool many = j + 1 >= kCoarseFrom;
        const bool warpk = 32 % d.R == 0 || d.R == 64;
        GmresDims db = d;
        const RowChunk* chb = ch;
        const int* cob = co;
        if (many && !warpk) {
            db.nchunk = (int)pb->chunks_coarse.size();
            chb = pb->d_chunks_coarse;
            cob = pb->d_cfg_chunk_off_coarse;
        } else if (many) {
            db.nchunk = (int)pb->chunks_mid.size();
            chb = pb->d_chunks_mid;
            cob = pb->d_cfg_chunk_off_mid;
        }
        // first projection h1 = V^H w (with ||w||^2 at h1[j+1]), w -= V h1;
        // systems that have converged (zero vectors from here on) are skipped
        // (few systems: the reductions, and the flags of the second
        // projection, run inside the projection kernels)
        GmDotsFuse fz1, fz2;
        fz1.cnt = fz2.cnt = cx.cnt;
        fz1.ncnt = fz2.ncnt = cx.ncnt;
        fz1.j = fz2.j = j;
        fz1.wn2 = cx.wn2;
        fz1.active = cx.active;
        fz1.skip2 = cx.skip2;
        fz1.eta2 = cx.eta2;
        const bool flags_done =
            gm_dots<V>(db, chb, cob, Vb, vstride, j + 1, 1, w, cx.active, cx.part, cx.h1, cx.hstride, s, 0, &fz1);
        gm_update<V, V>(d, ch, Vb, vstride, j + 1, cx.h1, cx.hstride, cx.active, -1.0, w, s, 0);
        // second projection only where the first removed more than half of ||w||^2
        if (!flags_done) gm_reorth_flags(d, cx.h1, cx.hstride, j, cx.wn2, cx.active, cx.skip2, s, cx.eta2);
        // its norm: ||w1 - V h2||^2 = ||w1||^2 - |h2|^2 (w1 measured by the
        // projection itself; h2 is small after the first pass, so no
        // cancellation), formed inside the fused kernel, else measured
        fz2.wn2 = cx.wn2b;
        const bool norm_done =
            gm_dots<V>(db, chb, cob, Vb, vstride, j + 1, 1, w, cx.skip2, cx.part, cx.h2, cx.hstride, s, 1, &fz2);
        gm_update<V, V>(d, ch, Vb, vstride, j + 1, cx.h2, cx.hstride, cx.skip2, -1.0, w, s);
        if (!norm_done) gm_dots<V>(d, ch, co, nullptr, 0, 0, 1, w, cx.skip2, cx.part, cx.wn2b, cx.hstride, s);
        // the Givens step stores its flags (any system still active, a
        // non-finite coefficient) straight into pinned host memory, in the
        // ring slot of this step; the host cleared the slot, whose previous
        // step (j - kRing) it has already read
        const int slot = j % kRing;
        volatile int* hf = pb->h_pinned + 2 + 2 * slot;
        hf[0] = 0;
        hf[1] = 0;
        int* df = pb->d_hpinned + 2 + 2 * slot;
        gm_givens(d, j, cx.h1, cx.h2, cx.hstride, cx.wn2, cx.wn2b, cx.skip2, cx.tol_cycle, cx.H, cx.cs, cx.sn,
                  cx.g, cx.vscale, cx.active, cx.kconv, cx.iters, df, df + 1, cx.rdiag,
                  sizeof(V) == sizeof(float2), s);
        // the next basis vector; for the FP32 product of the default rows,
        // also its scaled columns rf .* v, which that product then reads
        V* vnext = Vb + (long long)(j + 1) * vstride;
        float2* xs_next = nullptr;
        if (sizeof(V) == sizeof(float2) && !cx.adjoint && !pb->form && !pb->pen_parent &&
            pb->gen_mode != MSD_GEN_RECOMPUTE && !get_plan(pb, d.R, false, true).ch.SH) {
            xs_next = (float2*)pb->xs.get((size_t)pb->Ntot * d.R * sizeof(float2));
            pb->xs_src = vnext;
        }
        gm_scale<V, V>(d, ch, w, cx.vscale, cx.active, vnext, s, xs_next ? pb->d_rf32 : nullptr, xs_next);
        CK_LAUNCH();
        CK(cudaEventRecord(pb->ring_ev[slot], s));
    }
    // settle: the last queued steps decide whether any system is still active
    CK(cudaStreamSynchronize(s));
    if (j > 0) {
        const int slot = (j - 1) % kRing;
        if (pb->h_pinned[2 + 2 * slot + 1]) {
            check_tc("GMRES");
            fail(MSD_ERR_NONFINITE, "GMRES: non-finite Arnoldi coefficient");
        }
        any = pb->h_pinned[2 + 2 * slot];
    }
    if (any) {
        // budget exhausted mid-cycle: close the still-active systems at j columns
        std::vector<int> act(d.S), kc(d.S);
        CK(cudaMemcpyAsync(act.data(), cx.active, d.S * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(kc.data(), cx.kconv, d.S * sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int i = 0; i < d.S; ++i)
            if (act[i]) kc[i] = j;
        CK(cudaMemcpyAsync(cx.kconv, kc.data(), d.S * sizeof(int), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    *steps_taken = j;
    gm_lsq(d, cx.H, cx.cs, cx.sn, cx.rdiag, cx.g, cx.kconv, cx.y, cx.lsq_work, s);
    // x += V y, each system over its own kconv columns (y is zero beyond it)
    gm_update<V, double2>(d, ch, Vb, vstride, j, cx.y, cx.m, nullptr, 1.0, cx.x, s);
    CK_LAUNCH();
}

// Solve (P^-1 A) x = b, or its adjoint, for R columns per configuration.
// The right-hand side is the plane-wave one of betas_host, or b_dev (FP64,
// preconditioned, device) when given.
msd_status solve_impl(msd_problem* pb, int R, const double* betas_host, const msd_opts* opts_in,
                      void* rho_out, msd_stats* stats_host, const double2* b_dev = nullptr, bool adjoint = false) {
    if (!pb || R <= 0 || (!betas_host && !b_dev) || !rho_out) fail(MSD_ERR_ARG, "msd_solve_planewaves: bad argument");
    const auto t_start = std::chrono::steady_clock::now();
    msd_opts o;
    memset(&o, 0, sizeof(o));
    if (opts_in) o = *opts_in;
    if (o.gen_mode != MSD_GEN_AUTO && o.gen_mode != MSD_GEN_STREAMED && o.gen_mode != MSD_GEN_RECOMPUTE)
        fail(MSD_ERR_ARG, "msd_solve_planewaves: gen_mode");
    // a solve-level generator mode applies to this solve's forward products only
    struct ModeGuard {
        msd_problem* pb;
        int old;
        ~ModeGuard() { pb->gen_mode = old; }
    } mode_guard{pb, pb->gen_mode};
    if (o.gen_mode != MSD_GEN_AUTO && !adjoint) pb->gen_mode = o.gen_mode;
    if (o.tol <= 0) o.tol = 1e-10;
    if (o.maxit <= 0) o.maxit = 3000;
    if (o.restart <= 0) {
        // Automatic restart length: GMRES converges fastest unrestarted, and
        // HBM is large, so take the longest Krylov basis that fits in half of
        // the free device memory and keeps the per-system Hessenberg
        // matrices within 8 % of it (at least 2 GB), capped by maxit and by 4000.
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        const double vec = (double)pb->Ntot * R * ((o.precision == MSD_MIXED) ? 8 : 16);
        const double S_ = (double)pb->C * R;
        const long long m_mem = (long long)(0.5 * (double)free_b / vec) - 2;
        const long long m_hess = (long long)std::sqrt(std::max(2e9, 0.08 * (double)free_b) / (16.0 * S_));
        long long m = std::min<long long>({m_mem, m_hess, (long long)o.maxit, 4000LL});
        o.restart = (int)std::max<long long>(m, 10);
    }
    if (o.max_refine <= 0) o.max_refine = 60;
    if (o.inner_tol <= 0) o.inner_tol = 5e-6;
    if (o.reorth == 0) o.reorth = 0.5;
    if (!(o.reorth > 0 && o.reorth <= 1)) fail(MSD_ERR_ARG, "msd_solve_planewaves: reorth outside (0, 1]");
    if (o.precision != MSD_FP64 && o.precision != MSD_MIXED) fail(MSD_ERR_ARG, "msd_solve_planewaves: precision");
    const bool mixed = o.precision == MSD_MIXED;
    cudaStream_t s = pb->stream;

    SolveCtx cx;
    cx.pb = pb;
    cx.m = o.restart;
    cx.eta2 = o.reorth;
    cx.d.Ntot = pb->Ntot;
    cx.d.R = R;
    cx.d.C = pb->C;
    cx.d.S = pb->C * R;
    cx.d.m = o.restart;
    cx.d.nchunk = (int)pb->chunks.size();
    cx.hstride = o.restart + 2;
    const int S = cx.d.S, m = o.restart;
    const size_t nv = (size_t)pb->Ntot * R;

    int bi = 1;
    auto sb = [&](size_t bytes) { return pb->sbuf[bi++].get(bytes); };
    cx.b = (double2*)sb(nv * 16);
    cx.x = (double2*)sb(nv * 16);
    cx.r = (double2*)sb(nv * 16);
    cx.Ax = (double2*)sb(nv * 16);
    cx.h1 = (double2*)sb((size_t)S * cx.hstride * 16);
    cx.h2 = (double2*)sb((size_t)S * cx.hstride * 16);
    cx.wn2 = (double2*)sb((size_t)S * cx.hstride * 16);
    cx.wn2b = (double2*)sb((size_t)S * cx.hstride * 16);
    cx.lsq_work = (double2*)sb((size_t)S * (m + 1) * 16);
    cx.H = (double2*)sb((size_t)S * m * (m + 1) * 16);
    cx.cs = (double2*)sb((size_t)S * m * 16);
    cx.sn = (double2*)sb((size_t)S * m * 16);
    cx.g = (double2*)sb((size_t)S * (m + 1) * 16);
    cx.y = (double2*)sb((size_t)S * m * 2 * 16);
    cx.rdiag = cx.y + (size_t)S * m;
    double* dsys = (double*)sb((size_t)S * 4 * 8);
    cx.beta = dsys;
    cx.vscale = dsys + S;
    cx.tol_abs = dsys + 2 * S;
    cx.tol_cycle = dsys + 3 * S;
    int* isys = (int*)sb((size_t)(S * 4 + 2 + kDotsCounters + 1) * 4);
    cx.active = isys;
    cx.kconv = isys + S;
    cx.iters = isys + 2 * S;
    cx.skip2 = isys + 3 * S;
    cx.flags = isys + 4 * S;
    cx.cnt = isys + 4 * S + 2;
    cx.ncnt = kDotsCounters;
    CK(cudaMemsetAsync(cx.cnt, 0, (size_t)(cx.ncnt + 1) * sizeof(int), s));
    const size_t velem = mixed ? 8 : 16;
    void* Vb = sb((size_t)(m + 1) * nv * velem);
    void* w = sb(nv * velem);
    double* d_betas = (double*)sb((size_t)pb->C * R * 8);
    cx.part = (double2*)pb->sbuf[0].get((size_t)cx.d.nchunk * (m + 2) * R * sizeof(double2));

    cx.adjoint = adjoint;
    if (b_dev) {
        CK(cudaMemcpyAsync(cx.b, b_dev, nv * 16, cudaMemcpyDeviceToDevice, s));
    } else {
        CK(cudaMemcpyAsync(d_betas, betas_host, (size_t)pb->C * R * 8, cudaMemcpyHostToDevice, s));
        launch_rhs_planewave(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_centre, pb->d_radius, rhs_scale_of(pb),
                             pb->Nmax, R, d_betas, cx.b, s);
        CK_LAUNCH();
    }
    if (adjoint) {
        if (pb->form) fail(MSD_ERR_ARG, "adjoint solves need the default formulation");
        ensure_adjoint(pb, true);
        if (mixed) ensure_adjoint(pb, false);
    } else if ((pb->gen_mode != MSD_GEN_RECOMPUTE || pb->form) && !pb->pen_parent) {
        ensure_generators(pb, true);
        if (mixed) ensure_generators(pb, false);
    }
    gm_zero(nv, cx.x, s);
    CK(cudaMemsetAsync(cx.iters, 0, S * sizeof(int), s));
    // ||b|| per system
    norm2_f64(cx, cx.b, cx.wn2);
    std::vector<double2> hb((size_t)S * cx.hstride);
    CK(cudaMemcpyAsync(hb.data(), cx.wn2, hb.size() * 16, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<double> bnorm(S), tol_abs(S), relres(S, 1.0), prev(S, 1e300), tol_cycle(S);
    for (int i = 0; i < S; ++i) {
        bnorm[i] = std::sqrt(std::max(hb[(size_t)i * cx.hstride].x, 0.0));
        tol_abs[i] = o.tol * bnorm[i];
        if (!std::isfinite(bnorm[i])) fail(MSD_ERR_NONFINITE, "right-hand side is not finite");
    }
    CK(cudaMemcpyAsync(cx.tol_abs, tol_abs.data(), S * 8, cudaMemcpyHostToDevice, s));

    int total = 0, sweeps = 0;
    bool stagnated = false;
    const int max_sweeps = mixed ? o.max_refine : 1 << 30;
    while (true) {
        // FP64 residual of the current iterate
        if (sweeps == 0) {
            CK(cudaMemcpyAsync(cx.r, cx.b, nv * 16, cudaMemcpyDeviceToDevice, s));
        } else {
            operator_dev(pb, R, true, cx.adjoint, cx.x, cx.Ax);
            gm_residual(nv, cx.b, cx.Ax, cx.r, s);
        }
        norm2_f64(cx, cx.r, cx.wn2);
        CK(cudaMemcpyAsync(hb.data(), cx.wn2, hb.size() * 16, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        bool all = true, improved = false;
        for (int i = 0; i < S; ++i) {
            const double rn = std::sqrt(std::max(hb[(size_t)i * cx.hstride].x, 0.0));
            if (!std::isfinite(rn)) {
                check_tc("GMRES");
                fail(MSD_ERR_NONFINITE, "GMRES: non-finite residual");
            }
            relres[i] = bnorm[i] > 0 ? rn / bnorm[i] : 0.0;
            if (relres[i] > o.tol) {
                all = false;
                // a sweep that leaves the FP64 residual of every unconverged
                // system where it was has stagnated (FP32 sweeps can stall
                // on the rounding of the inner product)
                if (relres[i] < (1.0 - 1e-3) * prev[i]) improved = true;
            }
            // An FP32 sweep stops at inner_tol times its starting residual,
            // and not below the stopping tolerance: deeper, its estimate runs
            // ahead of the true residual, which FP32 rounding holds back.  A
            // sweep that starts within 2x of the tolerance aims at half of
            // it, so that the rounding of its correction cannot leave the
            // system just above the tolerance.
            const double floor_abs = (rn <= 2.0 * tol_abs[i] ? 0.5 : 1.0) * tol_abs[i];
            tol_cycle[i] = mixed ? std::max(floor_abs, o.inner_tol * rn) : tol_abs[i];
        }
        if (all) break;
        if (mixed && sweeps > 0 && !improved) {
            stagnated = true;
            break;
        }
        if (sweeps >= max_sweeps || total >= o.maxit) break;
        prev = relres;
        CK(cudaMemcpyAsync(cx.tol_cycle, tol_cycle.data(), S * 8, cudaMemcpyHostToDevice, s));
        int steps = 0;
        if (mixed)
            arnoldi_cycle<float2>(cx, (float2*)Vb, (float2*)w, false, o.maxit - total, &steps);
        else
            arnoldi_cycle<double2>(cx, (double2*)Vb, (double2*)w, true, o.maxit - total, &steps);
        total += steps;
        ++sweeps;
        if (steps == 0) break;
    }

    // densities out
    {
        const size_t bytes = nv * 16;
        if (is_device_ptr(rho_out)) {
            CK(cudaMemcpyAsync(rho_out, cx.x, bytes, cudaMemcpyDeviceToDevice, s));
        } else {
            CK(cudaMemcpyAsync(rho_out, cx.x, bytes, cudaMemcpyDeviceToHost, s));
        }
    }
    std::vector<int> it(S);
    CK(cudaMemcpyAsync(it.data(), cx.iters, S * 4, cudaMemcpyDeviceToHost, s));
    // unpreconditioned relative residual ||P r'|| / ||P b'|| from the final
    // FP64 residual r' of the preconditioned system
    std::vector<double> true_relres(S, -1.0);
    if (!adjoint && R <= 64 && !pb->pen_parent) {
        const int nch = (int)pb->chunks.size();
        launch_weighted_norms(pb->d_cfg, pb->d_chunks, nch, R, pb->d_radius, pb->d_bc, pb->d_J, pb->d_H, pb->d_dH,
                              pb->form ? pb->d_fdiag : nullptr,
                              cx.r, cx.b, cx.part, s);
        CK_LAUNCH();
        std::vector<double2> wp((size_t)nch * R);
        CK(cudaMemcpyAsync(wp.data(), cx.part, wp.size() * 16, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::vector<double> nu(S, 0.0), nv2(S, 0.0);
        for (int k = 0; k < nch; ++k)
            for (int r = 0; r < R; ++r) {
                nu[pb->chunks[k].cfg * R + r] += wp[(size_t)k * R + r].x;
                nv2[pb->chunks[k].cfg * R + r] += wp[(size_t)k * R + r].y;
            }
        for (int i = 0; i < S; ++i) true_relres[i] = nv2[i] > 0 ? std::sqrt(nu[i] / nv2[i]) : 0.0;
    }
    CK(cudaStreamSynchronize(s));
    check_tc("msd_solve_planewaves");
    const double solve_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    msd_status st = MSD_OK;
    for (int i = 0; i < S; ++i) {
        int flag = relres[i] <= o.tol ? MSD_OK : (stagnated ? MSD_STAGNATED : MSD_NOT_CONVERGED);
        if (flag != MSD_OK && st == MSD_OK) st = (msd_status)flag;
        if (stats_host) {
            stats_host[i].flag = flag;
            stats_host[i].iters = it[i];
            stats_host[i].refine_steps = sweeps > 0 ? sweeps - 1 : 0;
            stats_host[i].reserved = 0;
            stats_host[i].relres = relres[i];
            stats_host[i].true_relres = true_relres[i];
            stats_host[i].solve_ms = solve_ms;
        }
    }
    return st;
}

}  // namespace

// ---------------------------------------------------------------- C ABI

extern "C" {

const char* msd_last_error(void) { return g_err.c_str(); }

msd_status msd_create(int C, const int* disk_off, const double* centres, const double* radii,
                      const int8_t* bc, const double* k, const int* N, void* cuda_stream, msd_problem** out) {
    return guarded([&]() -> msd_status {
        if (!out) fail(MSD_ERR_ARG, "msd_create: out is NULL");
        *out = nullptr;
        if (C < 1 || !disk_off || !centres || !radii || !bc || !k || !N)
            fail(MSD_ERR_ARG, "msd_create: bad argument");
        if (disk_off[0] != 0) fail(MSD_ERR_ARG, "msd_create: disk_off[0] must be 0");
        for (int c = 0; c < C; ++c) {
            if (disk_off[c + 1] <= disk_off[c]) fail(MSD_ERR_ARG, "msd_create: every configuration needs a disk");
            if (!(k[c] > 0) || !std::isfinite(k[c])) fail(MSD_ERR_ARG, "msd_create: k must be positive");
            if (N[c] < 1 || N[c] > MSD_MAX_N) fail(MSD_ERR_ARG, "msd_create: N out of range");
        }
        const int Mtot = disk_off[C];
        for (int d = 0; d < Mtot; ++d) {
            if (!(radii[d] > 0) || !std::isfinite(radii[d]) || !std::isfinite(centres[2 * d]) ||
                !std::isfinite(centres[2 * d + 1]))
                fail(MSD_ERR_ARG, "msd_create: radii must be positive and centres finite");
            if (bc[d] != MSD_DIRICHLET && bc[d] != MSD_NEUMANN) fail(MSD_ERR_ARG, "msd_create: bc flag");
        }
        // overlap test (disjoint closed disks), per configuration: sort by x, sweep
        for (int c = 0; c < C; ++c) {
            const int a0 = disk_off[c], a1 = disk_off[c + 1];
            std::vector<int> idx(a1 - a0);
            double rmax = 0;
            for (int i = a0; i < a1; ++i) {
                idx[i - a0] = i;
                rmax = std::max(rmax, radii[i]);
            }
            std::sort(idx.begin(), idx.end(), [&](int u, int v) { return centres[2 * u] < centres[2 * v]; });
            for (size_t i = 0; i < idx.size(); ++i)
                for (size_t j = i + 1; j < idx.size(); ++j) {
                    const int u = idx[i], v = idx[j];
                    const double dx = centres[2 * v] - centres[2 * u];
                    if (dx > 2 * rmax) break;
                    const double dy = centres[2 * v + 1] - centres[2 * u + 1];
                    if (std::hypot(dx, dy) <= radii[u] + radii[v])
                        fail(MSD_ERR_OVERLAP, "msd_create: disks " + std::to_string(u) + " and " +
                                                  std::to_string(v) + " intersect");
                }
        }
        msd_problem* pb = new msd_problem();
        try {
            pb->stream = (cudaStream_t)cuda_stream;
            pb->C = C;
            pb->Mtot = Mtot;
            long long row = 0, gen = 0;
            std::vector<int> disk_cfg(Mtot);
            std::vector<long long> gt_blk;
            for (int c = 0; c < C; ++c) {
                MsdConfig m;
                memset(&m, 0, sizeof(m));
                m.k = k[c];
                m.N = N[c];
                m.n = 2 * N[c] + 1;
                m.L = 4 * N[c] + 1;
                m.M = disk_off[c + 1] - disk_off[c];
                m.Mp = (m.M + MSD_TILE_P - 1) / MSD_TILE_P * MSD_TILE_P;
                m.disk_off = disk_off[c];
                m.row_off = row;
                m.gen_off = gen;
                m.Mq = (m.M + 7) / 8 * 8;
                m.gt_off = pb->gt_floats;
                m.xrow_off = pb->xrows;
                const long long ptiles = (m.M + 127) / 128;
                pb->gt_floats += ptiles * m.L * (long long)m.Mq * 512;
                gt_blk.push_back(pb->gt_blocks);
                pb->gt_blocks += ptiles * (m.Mq / 4);
                pb->xrows += (long long)m.Mq * m.n;
                row += (long long)m.M * m.n;
                gen += (long long)m.M * m.Mp * m.L;
                pb->offdiag_L += (double)m.M * (m.M - 1) * m.L;
                pb->offdiag_n2 += (double)m.M * (m.M - 1) * (double)m.n * m.n;
                pb->cfg.push_back(m);
                pb->Nmax = std::max(pb->Nmax, m.N);
                pb->Mmax = std::max(pb->Mmax, m.M);
                for (int d = disk_off[c]; d < disk_off[c + 1]; ++d) disk_cfg[d] = c;
            }
            pb->Ntot = row;
            pb->gen_elems = gen;
            std::vector<double2> cen(Mtot);
            for (int d = 0; d < Mtot; ++d) cen[d] = make_double2(centres[2 * d], centres[2 * d + 1]);
            pb->d_cfg = dalloc_copy(pb->cfg.data(), C);
            pb->d_gt_blk = dalloc_copy(gt_blk.data(), C);
            pb->d_centre = dalloc_copy(cen.data(), Mtot);
            pb->d_radius = dalloc_copy(radii, Mtot);
            pb->d_bc = dalloc_copy(bc, Mtot);
            pb->d_disk_cfg = dalloc_copy(disk_cfg.data(), Mtot);
            pb->d_J = dalloc<double2>(row);
            pb->d_dJ = dalloc<double2>(row);
            pb->d_H = dalloc<double2>(row);
            pb->d_dH = dalloc<double2>(row);
            pb->d_lf64 = dalloc<double2>(row);
            pb->d_rhs_scale = dalloc<double2>(row);
            pb->d_rf64 = dalloc<double>(row);
            pb->d_lf32 = dalloc<float2>(row);
            pb->d_rf32 = dalloc<float>(row);
            pb->d_flags = dalloc<int>(4);
            CK(cudaMemsetAsync(pb->d_flags, 0, 4 * sizeof(int), pb->stream));
            CK(cudaMallocHost((void**)&pb->h_pinned, 64));
            CK(cudaHostGetDevicePointer((void**)&pb->d_hpinned, pb->h_pinned, 0));
            for (auto& e : pb->ring_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            // reduction chunks: at least 512 rows each (two or more rows per
            // thread of a reduction block) and about 256 overall, never
            // across configurations
            auto make_chunks = [&](long long target_rows, std::vector<RowChunk>& out, RowChunk** d_out,
                                   int** d_off) {
                std::vector<int> coff(C + 1, 0);
                for (int c = 0; c < C; ++c) {
                    const MsdConfig& m = pb->cfg[c];
                    const long long rows = (long long)m.M * m.n;
                    for (long long r0 = 0; r0 < rows; r0 += target_rows) {
                        RowChunk ch;
                        ch.cfg = c;
                        ch.pad = 0;
                        ch.row0 = m.row_off + r0;
                        ch.row1 = m.row_off + std::min(rows, r0 + target_rows);
                        out.push_back(ch);
                    }
                    coff[c + 1] = (int)out.size();
                }
                *d_out = dalloc_copy(out.data(), out.size());
                *d_off = dalloc_copy(coff.data(), coff.size());
            };
            make_chunks(std::max<long long>(512, row / 256), pb->chunks, &pb->d_chunks, &pb->d_cfg_chunk_off);
            make_chunks(std::max<long long>(4096, row / 64), pb->chunks_coarse, &pb->d_chunks_coarse,
                        &pb->d_cfg_chunk_off_coarse);
            make_chunks(std::max<long long>(1024, row / 128), pb->chunks_mid, &pb->d_chunks_mid,
                        &pb->d_cfg_chunk_off_mid);
            launch_disk_diagonals(pb->d_cfg, Mtot, pb->d_disk_cfg, pb->d_radius, pb->d_bc, pb->Nmax, pb->d_J,
                                  pb->d_dJ, pb->d_H, pb->d_dH, pb->d_lf64, pb->d_rf64, pb->d_lf32, pb->d_rf32,
                                  pb->d_rhs_scale, pb->d_flags, pb->stream);
            CK_LAUNCH();
            check_flags(pb, "disk diagonals");
        } catch (...) {
            msd_destroy(pb);
            throw;
        }
        *out = pb;
        return MSD_OK;
    });
}

void msd_destroy(msd_problem* pb) {
    if (!pb) return;
    if (pb->stream) cudaStreamSynchronize(pb->stream);
    void* ptrs[] = {pb->d_cfg, pb->d_centre, pb->d_radius, pb->d_bc, pb->d_disk_cfg, pb->d_J, pb->d_dJ,
                    pb->d_H, pb->d_dH, pb->d_lf64, pb->d_rhs_scale, pb->d_rf64, pb->d_lf32, pb->d_rf32,
                    pb->d_flags, pb->d_G64, pb->d_G32, pb->d_chunks, pb->d_cfg_chunk_off,
                    pb->d_chunks_coarse, pb->d_cfg_chunk_off_coarse, pb->d_chunks_mid, pb->d_cfg_chunk_off_mid,
                    pb->d_GA64, pb->d_GA32, pb->d_clf64, pb->d_clf32, pb->d_GT, pb->d_gt_blk, pb->d_Np};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& kv : pb->plans)
        if (kv.second.d_work) cudaFree(kv.second.d_work);
    free_recompute_plans(pb);
    if (pb->d_gen_full) cudaFree(pb->d_gen_full);
    pb->genbuf.release();
    if (pb->h_pinned) cudaFreeHost(pb->h_pinned);
    for (cudaEvent_t e : pb->events) cudaEventDestroy(e);
    for (cudaEvent_t e : pb->ring_ev)
        if (e) cudaEventDestroy(e);
    pb->xs.release();
    pb->xt.release();
    pb->part.release();
    for (auto& b : pb->sbuf) b.release();
    for (auto& b : pb->gbuf) b.release();
    for (auto& b : pb->nfbuf) b.release();
    for (auto& b : pb->dortbuf) b.release();
    pb->fbuf.release();
    if (pb->pen_minus) msd_destroy(pb->pen_minus);
    if (pb->pen_shadow) msd_destroy(pb->pen_shadow);
    pb->penbuf.release();
    for (auto& b : pb->penio) b.release();
    delete pb;
}

int64_t msd_num_unknowns(const msd_problem* pb) { return pb ? pb->Ntot : -1; }

int64_t msd_row_offset(const msd_problem* pb, int config) {
    if (!pb || config < 0 || config > pb->C) return -1;
    return config == pb->C ? pb->Ntot : pb->cfg[config].row_off;
}

msd_status msd_disk_diagonals(msd_problem* pb, void* out) {
    return guarded([&]() -> msd_status {
        if (!pb || !out) fail(MSD_ERR_ARG, "msd_disk_diagonals: bad argument");
        const size_t bytes = (size_t)pb->Ntot * 16;
        OutStage o(pb, pb->sbuf[20], out, 4 * bytes);
        const double2* src[4] = {pb->d_J, pb->d_dJ, pb->d_H, pb->d_dH};
        for (int i = 0; i < 4; ++i)
            CK(cudaMemcpyAsync((char*)o.dev + i * bytes, src[i], bytes, cudaMemcpyDeviceToDevice, pb->stream));
        o.finish();
        return MSD_OK;
    });
}

msd_status msd_pair_generators(msd_problem* pb, int config, void* out) {
    return guarded([&]() -> msd_status {
        if (!pb || !out || config < 0 || config >= pb->C) fail(MSD_ERR_ARG, "msd_pair_generators: bad argument");
        ensure_generators(pb, true);
        const MsdConfig& c = pb->cfg[config];
        const size_t rowb = (size_t)c.M * c.L * 16;
        OutStage o(pb, pb->sbuf[20], out, rowb * c.M);
        CK(cudaMemcpy2DAsync(o.dev, rowb, pb->d_G64 + c.gen_off, (size_t)c.Mp * c.L * 16, rowb, c.M,
                             cudaMemcpyDeviceToDevice, pb->stream));
        o.finish();
        return MSD_OK;
    });
}

msd_status msd_rhs_planewave(msd_problem* pb, int R, const double* betas_host, void* out) {
    return guarded([&]() -> msd_status {
        if (!pb || R <= 0 || !betas_host || !out) fail(MSD_ERR_ARG, "msd_rhs_planewave: bad argument");
        double* d_betas = (double*)pb->sbuf[21].get((size_t)pb->C * R * 8);
        CK(cudaMemcpyAsync(d_betas, betas_host, (size_t)pb->C * R * 8, cudaMemcpyHostToDevice, pb->stream));
        OutStage o(pb, pb->sbuf[20], out, (size_t)pb->Ntot * R * 16);
        launch_rhs_planewave(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_centre, pb->d_radius, rhs_scale_of(pb),
                             pb->Nmax, R, d_betas, (double2*)o.dev, pb->stream);
        CK_LAUNCH();
        o.finish();
        return MSD_OK;
    });
}

msd_status msd_matvec(msd_problem* pb, int R, int precision, const void* x_dev, void* y_dev) {
    return guarded([&]() -> msd_status {
        if (!pb || R <= 0 || !x_dev || !y_dev) fail(MSD_ERR_ARG, "msd_matvec: bad argument");
        if (precision != MSD_FP64 && precision != MSD_FP32) fail(MSD_ERR_ARG, "msd_matvec: precision");
        if (!is_device_ptr(x_dev) || !is_device_ptr(y_dev)) fail(MSD_ERR_ARG, "msd_matvec: x and y must be device memory");
        if (ranges_overlap(x_dev, y_dev, (size_t)pb->Ntot * R * (precision == MSD_FP64 ? 16 : 8)))
            fail(MSD_ERR_ARG, "msd_matvec: x and y must not overlap");
        matvec_dev(pb, R, precision == MSD_FP64, x_dev, y_dev);
        return MSD_OK;
    });
}

msd_status msd_solve_planewaves(msd_problem* pb, int R, const double* betas_host, const msd_opts* opts,
                                void* rho_out, msd_stats* stats_host) {
    return guarded([&]() -> msd_status { return solve_impl(pb, R, betas_host, opts, rho_out, stats_host); });
}

msd_status msd_update_geometry(msd_problem* pb, const double* centres, const double* radii, const double* k_host) {
    return guarded([&]() -> msd_status {
        if (!pb) fail(MSD_ERR_ARG, "msd_update_geometry: bad handle");
        if (k_host) {
            for (int c = 0; c < pb->C; ++c) {
                if (!(k_host[c] > 0) || !std::isfinite(k_host[c])) fail(MSD_ERR_ARG, "msd_update_geometry: k must be positive");
                pb->cfg[c].k = k_host[c];
            }
            CK(cudaMemcpyAsync(pb->d_cfg, pb->cfg.data(), pb->C * sizeof(MsdConfig), cudaMemcpyHostToDevice, pb->stream));
        }
        if (centres)
            CK(cudaMemcpyAsync(pb->d_centre, centres, (size_t)pb->Mtot * 16,
                               is_device_ptr(centres) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, pb->stream));
        if (radii)
            CK(cudaMemcpyAsync(pb->d_radius, radii, (size_t)pb->Mtot * 8,
                               is_device_ptr(radii) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, pb->stream));
        CK(cudaMemsetAsync(pb->d_flags, 0, sizeof(int), pb->stream));
        launch_disk_diagonals(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_radius, pb->d_bc, pb->Nmax, pb->d_J,
                              pb->d_dJ, pb->d_H, pb->d_dH, pb->d_lf64, pb->d_rf64, pb->d_lf32, pb->d_rf32,
                              pb->d_rhs_scale, pb->d_flags, pb->stream);
        CK_LAUNCH();
        if (pb->d_G64 || pb->d_G32) launch_full_generators(pb, pb->d_G64, pb->d_G32);
        CK_LAUNCH();
        check_flags(pb, "msd_update_geometry");
        apply_truncation(pb);
        if (pb->form) form_rows(pb);
        if (pb->pen_minus) {
            const msd_status st = msd_update_geometry(pb->pen_minus, centres, radii, nullptr);
            if (st != MSD_OK) fail(st, std::string("msd_update_geometry (interior wavenumber): ") + msd_last_error());
            pen_rows(pb);
        }
        pb->geom_version += 1;  // adjoint operator data is rebuilt on next use
        return MSD_OK;
    });
}

msd_status msd_set_truncation(msd_problem* pb, const int* Np) {
    return guarded([&]() -> msd_status {
        if (!pb) fail(MSD_ERR_ARG, "msd_set_truncation: bad handle");
        if (pb->form || pb->pen_minus || pb->pen_parent)
            fail(MSD_ERR_ARG, "msd_set_truncation: needs the default rows (no formulation, not penetrable)");
        if (Np)
            for (const MsdConfig& c : pb->cfg)
                for (int d = c.disk_off; d < c.disk_off + c.M; ++d)
                    if (Np[d] < 0 || Np[d] > c.N)
                        fail(MSD_ERR_ARG, "msd_set_truncation: N_p of disk " + std::to_string(d) +
                                              " outside 0..N of its configuration");
        CK(cudaStreamSynchronize(pb->stream));
        if (pb->d_Np) cudaFree(pb->d_Np);
        pb->d_Np = nullptr;
        pb->Np.clear();
        if (Np) {
            pb->Np.assign(Np, Np + pb->Mtot);
            pb->d_Np = dalloc_copy(pb->Np.data(), pb->Mtot);
        }
        // fresh factors of every row, then the mask
        CK(cudaMemsetAsync(pb->d_flags, 0, sizeof(int), pb->stream));
        launch_disk_diagonals(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_radius, pb->d_bc, pb->Nmax, pb->d_J,
                              pb->d_dJ, pb->d_H, pb->d_dH, pb->d_lf64, pb->d_rf64, pb->d_lf32, pb->d_rf32,
                              pb->d_rhs_scale, pb->d_flags, pb->stream);
        CK_LAUNCH();
        check_flags(pb, "msd_set_truncation");
        apply_truncation(pb);
        count_offdiag(pb);
        pb->geom_version += 1;  // adjoint row factors are rebuilt on next use
        CK(cudaStreamSynchronize(pb->stream));
        return MSD_OK;
    });
}

msd_status msd_set_generator_mode(msd_problem* pb, int mode, int64_t chunk_bytes) {
    return guarded([&]() -> msd_status {
        if (!pb || chunk_bytes < 0) fail(MSD_ERR_ARG, "msd_set_generator_mode: bad argument");
        if (mode != MSD_GEN_AUTO && mode != MSD_GEN_STREAMED && mode != MSD_GEN_RECOMPUTE)
            fail(MSD_ERR_ARG, "msd_set_generator_mode: mode");
        if (mode == MSD_GEN_AUTO) {
            size_t free_b = 0, total_b = 0;
            CK(cudaMemGetInfo(&free_b, &total_b));
            const double need = (double)pb->gen_elems * (16.0 + 8.0);  // complex128 and complex64 copies
            mode = need <= 0.5 * (double)free_b ? MSD_GEN_STREAMED : MSD_GEN_RECOMPUTE;
        }
        const size_t budget = chunk_bytes ? (size_t)chunk_bytes : (64ull << 20);
        CK(cudaStreamSynchronize(pb->stream));
        if (budget != pb->gen_chunk_bytes) free_recompute_plans(pb);
        pb->gen_chunk_bytes = budget;
        pb->gen_mode = mode;
        if (mode == MSD_GEN_RECOMPUTE) {
            if (pb->d_G64) cudaFree(pb->d_G64);
            if (pb->d_G32) cudaFree(pb->d_G32);
            if (pb->d_GT) cudaFree(pb->d_GT);
            pb->d_G64 = nullptr;
            pb->d_G32 = nullptr;
            pb->d_GT = nullptr;
            pb->gt_version = -1;
            pb->xt.release();
        } else {
            free_recompute_plans(pb);
            pb->genbuf.release();
        }
        return MSD_OK;
    });
}

msd_status msd_plan_info(msd_problem* pb, int R, int precision, int* out, double* tuned_ms) {
    return guarded([&]() -> msd_status {
        if (!pb || R <= 0 || !out) fail(MSD_ERR_ARG, "msd_plan_info: bad argument");
        if (precision != MSD_FP64 && precision != MSD_FP32) fail(MSD_ERR_ARG, "msd_plan_info: precision");
        const bool fp64 = precision == MSD_FP64;
        if (pb->gen_mode == MSD_GEN_RECOMPUTE && !pb->form && !pb->pen_minus) {
            // the plan of recomputed products (chunked generators)
            RecomputePlan& rp = get_recompute_plan(pb, R, fp64);
            out[0] = rp.ch.KB + 100 * rp.ch.P2;
            out[1] = rp.ch.RT;
            out[2] = rp.nsplit;
            out[3] = 0;
            if (tuned_ms) *tuned_ms = 0;
            return MSD_OK;
        }
        ensure_generators(pb, fp64);
        MatvecPlan& plan = get_plan(pb, R, fp64, true);
        out[0] = plan.ch.KB + 100 * plan.ch.P2;
        out[1] = plan.ch.RT;
        out[2] = plan.nsplit;
        out[3] = plan.candidates;
        if (tuned_ms) *tuned_ms = plan.tuned_ms;
        return MSD_OK;
    });
}

msd_status msd_set_tile(msd_problem* pb, int R, int precision, int KB, int RT) {
    return guarded([&]() -> msd_status {
        if (!pb || R <= 0) fail(MSD_ERR_ARG, "msd_set_tile: bad argument");
        if (precision != MSD_FP64 && precision != MSD_FP32) fail(MSD_ERR_ARG, "msd_set_tile: precision");
        const bool fp64 = precision == MSD_FP64;
        MatvecChoice cand[128];
        const int nc = matvec_candidates(R, pb->Nmax, fp64, cand, 128, true);
        int hit = -1;
        for (int i = 0; i < nc; ++i)
            if (cand[i].KB + 100 * cand[i].P2 == KB && cand[i].RT == RT) hit = i;
        if (hit < 0) fail(MSD_ERR_ARG, "msd_set_tile: (KB, RT) is not an instantiated shape that fits");
        const long long key = (long long)R * 4 + (fp64 ? 0 : 1);
        for (int sh = 0; sh < 2; ++sh) {
            auto it = pb->plans.find(plan_key(R, fp64, sh != 0));
            if (it != pb->plans.end()) {
                CK(cudaStreamSynchronize(pb->stream));  // the old work list may still be read
                if (it->second.d_work) cudaFree(it->second.d_work);
                pb->plans.erase(it);
            }
        }
        auto rit = pb->rplans.find(key);
        if (rit != pb->rplans.end()) {
            CK(cudaStreamSynchronize(pb->stream));
            for (auto& ch : rit->second.chunks) {
                cudaFree(ch.d_cfg);
                cudaFree(ch.d_blocks);
                cudaFree(ch.d_work);
            }
            pb->rplans.erase(rit);
        }
        pb->pinned[key] = cand[hit];
        return MSD_OK;
    });
}

msd_status msd_matvec_timing(msd_problem* pb, int enable, double* kernel_ms, int64_t* launches,
                             double* flops, double* bytes) {
    return guarded([&]() -> msd_status {
        if (!pb) fail(MSD_ERR_ARG, "msd_matvec_timing: bad handle");
        flush_timing(pb);
        check_tc("msd_matvec_timing");
        if (kernel_ms) *kernel_ms = pb->timed_ms;
        if (launches) *launches = pb->timed_launches;
        if (flops) *flops = pb->timed_flops;
        if (bytes) *bytes = pb->timed_bytes;
        if (enable >= 0) {
            pb->timing = enable != 0;
            pb->timed_ms = pb->timed_flops = pb->timed_bytes = 0;
            pb->timed_launches = 0;
        }
        return MSD_OK;
    });
}

int64_t msd_kernel_launches(void) { return g_msd_launches.load(); }

void msd_test_expire_waits(int on) { g_msd_expire_waits.store(on ? 1 : 0); }

msd_status msd_grad_farfield_misfit(msd_problem* pb, int R, const double* betas_host, int T,
                                    const double* thetas_host, const void* F_target, const msd_opts* opts,
                                    double* J_out, double* dO, double* da, double* dk) {
    return guarded([&]() -> msd_status {
        if (!pb || R <= 0 || T <= 0 || !betas_host || !thetas_host || !F_target)
            fail(MSD_ERR_ARG, "msd_grad_farfield_misfit: bad argument");
        if (pb->form) fail(MSD_ERR_ARG, "msd_grad_farfield_misfit: needs the default formulation");
        if (pb->d_Np) fail(MSD_ERR_ARG, "msd_grad_farfield_misfit: not with per-disk truncation orders");
        cudaStream_t s = pb->stream;
        const long long nv = pb->Ntot * R;
        const size_t nF = (size_t)pb->C * T * R;
        msd_opts o;
        memset(&o, 0, sizeof(o));
        if (opts) o = *opts;
        if (o.tol <= 0) o.tol = 1e-12;
        // work buffers (library-owned, separate from the solver's)
        double2* rho = (double2*)pb->gbuf[0].get(nv * 16);
        double2* mu = (double2*)pb->gbuf[1].get(nv * 16);
        double2* F = (double2*)pb->gbuf[2].get(nF * 16 * 3);
        double2* w = F + nF;
        double2* Ft = w + nF;
        double2* u = (double2*)pb->gbuf[3].get(nv * 16);
        double2* sv = (double2*)pb->gbuf[4].get(nv * 16);
        double2* tv = (double2*)pb->gbuf[5].get(nv * 16);
        const int nmax = 2 * pb->Nmax + 1;
        double2* E = (double2*)pb->gbuf[6].get((size_t)pb->C * nmax * T * 16);
        // thetas, betas, J, gO, ga, gk
        double* d_par = (double*)pb->gbuf[7].get((size_t)(T + pb->C * R + pb->C + 3 * pb->Mtot + pb->C) * 8);
        double* d_th = d_par;
        double* d_beta = d_th + T;
        double* d_J = d_beta + (size_t)pb->C * R;
        double* d_gO = d_J + pb->C;
        double* d_ga = d_gO + 2 * pb->Mtot;
        double* d_gk = d_ga + pb->Mtot;
        CK(cudaMemcpyAsync(d_th, thetas_host, (size_t)T * 8, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_beta, betas_host, (size_t)pb->C * R * 8, cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(d_J, 0, (size_t)(pb->C + 3 * pb->Mtot + pb->C) * 8, s));
        CK(cudaMemcpyAsync(Ft, F_target, nF * 16, is_device_ptr(F_target) ? cudaMemcpyDeviceToDevice
                                                                            : cudaMemcpyHostToDevice, s));
        // 1. forward solve and far field (Prop. 4.1, section 5, section 4.4)
        msd_stats* st_fwd = nullptr;
        msd_status st = solve_impl(pb, R, betas_host, &o, rho, st_fwd);
        if (st != MSD_OK) fail(st, "msd_grad_farfield_misfit: forward solve did not converge");
        launch_farfield(pb->d_cfg, pb->C, pb->cfg.data(), pb->d_centre, pb->d_radius, pb->d_J, R, T, d_th, rho,
                        nullptr, F, s);
        launch_misfit(pb->C, T, R, F, Ft, w, d_J, s);
        // 2. adjoint right-hand side C^H w and adjoint solve (P^-1 A)^H mu = C^H w
        launch_ff_table(pb->d_cfg, pb->C, nmax, T, d_th, E, s);
        launch_farfield_adj(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_centre, pb->d_radius, pb->d_J, nmax, T, R,
                            d_th, E, w, u, s);
        CK_LAUNCH();
        st = solve_impl(pb, R, nullptr, &o, mu, nullptr, u, true);
        if (st != MSD_OK) fail(st, "msd_grad_farfield_misfit: adjoint solve did not converge");
        // 3. raw Toeplitz sums s = T(r .* rho), t = T^H(conj(l) .* mu)
        product_dev(pb, R, true, false, true, rho, sv);
        product_dev(pb, R, true, true, true, mu, tv);
        // 4. pair correlations, far-field term, per-row terms
        double2* muh = u;  // u is no longer needed
        double2* rhoh = (double2*)pb->gbuf[8].get(nv * 16);
        launch_scale_pair_inputs(pb->Ntot, R, pb->d_lf64, pb->d_rf64, mu, rho, muh, rhoh, s);
        launch_pair_grad(pb->d_cfg, pb->C, pb->cfg.data(), pb->d_centre, pb->d_G64, R, muh, rhoh, d_gO, d_gk, s);
        launch_farfield_grad(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_centre, pb->d_radius, pb->d_J, pb->d_dJ, nmax,
                             T, R, d_th, E, w, rho, d_gO, d_ga, d_gk, s);
        launch_grad_rows(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_centre, pb->d_radius, pb->d_bc, pb->d_J,
                         pb->d_dJ, pb->d_H, pb->d_dH, R, d_beta, mu, rho, sv, tv, d_gO, d_ga, d_gk, s);
        CK_LAUNCH();
        // 5. results
        auto out = [&](void* dst, const double* src, size_t n) {
            if (!dst) return;
            CK(cudaMemcpyAsync(dst, src, n * 8, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               s));
        };
        out(J_out, d_J, pb->C);
        out(dO, d_gO, 2 * (size_t)pb->Mtot);
        out(da, d_ga, pb->Mtot);
        out(dk, d_gk, pb->C);
        CK(cudaStreamSynchronize(s));
        return MSD_OK;
    });
}

msd_status msd_farfield(msd_problem* pb, const void* rho, int R, int T, const double* thetas_host, void* F_out) {
    return guarded([&]() -> msd_status {
        if (!pb || !rho || R <= 0 || T <= 0 || !thetas_host || !F_out) fail(MSD_ERR_ARG, "msd_farfield: bad argument");
        double* d_th = (double*)pb->sbuf[21].get((size_t)T * 8);
        CK(cudaMemcpyAsync(d_th, thetas_host, (size_t)T * 8, cudaMemcpyHostToDevice, pb->stream));
        const double2* d_rho = (const double2*)stage_in(pb, pb->sbuf[22], rho, (size_t)pb->Ntot * R * 16);
        OutStage o(pb, pb->sbuf[23], F_out, (size_t)pb->C * T * R * 16);
        launch_farfield(pb->d_cfg, pb->C, pb->cfg.data(), pb->d_centre, pb->d_radius, field_factor_of(pb), R, T, d_th, d_rho,
                        nullptr, (double2*)o.dev, pb->stream);
        CK_LAUNCH();
        o.finish();
        return MSD_OK;
    });
}

msd_status msd_rhs_pointsource(msd_problem* pb, int R, const double* sources_host, void* out) {
    return guarded([&]() -> msd_status {
        if (!pb || R <= 0 || !sources_host || !out) fail(MSD_ERR_ARG, "msd_rhs_pointsource: bad argument");
        double2* d_src = (double2*)pb->sbuf[21].get((size_t)pb->C * R * 16);
        CK(cudaMemcpyAsync(d_src, sources_host, (size_t)pb->C * R * 16, cudaMemcpyHostToDevice, pb->stream));
        OutStage o(pb, pb->sbuf[20], out, (size_t)pb->Ntot * R * 16);
        launch_rhs_pointsource(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_centre, pb->d_radius, rhs_scale_of(pb), R,
                               d_src, (double2*)o.dev, pb->stream);
        CK_LAUNCH();
        o.finish();
        return MSD_OK;
    });
}

msd_status msd_solve_pointsources(msd_problem* pb, int R, const double* sources_host, const msd_opts* opts,
                                  void* rho_out, msd_stats* stats_host) {
    return guarded([&]() -> msd_status {
        if (!pb || R <= 0 || !sources_host || !rho_out) fail(MSD_ERR_ARG, "msd_solve_pointsources: bad argument");
        double2* d_src = (double2*)pb->nfbuf[1].get((size_t)pb->C * R * 16);
        CK(cudaMemcpyAsync(d_src, sources_host, (size_t)pb->C * R * 16, cudaMemcpyHostToDevice, pb->stream));
        double2* b = (double2*)pb->nfbuf[2].get((size_t)pb->Ntot * R * 16);
        launch_rhs_pointsource(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_centre, pb->d_radius, rhs_scale_of(pb), R,
                               d_src, b, pb->stream);
        CK_LAUNCH();
        return solve_impl(pb, R, nullptr, opts, rho_out, stats_host, b);
    });
}

msd_status msd_set_penetrable(msd_problem* pb, const double* k_minus, const double* mu) {
    return guarded([&]() -> msd_status {
        if (!pb || pb->pen_parent) fail(MSD_ERR_ARG, "msd_set_penetrable: bad handle");
        if (!k_minus) {
            pen_release(pb);
            return MSD_OK;
        }
        if (pb->d_Np) fail(MSD_ERR_ARG, "msd_set_penetrable: not with per-disk truncation orders");
        if (pb->form) fail(MSD_ERR_ARG, "msd_set_penetrable: needs the default formulation");
        const int C = pb->C, Mtot = pb->Mtot;
        for (int c = 0; c < C; ++c)
            if (!(k_minus[c] > 0) || !std::isfinite(k_minus[c])) fail(MSD_ERR_ARG, "msd_set_penetrable: k- must be positive");
        std::vector<double> muv(Mtot, 1.0);
        if (mu)
            for (int d = 0; d < Mtot; ++d) {
                if (!(mu[d] > 0) || !std::isfinite(mu[d])) fail(MSD_ERR_ARG, "msd_set_penetrable: mu must be positive");
                muv[d] = mu[d];
            }
        std::vector<double> cen(2 * (size_t)Mtot), rad(Mtot);
        CK(cudaMemcpyAsync(cen.data(), pb->d_centre, cen.size() * 8, cudaMemcpyDeviceToHost, pb->stream));
        CK(cudaMemcpyAsync(rad.data(), pb->d_radius, rad.size() * 8, cudaMemcpyDeviceToHost, pb->stream));
        CK(cudaStreamSynchronize(pb->stream));
        std::vector<int> doff(C + 1), Nv(C), sdoff(C + 1);
        std::vector<double> kp(C);
        for (int c = 0; c < C; ++c) {
            doff[c] = pb->cfg[c].disk_off;
            Nv[c] = pb->cfg[c].N;
            kp[c] = pb->cfg[c].k;
        }
        doff[C] = Mtot;
        pen_release(pb);
        std::vector<int8_t> bc0(2 * (size_t)Mtot, (int8_t)MSD_DIRICHLET);
        msd_problem* pm = nullptr;
        msd_status st = msd_create(C, doff.data(), cen.data(), rad.data(), bc0.data(), k_minus, Nv.data(), pb->stream, &pm);
        if (st != MSD_OK) fail(st, std::string("msd_set_penetrable (interior wavenumber): ") + msd_last_error());
        pb->pen_minus = pm;
        // Krylov layout: 2 M disk slots per configuration, placed apart on a
        // line (their geometry is never used)
        std::vector<double> scen, srad;
        sdoff[0] = 0;
        for (int c = 0; c < C; ++c) {
            const int M = doff[c + 1] - doff[c];
            double amax = 0;
            for (int d = doff[c]; d < doff[c + 1]; ++d) amax = std::max(amax, rad[d]);
            for (int j = 0; j < 2 * M; ++j) {
                scen.push_back(j * (2.0 * amax + 1.0));
                scen.push_back(0.0);
                srad.push_back(rad[doff[c] + (j % M)]);
            }
            sdoff[c + 1] = sdoff[c] + 2 * M;
        }
        msd_problem* sh = nullptr;
        st = msd_create(C, sdoff.data(), scen.data(), srad.data(), bc0.data(), kp.data(), Nv.data(), pb->stream, &sh);
        if (st != MSD_OK) fail(st, std::string("msd_set_penetrable (solver layout): ") + msd_last_error());
        sh->pen_parent = pb;
        pb->pen_shadow = sh;
        const size_t n = (size_t)pb->Ntot;
        char* b = (char*)pb->penbuf.get(n * 4 * 16 + n * 4 * 8 + 2 * n * 16 + (size_t)Mtot * 8);
        pb->d_penA64 = (double2*)b;
        pb->d_penA32 = (float2*)(pb->d_penA64 + 4 * n);
        pb->d_penS = (double2*)(pb->d_penA32 + 4 * n);
        pb->d_pen_mu = (double*)(pb->d_penS + 2 * n);
        CK(cudaMemcpyAsync(pb->d_pen_mu, muv.data(), (size_t)Mtot * 8, cudaMemcpyHostToDevice, pb->stream));
        pen_rows(pb);
        return MSD_OK;
    });
}

msd_status msd_penetrable_matvec(msd_problem* pb, int R, int precision, const void* xp, const void* xm, void* yp,
                                 void* ym) {
    return guarded([&]() -> msd_status {
        if (!pb || !pb->pen_shadow || R <= 0 || !xp || !xm || !yp || !ym)
            fail(MSD_ERR_ARG, "msd_penetrable_matvec: bad argument (msd_set_penetrable first)");
        if (precision != MSD_FP64)
            fail(MSD_ERR_ARG, "msd_penetrable_matvec: MSD_FP64 only (FP32 products run inside mixed-precision solves)");
        for (const void* p : {xp, xm, (const void*)yp, (const void*)ym})
            if (!is_device_ptr(p)) fail(MSD_ERR_ARG, "msd_penetrable_matvec: device memory expected");
        const size_t nv = (size_t)pb->Ntot * R;
        double2* X = (double2*)pb->penio[0].get(2 * nv * 16);
        double2* Y = (double2*)pb->penio[1].get(2 * nv * 16);
        launch_pen_layout(pb->d_cfg, pb->C, pb->Ntot, R, true, X, (double2*)xp, (double2*)xm, pb->stream);
        pen_matvec(pb, R, true, X, Y);
        launch_pen_layout(pb->d_cfg, pb->C, pb->Ntot, R, false, Y, (double2*)yp, (double2*)ym, pb->stream);
        CK_LAUNCH();
        CK(cudaStreamSynchronize(pb->stream));
        return MSD_OK;
    });
}

}  // extern "C"

namespace {

// Transmission solve for plane waves (betas_host [C][R]) or point sources
// (sources_host [C][R][2]).
msd_status solve_penetrable_impl(msd_problem* pb, int R, const double* betas_host, const double* sources_host,
                                 const msd_opts* opts, void* rho_plus, void* rho_minus, msd_stats* stats_host) {
    if (!pb || !pb->pen_shadow || R <= 0 || (!betas_host && !sources_host) || !rho_plus || !rho_minus)
        fail(MSD_ERR_ARG, "msd_solve_penetrable: bad argument (msd_set_penetrable first)");
    cudaStream_t s = pb->stream;
    const size_t nv = (size_t)pb->Ntot * R;
    double2* bp = (double2*)pb->penio[0].get(2 * nv * 16);
    double2* bm = bp + nv;
    if (betas_host) {
        double* d_betas = (double*)pb->penio[3].get((size_t)pb->C * R * 8);
        CK(cudaMemcpyAsync(d_betas, betas_host, (size_t)pb->C * R * 8, cudaMemcpyHostToDevice, s));
        launch_rhs_planewave(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_centre, pb->d_radius, pb->d_penS, pb->Nmax,
                             R, d_betas, bp, s);
        launch_rhs_planewave(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_centre, pb->d_radius, pb->d_penS + pb->Ntot,
                             pb->Nmax, R, d_betas, bm, s);
    } else {
        double2* d_src = (double2*)pb->penio[3].get((size_t)pb->C * R * 16);
        CK(cudaMemcpyAsync(d_src, sources_host, (size_t)pb->C * R * 16, cudaMemcpyHostToDevice, s));
        launch_rhs_pointsource(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_centre, pb->d_radius, pb->d_penS, R, d_src,
                               bp, s);
        launch_rhs_pointsource(pb->d_cfg, pb->Mtot, pb->d_disk_cfg, pb->d_centre, pb->d_radius,
                               pb->d_penS + pb->Ntot, R, d_src, bm, s);
    }
    double2* b = (double2*)pb->penio[1].get(2 * nv * 16);
    launch_pen_layout(pb->d_cfg, pb->C, pb->Ntot, R, true, b, bp, bm, s);
    CK_LAUNCH();
    double2* x = (double2*)pb->penio[2].get(2 * nv * 16);
    const msd_status st = solve_impl(pb->pen_shadow, R, nullptr, opts, x, stats_host, b);
    OutStage op(pb, pb->nfbuf[0], rho_plus, nv * 16), om(pb, pb->nfbuf[3], rho_minus, nv * 16);
    launch_pen_layout(pb->d_cfg, pb->C, pb->Ntot, R, false, x, (double2*)op.dev, (double2*)om.dev, s);
    CK_LAUNCH();
    op.finish();
    om.finish();
    CK(cudaStreamSynchronize(s));
    return st;
}

}  // namespace

extern "C" {

msd_status msd_solve_penetrable(msd_problem* pb, int R, const double* betas_host, const msd_opts* opts,
                                void* rho_plus, void* rho_minus, msd_stats* stats_host) {
    return guarded([&]() -> msd_status {
        if (!betas_host) fail(MSD_ERR_ARG, "msd_solve_penetrable: betas_host is NULL");
        return solve_penetrable_impl(pb, R, betas_host, nullptr, opts, rho_plus, rho_minus, stats_host);
    });
}

msd_status msd_solve_penetrable_pointsources(msd_problem* pb, int R, const double* sources, const msd_opts* opts,
                                             void* rho_plus, void* rho_minus, msd_stats* stats_host) {
    return guarded([&]() -> msd_status {
        if (!sources) fail(MSD_ERR_ARG, "msd_solve_penetrable_pointsources: sources is NULL");
        return solve_penetrable_impl(pb, R, nullptr, sources, opts, rho_plus, rho_minus, stats_host);
    });
}

msd_status msd_set_formulation(msd_problem* pb, const double* op_weights, const double* rhs_weights,
                               const double* rep_weights) {
    return guarded([&]() -> msd_status {
        if (!pb) fail(MSD_ERR_ARG, "msd_set_formulation: bad handle");
        if (!op_weights) {
            pb->form = false;
            return MSD_OK;
        }
        if (!rhs_weights || !rep_weights) fail(MSD_ERR_ARG, "msd_set_formulation: bad argument");
        if (pb->pen_minus) fail(MSD_ERR_ARG, "msd_set_formulation: not with penetrable obstacles");
        if (pb->d_Np) fail(MSD_ERR_ARG, "msd_set_formulation: not with per-disk truncation orders");
        MsdFormulation w{};
        for (int c = 0; c < 2; ++c) {
            for (int o = 0; o < 5; ++o)
                w.op[c][o] = make_double2(op_weights[(c * 5 + o) * 2], op_weights[(c * 5 + o) * 2 + 1]);
            for (int o = 0; o < 2; ++o)
                w.rhs[c][o] = make_double2(rhs_weights[(c * 2 + o) * 2], rhs_weights[(c * 2 + o) * 2 + 1]);
        }
        for (int o = 0; o < 2; ++o) w.rep[o] = make_double2(rep_weights[2 * o], rep_weights[2 * o + 1]);
        for (const double2* v = &w.op[0][0]; v < &w.op[0][0] + 10; ++v)
            if (!std::isfinite(v->x) || !std::isfinite(v->y)) fail(MSD_ERR_ARG, "msd_set_formulation: weight");
        pb->fw = w;
        pb->form = true;
        form_rows(pb);
        return MSD_OK;
    });
}

msd_status msd_penetrable_interior_field(msd_problem* pb, int config, const void* rho_minus, int R, int64_t P,
                                         const double* points, void* u_out) {
    return guarded([&]() -> msd_status {
        if (!pb || !pb->pen_minus || !rho_minus || R <= 0 || P <= 0 || !points || !u_out || config < 0 ||
            config >= pb->C)
            fail(MSD_ERR_ARG, "msd_penetrable_interior_field: bad argument (msd_set_penetrable first)");
        msd_problem* pm = pb->pen_minus;
        const double2* d_rho = (const double2*)stage_in(pb, pb->nfbuf[0], rho_minus, (size_t)pb->Ntot * R * 16);
        const double2* d_pts = (const double2*)stage_in(pb, pb->nfbuf[1], points, (size_t)P * 16);
        double2* W = (double2*)pb->nfbuf[2].get((size_t)pb->Ntot * R * 2 * 16);
        OutStage o(pb, pb->nfbuf[3], u_out, (size_t)P * R * 16);
        launch_nearfield_inside(pm->d_cfg, config, pm->cfg[config], pm->cfg[config].k, pm->d_centre, pm->d_radius,
                                pm->d_J, pm->d_H, d_rho, R, W, W + (size_t)pb->Ntot * R, d_pts, P, (double2*)o.dev,
                                pb->stream);
        CK_LAUNCH();
        o.finish();
        return MSD_OK;
    });
}

}  // extern "C"

namespace {

// Arguments of a named formulation: CFIE needs 0 <= alpha <= 1, CFIE and
// Brakhage-Werner a coupling eta with a non-zero imaginary part (section 3).
void check_kind(const char* where, int kind, double alpha, const double* eta) {
    if (kind != MSD_FORM_EFIE && kind != MSD_FORM_MFIE && kind != MSD_FORM_CFIE && kind != MSD_FORM_BWIE)
        fail(MSD_ERR_ARG, std::string(where) + ": unknown formulation kind");
    if (kind == MSD_FORM_CFIE && !(alpha >= 0.0 && alpha <= 1.0))
        fail(MSD_ERR_ARG, std::string(where) + ": CFIE needs 0 <= alpha <= 1");
    if ((kind == MSD_FORM_CFIE || kind == MSD_FORM_BWIE) && eta &&
        (!std::isfinite(eta[0]) || !std::isfinite(eta[1]) || eta[1] == 0.0))
        fail(MSD_ERR_ARG, std::string(where) + ": eta needs a finite, non-zero imaginary part");
}

}  // namespace

extern "C" {

msd_status msd_set_formulation_kind(msd_problem* pb, int kind, double alpha, const double* eta) {
    return guarded([&]() -> msd_status {
        if (!pb) fail(MSD_ERR_ARG, "msd_set_formulation_kind: bad handle");
        check_kind("msd_set_formulation_kind", kind, alpha, eta);
        if (pb->pen_minus) fail(MSD_ERR_ARG, "msd_set_formulation_kind: not with penetrable obstacles");
        if (pb->d_Np) fail(MSD_ERR_ARG, "msd_set_formulation_kind: not with per-disk truncation orders");
        MsdFormulation w{};
        w.kind = kind;
        w.alpha = alpha;
        w.eta_ik = eta ? 0 : 1;
        w.eta = eta ? make_double2(eta[0], eta[1]) : make_double2(0.0, 0.0);
        pb->fw = w;
        pb->form = true;
        form_rows(pb);
        return MSD_OK;
    });
}

msd_status msd_formulation_weights(int kind, double alpha, const double* eta, double k, double* op_weights,
                                   double* rhs_weights, double* rep_weights) {
    return guarded([&]() -> msd_status {
        check_kind("msd_formulation_weights", kind, alpha, eta);
        if (!eta && (kind == MSD_FORM_CFIE || kind == MSD_FORM_BWIE) && !(k > 0.0 && std::isfinite(k)))
            fail(MSD_ERR_ARG, "msd_formulation_weights: eta = i k needs k > 0");
        const double2 e = eta ? make_double2(eta[0], eta[1]) : make_double2(0.0, k);
        for (int c = 0; c < 2; ++c) {
            double2 op[5], rhs[2], rep[2];
            msd_standard_weights(kind, alpha, e, c, op, rhs, rep);
            for (int o = 0; o < 5 && op_weights; ++o) {
                op_weights[(c * 5 + o) * 2] = op[o].x;
                op_weights[(c * 5 + o) * 2 + 1] = op[o].y;
            }
            for (int o = 0; o < 2 && rhs_weights; ++o) {
                rhs_weights[(c * 2 + o) * 2] = rhs[o].x;
                rhs_weights[(c * 2 + o) * 2 + 1] = rhs[o].y;
            }
            for (int o = 0; o < 2 && rep_weights && c == 0; ++o) {
                rep_weights[2 * o] = rep[o].x;
                rep_weights[2 * o + 1] = rep[o].y;
            }
        }
        return MSD_OK;
    });
}

msd_status msd_nearfield(msd_problem* pb, int config, const void* rho, int R, int64_t P, const double* points,
                         void* u_out) {
    return guarded([&]() -> msd_status {
        if (!pb || !rho || R <= 0 || P <= 0 || !points || !u_out || config < 0 || config >= pb->C)
            fail(MSD_ERR_ARG, "msd_nearfield: bad argument");
        const double2* d_rho = (const double2*)stage_in(pb, pb->nfbuf[0], rho, (size_t)pb->Ntot * R * 16);
        const double2* d_pts = (const double2*)stage_in(pb, pb->nfbuf[1], points, (size_t)P * 16);
        double2* W = (double2*)pb->nfbuf[2].get((size_t)pb->Ntot * R * 16);
        OutStage o(pb, pb->nfbuf[3], u_out, (size_t)P * R * 16);
        launch_nearfield(pb->d_cfg, config, pb->cfg[config], pb->d_centre, pb->d_radius, field_factor_of(pb), d_rho, R, W,
                         d_pts, P, (double2*)o.dev, pb->stream);
        CK_LAUNCH();
        o.finish();
        return MSD_OK;
    });
}

}  // extern "C"

namespace {

// T = conj(F)^T F and its eigenvalues for pb->C far-field matrices F (device,
// [C][n][n]); outputs to caller buffers (host or device, T_out may be NULL).
void dort_eigen(msd_problem* pb, int n, const double2* F, void* T_out, void* eig_out) {
    cudaStream_t s = pb->stream;
    const size_t nn = (size_t)pb->C * n * n;
    double2* T = (double2*)pb->dortbuf[3].get(nn * 16);
    double* eig = (double*)pb->dortbuf[4].get((size_t)pb->C * n * 8);
    void* work = pb->dortbuf[5].get(dort_work_bytes(pb->C, n));
    CK(dort_set_smem_limits(n));
    CK(launch_dort(pb->C, n, F, T, work, eig, &pb->h_pinned[10], s));
    CK_LAUNCH();
    auto out = [&](void* dst, const void* src, size_t bytes) {
        if (dst)
            CK(cudaMemcpyAsync(dst, src, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               s));
    };
    out(T_out, T, nn * 16);
    out(eig_out, eig, (size_t)pb->C * n * 8);
}

// After the stream reached dort_eigen's flag copy.
void dort_check(msd_problem* pb) {
    if (pb->h_pinned[10]) fail(MSD_ERR_CUDA, "msd_dort: a grid barrier of the tridiagonalisation timed out");
}

}  // namespace

extern "C" {

msd_status msd_dort(msd_problem* pb, int n_alpha, const msd_opts* opts, void* F_out, void* T_out, void* eig_out,
                    msd_stats* stats_host) {
    return guarded([&]() -> msd_status {
        if (!pb || n_alpha <= 0 || n_alpha > MSD_MAX_DORT || !eig_out) fail(MSD_ERR_ARG, "msd_dort: bad argument");
        const int n = n_alpha, C = pb->C;
        const double pi = 3.14159265358979323846;
        std::vector<double> betas((size_t)C * n), thetas(n);
        for (int j = 0; j < n; ++j) {
            const double a = 2.0 * pi * j / n;
            thetas[j] = a + pi;  // measured opposite to the emitting direction
            for (int c = 0; c < C; ++c) betas[(size_t)c * n + j] = a;
        }
        cudaStream_t s = pb->stream;
        const size_t nn = (size_t)C * n * n;
        double2* rho = (double2*)pb->dortbuf[0].get((size_t)pb->Ntot * n * 16);
        const msd_status st = solve_impl(pb, n, betas.data(), opts, rho, stats_host);
        double* d_th = (double*)pb->dortbuf[1].get((size_t)n * 8);
        CK(cudaMemcpyAsync(d_th, thetas.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
        double2* F = (double2*)pb->dortbuf[2].get(nn * 16);
        launch_farfield(pb->d_cfg, C, pb->cfg.data(), pb->d_centre, pb->d_radius, field_factor_of(pb), n, n, d_th, rho, nullptr,
                        F, s);
        CK_LAUNCH();
        if (F_out)
            CK(cudaMemcpyAsync(F_out, F, nn * 16,
                               is_device_ptr(F_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        dort_eigen(pb, n, F, T_out, eig_out);
        CK(cudaStreamSynchronize(s));
        dort_check(pb);
        return st;
    });
}

msd_status msd_dort_eigen(msd_problem* pb, int n_alpha, const void* F, void* T_out, void* eig_out) {
    return guarded([&]() -> msd_status {
        if (!pb || n_alpha <= 0 || n_alpha > MSD_MAX_DORT || !F || !eig_out)
            fail(MSD_ERR_ARG, "msd_dort_eigen: bad argument");
        const size_t nn = (size_t)pb->C * n_alpha * n_alpha;
        const double2* d_F = (const double2*)stage_in(pb, pb->dortbuf[2], F, nn * 16);
        dort_eigen(pb, n_alpha, d_F, T_out, eig_out);
        CK(cudaStreamSynchronize(pb->stream));
        dort_check(pb);
        return MSD_OK;
    });
}

msd_status msd_dort_eigenvectors(msd_problem* pb, int n_alpha, const void* F, int K, void* eig_out, void* vec_out) {
    return guarded([&]() -> msd_status {
        if (!pb || n_alpha <= 0 || n_alpha > MSD_MAX_DORT || !F || K <= 0 || K > n_alpha || !vec_out)
            fail(MSD_ERR_ARG, "msd_dort_eigenvectors: bad argument (1 <= K <= n_alpha)");
        const int n = n_alpha;
        const size_t nn = (size_t)pb->C * n * n;
        const double2* d_F = (const double2*)stage_in(pb, pb->dortbuf[2], F, nn * 16);
        dort_eigen(pb, n, d_F, nullptr, eig_out);  // eigenvalues (and the reduction kept in the work buffer)
        const double* eig = (const double*)pb->dortbuf[4].p;
        void* work = pb->dortbuf[5].p;
        void* scratch = pb->dortbuf[0].get(dort_vec_scratch_bytes(pb->C, n, K));
        OutStage o(pb, pb->dortbuf[1], vec_out, (size_t)pb->C * K * n * 16);
        CK(launch_dort_vectors(pb->C, n, K, work, eig, scratch, (double2*)o.dev, pb->stream));
        CK_LAUNCH();
        o.finish();
        CK(cudaStreamSynchronize(pb->stream));
        dort_check(pb);
        return MSD_OK;
    });
}

msd_status msd_herglotz_wave(msd_problem* pb, int config, int n_alpha, int K, const void* g, int64_t P,
                             const double* points, void* u_out) {
    return guarded([&]() -> msd_status {
        if (!pb || config < 0 || config >= pb->C || n_alpha <= 0 || K <= 0 || !g || P <= 0 || !points || !u_out)
            fail(MSD_ERR_ARG, "msd_herglotz_wave: bad argument");
        const double2* d_g = (const double2*)stage_in(pb, pb->nfbuf[0], g, (size_t)K * n_alpha * 16);
        const double2* d_pts = (const double2*)stage_in(pb, pb->nfbuf[1], points, (size_t)P * 16);
        OutStage o(pb, pb->nfbuf[3], u_out, (size_t)P * K * 16);
        launch_herglotz(pb->cfg[config].k, n_alpha, K, d_g, P, d_pts, (double2*)o.dev, pb->stream);
        CK_LAUNCH();
        o.finish();
        return MSD_OK;
    });
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free product
//
// msd_matvec_noalloc: the block-Toeplitz product of msd_matvec for callers
// that may not allocate device memory when they call it.  Its work list,
// scaled-input buffer and per-split partial sums live in one file-scope
// device array instead of library buffers obtained from cudaMalloc.

namespace {

constexpr size_t kStaticScratchBytes = 32ull << 20;  // 32 MiB held by every GPU that loads the library
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch, per device (host code may not take
// the address of a __device__ variable directly).
void* g_static_scratch_dev[kMaxDevices] = {};

// Work list of the product (configuration-major, then target tile, then
// source split), written on the device so that no host buffer is needed.
__global__ void k_fill_static_work(const MsdConfig* __restrict__ cfg, int C, int ns, int nwork,
                                   MatvecWork* __restrict__ out) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwork) return;
    const int w0 = w;
    for (int c = 0; c < C; ++c) {
        const int cnt = (cfg[c].Mp / MSD_TILE_P) * ns;
        if (w < cnt) {
            const int tile = w / ns, split = w % ns, M = cfg[c].M;
            MatvecWork x;
            x.cfg = c;
            x.p0 = tile * MSD_TILE_P;
            x.q0 = (int)((long long)M * split / ns);
            x.q1 = (int)((long long)M * (split + 1) / ns);
            x.split = split;
            x.pad = 0;
            out[w0] = x;
            return;
        }
        w -= cnt;
    }
}

void* static_scratch_address() {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(MSD_ERR_ARG, "msd_matvec_noalloc: device index out of range");
    if (!g_static_scratch_dev[dev]) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_static_scratch));
        g_static_scratch_dev[dev] = p;
    }
    return g_static_scratch_dev[dev];
}

}  // namespace

extern "C" msd_status msd_matvec_noalloc(msd_problem* pb, int R, int precision, const void* x_dev, void* y_dev) {
    return guarded([&]() -> msd_status {
        if (!pb || R <= 0 || !x_dev || !y_dev) fail(MSD_ERR_ARG, "msd_matvec_noalloc: bad argument");
        if (precision != MSD_FP64 && precision != MSD_FP32) fail(MSD_ERR_ARG, "msd_matvec_noalloc: precision");
        if (!is_device_ptr(x_dev) || !is_device_ptr(y_dev))
            fail(MSD_ERR_ARG, "msd_matvec_noalloc: x and y must be device memory");
        if (ranges_overlap(x_dev, y_dev, (size_t)pb->Ntot * R * (precision == MSD_FP64 ? 16 : 8)))
            fail(MSD_ERR_ARG, "msd_matvec_noalloc: x and y must not overlap");
        if (pb->form) fail(MSD_ERR_ARG, "msd_matvec_noalloc: needs the default formulation");
        const bool fp64 = precision == MSD_FP64;
        if ((fp64 && !pb->d_G64) || (!fp64 && !pb->d_G32))
            fail(MSD_ERR_ARG, "msd_matvec_noalloc: the generators of this precision are not built yet "
                              "(call msd_matvec or msd_solve_planewaves once first)");
        const MatvecChoice dc = matvec_default_choice(R, pb->Nmax, fp64);
        if (matvec_smem_bytes(dc, pb->Nmax, fp64) > kMatvecSmemCap)
            fail(MSD_ERR_ARG, "msd_matvec_noalloc: truncation order too large for the shared-memory tile");
        unsigned char* base = (unsigned char*)static_scratch_address();
        // layout: [work list][xs][partials], each 256-byte aligned
        const size_t elem = fp64 ? 16 : 8;
        const size_t vec = (size_t)pb->Ntot * R * elem;
        long long tiles = 0;
        for (auto& c : pb->cfg) tiles += c.Mp / MSD_TILE_P;
        auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
        auto need = [&](int ns) { return up((size_t)tiles * ns * sizeof(MatvecWork)) + up(vec) + (size_t)ns * vec; };
        if (need(1) > kStaticScratchBytes)
            fail(MSD_ERR_ARG, "msd_matvec_noalloc: N_tot * R too large for the 32 MiB static work area");
        // source splits: as many as fill one wave of resident CTAs and fit
        int sms = 0, dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const long long slots = (long long)sms * matvec_blocks_per_sm(dc, pb->Nmax, fp64);
        const long long units = tiles * (R / dc.RT);
        int ns = (int)std::max<long long>(1, std::min<long long>(slots / std::max<long long>(1, units),
                                                                 std::max(1, pb->Mmax / 2)));
        while (ns > 1 && need(ns) > kStaticScratchBytes) --ns;
        const int nwork = (int)(tiles * ns);
        MatvecWork* work = (MatvecWork*)base;
        unsigned char* xs = base + up((size_t)nwork * sizeof(MatvecWork));
        unsigned char* part = xs + up(vec);
        k_fill_static_work<<<(nwork + 127) / 128, 128, 0, pb->stream>>>(pb->d_cfg, pb->C, ns, nwork, work);
        g_msd_launches += 1;
        CK_LAUNCH();
        // every (split, row, column) of the partials and every element of xs
        // is written by this call before it is read, so no clearing is needed
        if (fp64)
            launch_matvec_f64(pb->d_cfg, work, nwork, pb->Nmax, pb->d_G64, pb->d_rf64, pb->d_lf64, pb->Ntot, R,
                              (const double2*)x_dev, (double2*)xs, (double2*)part, ns, (double2*)y_dev, pb->stream,
                              nullptr, nullptr);
        else
            launch_matvec_f32(pb->d_cfg, work, nwork, pb->Nmax, pb->d_G32, pb->d_rf32, pb->d_lf32, pb->Ntot, R,
                              (const float2*)x_dev, (float2*)xs, (float2*)part, ns, (float2*)y_dev, pb->stream,
                              nullptr, nullptr);
        CK_LAUNCH();
        return MSD_OK;
    });
}
