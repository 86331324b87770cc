// Internal declarations shared by the CUDA translation units of libmsd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/msd.h"

// ---------------------------------------------------------------- complex helpers

__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) {
    return make_double2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) {
    return make_double2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) {
    return make_double2(a.x * s, a.y * s);
}
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    // Smith's algorithm (avoids overflow of |b|^2 for large |b|)
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.y + b.x * r;
        return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
__host__ __device__ __forceinline__ double2 cinv(double2 b) { return cdiv(make_double2(1.0, 0.0), b); }

// acc += a * b (complex multiply-accumulate, 4 FMAs)
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// ---------------------------------------------------------------- problem layout

// One batched configuration.  Rows of configuration c occupy
// [row_off, row_off + M*n); generators of c occupy M*Mp*L complex values
// starting at gen_off, laid out [q][p][l + 2N] with p padded to Mp.
struct MsdConfig {
    double k;
    int N, n, L;      // truncation, modes per disk (2N+1), generator length (4N+1)
    int M, Mp;        // disks, disks padded to a multiple of 32
    int disk_off;     // first global disk index
    int Mq;           // disks padded to a multiple of 8 (sources of the shift-GEMM product)
    long long row_off;  // first unknown row
    long long gen_off;  // first generator element
    // shift-GEMM tensor-core product (k_matvec_tcs.cu): first float of this
    // configuration's generators in the A-operand order, and the sum of
    // Mq * n over the configurations before it (its source rows per column)
    long long gt_off;
    long long xrow_off;
};

// One CTA of the block-Toeplitz product: a tile of 32 target disks
// [p0, p0+32) of configuration cfg, summed over sources [q0, q1), writing
// its raw sums into partial slot `split` (pad = 0) or adding them to it
// (pad = 1: a later source block of a product with recomputed generators).
struct MatvecWork {
    int cfg, p0, q0, q1, split, pad;
};

// A contiguous range of rows of one configuration (reduction chunk).
struct RowChunk {
    int cfg;
    int pad;
    long long row0, row1;
};

#define MSD_TILE_P 32

// Tile shape of one product kernel instance: register window KB (modes per
// thread), column tile RT and register column block RB, I = ceil(n / KB)
// thread rows; or the tensor-core kernel (TC > 0, FP32, R % TC == 0).  matvec_default_choice is the cost model; the autotuner in
// the problem's plan times matvec_candidates and keeps the fastest.
struct MatvecChoice {
    int KB, RT, RB, I;
    int TC;  // > 0: tensor-core kernel with TC columns per CTA (KB, RB, I unused; RT = TC)
    int P2;  // FP32: 1 = complex multiply-adds as paired FMAs (fma.rn.f32x2), 0 = four FFMAs
    int SH;  // shift-GEMM tensor-core kernel (FP32, RT = MSD_TCS_COLS columns per CTA): 1 = mode
             // blocks of <= 8 two per CTA, 2 = one block of <= 16 modes per CTA; 0 = not used
    int ONE;  // FP64: 1 = one shared-memory stage (two would exceed 227 KB at this truncation order)
};
#define MSD_TCS_COLS 8
MatvecChoice matvec_default_choice(int R, int Nmax, bool fp64);
// allow_sh: include the shift-GEMM kernel (forward products with stored
// generators of the default rows only)
int matvec_candidates(int R, int Nmax, bool fp64, MatvecChoice* out, int cap, bool allow_sh = false);
size_t matvec_smem_bytes(const MatvecChoice& c, int Nmax, bool fp64);
int matvec_blocks_per_sm(const MatvecChoice& c, int Nmax, bool fp64);
// tensor-core product (k_matvec_tc.cu): targets in tiles of floor(128 / n)
// disks that never cross a 32-disk boundary
bool tc_supported(int R, int Nmax, int RC);
int tc_tile_disks(int n);
size_t tc_smem_bytes(int RC);
void launch_bt_tc(int RC, const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, const float2* G,
                  const float2* xs, float2* part, long long Ntot, int R, cudaStream_t s, const int* live = nullptr);
int tc_status_and_clear();
// shift-GEMM tensor-core product (k_matvec_tcs.cu): GT = generators in the
// A-operand order (built from the complex64 generators), XT = scaled columns
// in the slab order (built from x each product); work items: p0 a multiple
// of 128, q0/q1 source range, pad = m0 | mb << 8 | nmb << 12 (first mode,
// modes per block, blocks)
size_t tcs_smem_bytes(int Nmax);
bool tcs_supported(int R, int Nmax);
// blocks of <= 8 modes grouped two per CTA (N = 16 mb <= 128 per MMA), or
// wide: one block of <= 16 modes per CTA (N <= 256 per MMA)
void tcs_mode_blocks(int n, int* mb, int* nblocks, bool wide);
// live: NULL, or active flags [C*R]; a CTA whose columns are all inactive
// writes zero raw sums and does no other work (the caller reads none of
// those columns)
void launch_bt_tcs(const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, int Nmax, const float* GT,
                   const float* XT, float2* part, long long Ntot, int R, cudaStream_t s,
                   const int* live = nullptr);
void launch_tcs_build_gt(const MsdConfig* d_cfg, int C, const long long* d_blk_off, long long nblocks,
                         const float2* G32, float* GT, cudaStream_t s);
void launch_tcs_prep_x(const MsdConfig* d_cfg, int C, long long rows4, int R, const float* rf, const float2* x,
                       float* XT, cudaStream_t s);
// Dynamic shared memory of one CUDA-core product CTA at most (227 KB per
// CTA less the kernel's static mbarriers, rounded down to 1 KB).
constexpr size_t kMatvecSmemCap = 226 * 1024;
// bit 0 set (and cleared): a bulk-copy wait of the CUDA-core product expired
int bt_status_and_clear();
int tcs_status_and_clear();
// Set by msd_test_expire_waits: kernels with bounded waits take their
// expiry path once per launch (tests of the error path; no fault involved).
extern std::atomic<int> g_msd_expire_waits;  // bit 0: a pipeline wait of the tensor-core kernel expired
// the pieces of a product: xs = r .* x; y = x + l .* sum of the partials
void launch_scale_cols(bool fp64, long long Ntot, int R, const void* rf, const void* x, void* xs, cudaStream_t s);
void launch_finalize(bool fp64, long long Ntot, int R, int nsplit, const void* lf, const void* x, const void* part,
                     void* y, cudaStream_t s);
// the Toeplitz kernel alone on pre-scaled columns xs (autotuner timing,
// recomputed products); work items with pad != 0 add to their partial slot
void launch_bt_only(const MatvecChoice& c, bool fp64, const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork,
                    int Nmax, const void* G, const void* xs, void* part, long long Ntot, int R, cudaStream_t s);

// Number of kernels the library has launched (host-side counter, all threads).
extern std::atomic<long long> g_msd_launches;

// ---------------------------------------------------------------- launchers (one per kernel family)

// K1: Bessel diagonals and the row/column factors of the preconditioned operator.
void launch_disk_diagonals(const MsdConfig* d_cfg, int Mtot, const int* d_disk_cfg,
                           const double* d_radius, const int8_t* d_bc, int Nmax,
                           double2* J, double2* dJ, double2* H, double2* dH,
                           double2* lf64, double* rf64, float2* lf32, float* rf32,
                           double2* rhs_scale, int* d_flags, cudaStream_t s);

// K2: Toeplitz generators of the ordered pairs of a list of blocks
// (configuration, target range [P0, P0+Pc), source range [Q0, Q0+Qb)),
// complex128 and/or complex64, block e at out[out_off + ((q-Q0) Pc + p-P0) L].
// item_off is the running count of (q, p) items before the block.
struct GenBlock {
    int cfg, P0, Pc, Q0, Qb, pad;
    long long item_off, out_off;
};
// f32_math: complex64-only output with FP32 arithmetic for the far pairs
void launch_generator_blocks(const MsdConfig* d_cfg, const GenBlock* d_blocks, int nblocks, long long nitems,
                             const double2* d_centre, double2* G64, float2* G32, int* d_flags, cudaStream_t s,
                             bool f32_math = false);

// ||P u||^2 and ||P v||^2 per (row chunk, column) with the preconditioner's
// diagonal P (unpreconditioned residual norms); R <= 64.
// diag (may be NULL): the self-block diagonal P of a formulation; NULL takes
// the default rows' P from J, H, H'.
void launch_weighted_norms(const MsdConfig* d_cfg, const RowChunk* d_chunks, int nchunk, int R,
                           const double* d_radius, const int8_t* d_bc, const double2* J, const double2* H,
                           const double2* dH, const double2* diag, const double2* u, const double2* v,
                           double2* part, cudaStream_t s);

// Penetrable obstacles (section 7): per parent row the 2 x 2 factor A =
// B^-1 C of the combined product (A64, A32 [Ntot][4]: A11, A12, A21, A22) and
// the right-hand-side scales S64 [2][Ntot] (B^-1 [-J+; -k+ J+']), from the
// Bessel diagonals at k+ (p) and k- (m) and mu per disk; flags bit 0 when a
// factor is not finite.
void launch_pen_rows(const MsdConfig* cfg_p, const MsdConfig* cfg_m, int Mtot, long long Ntot, const int* disk_cfg,
                     const double* radius, const double* mu, const double2* Jp, const double2* dJp,
                     const double2* Hp, const double2* dHp, const double2* Jm, const double2* dJm,
                     const double2* Hm, const double2* dHm, double2* A64, float2* A32, double2* S64, int* flags,
                     cudaStream_t s);
// xs+- = sqrt(a) J+- rho+- (parent layout) from x in the transmission layout
void launch_pen_scale(bool fp64, const MsdConfig* cfg, int C, long long Ntot, int R, const void* rfp,
                      const void* rfm, const void* x, void* xsp, void* xsm, cudaStream_t s);
// y = x + A [z+; z-] in the transmission layout
void launch_pen_finalize(bool fp64, const MsdConfig* cfg, int C, long long Ntot, int R, const void* A, const void* x,
                         const void* partp, int nsp, const void* partm, int nsm, void* y, cudaStream_t s);
// transmission layout <-> (rho+, rho-) in the parent layout (FP64)
void launch_pen_layout(const MsdConfig* cfg, int C, long long Ntot, int R, bool to_pen, double2* pen, double2* xp,
                       double2* xm, cudaStream_t s);

// Per-disk truncation N_p <= N (section 5): zero the row factors l, the
// column factors r and the right-hand-side scale of the rows |m| > N_p.
void launch_mask_rows(const MsdConfig* d_cfg, int Mtot, const int* d_disk_cfg, const int* d_Np, double2* lf64,
                      float2* lf32, double* rf64, float* rf32, double2* rhs_scale, cudaStream_t s);

// Integral-equation formulation (sections 3, 4.2, 5): per boundary
// condition c (0 Dirichlet, 1 Neumann) the weights of I, L, M, N, D in the
// rows of its disks and of U, dU in their right-hand side, and the weights
// of the single- and double-layer potentials in the field representation.
struct MsdFormulation {
    double2 op[2][5];
    double2 rhs[2][2];
    double2 rep[2];
    // kind >= 0 (MSD_FORM_*): the weights above are ignored and each row
    // takes those of the named formulation (msd_standard_weights) with
    // alpha, and eta or, when eta_ik is set, i k of the row's configuration.
    int kind = -1;
    int eta_ik = 0;
    double alpha = 0.0;
    double2 eta = {0.0, 0.0};
};

// Weights of a named formulation (section 3 integral equations; the
// Brakhage-Werner sound-hard rows are the normal trace of its
// representation) for the rows of boundary condition cls: op[5] = weights
// of I, L, M, N, D, rhs[2] = weights of U, dU, rep[2] = weights of L, M in
// the field representation.  Returns false for an unknown kind.
__host__ __device__ inline bool msd_standard_weights(int kind, double alpha, double2 eta, int cls, double2 op[5],
                                                     double2 rhs[2], double2 rep[2]) {
    const double2 z = make_double2(0.0, 0.0), one = make_double2(1.0, 0.0);
    for (int o = 0; o < 5; ++o) op[o] = z;
    rhs[0] = rhs[1] = z;
    rep[0] = one;
    rep[1] = z;
    if (kind == MSD_FORM_BWIE) {
        // u = -(eta L + M) psi: trace (I/2 - eta L - M) psi = -U on sound-soft
        // rows, normal trace (eta I/2 - eta N - D) psi = -dU on sound-hard rows
        rep[0] = make_double2(-eta.x, -eta.y);
        rep[1] = make_double2(-1.0, 0.0);
        if (cls == MSD_DIRICHLET) {
            op[0] = make_double2(0.5, 0.0);
            op[1] = make_double2(-eta.x, -eta.y);
            op[2] = make_double2(-1.0, 0.0);
            rhs[0] = one;
        } else {
            op[0] = make_double2(0.5 * eta.x, 0.5 * eta.y);
            op[3] = make_double2(-eta.x, -eta.y);
            op[4] = make_double2(-1.0, 0.0);
            rhs[1] = one;
        }
        return true;
    }
    if (kind != MSD_FORM_EFIE && kind != MSD_FORM_MFIE && kind != MSD_FORM_CFIE) return false;
    if (cls == MSD_NEUMANN) {  // single-layer representations: (-I/2 + N) rho = -dU
        op[0] = make_double2(-0.5, 0.0);
        op[3] = one;
        rhs[1] = one;
        return true;
    }
    if (kind == MSD_FORM_EFIE) {  // L rho = -U
        op[1] = one;
        rhs[0] = one;
    } else if (kind == MSD_FORM_MFIE) {  // (I/2 + N) rho = -dU
        op[0] = make_double2(0.5, 0.0);
        op[3] = one;
        rhs[1] = one;
    } else {  // CFIE: alpha eta L + (1 - alpha)(I/2 + N) = -(alpha eta U + (1 - alpha) dU)
        const double2 ae = make_double2(alpha * eta.x, alpha * eta.y);
        op[0] = make_double2(0.5 * (1.0 - alpha), 0.0);
        op[1] = ae;
        op[3] = make_double2(1.0 - alpha, 0.0);
        rhs[0] = ae;
        rhs[1] = make_double2(1.0 - alpha, 0.0);
    }
    return true;
}
// Per-row factors: l1, l2 (FP64, FP32) of the combined product, rf2 =
// sqrt(a) J', the right-hand-side scale -(w_U J + k w_dU J')/P, the field
// factor w_L' J - k w_M' J' and the self-block diagonal P.  d_flags bit 0 is
// set when a factor is not finite (P = 0).
void launch_form_rows(const MsdConfig* d_cfg, int Mtot, const int* d_disk_cfg, const double* d_radius,
                      const int8_t* d_bc, const double2* J, const double2* dJ, const double2* H, const double2* dH,
                      const MsdFormulation& w, double2* l1_64, double2* l2_64, float2* l1_32, float2* l2_32,
                      double* rf2_64, float* rf2_32, double2* rhs_scale, double2* ff, double2* diag, int* d_flags,
                      cudaStream_t s);
// xs [Ntot][2R] = (rf .* x | rf2 .* x);  y = x + l1 .* sum part[:, :, 0:R] + l2 .* sum part[:, :, R:2R]
void launch_form_scale(bool fp64, long long Ntot, int R, const void* rf, const void* rf2, const void* x, void* xs,
                       cudaStream_t s);
void launch_form_finalize(bool fp64, long long Ntot, int R, int nsplit, const void* l1, const void* l2,
                          const void* x, const void* part, void* y, cudaStream_t s);

// Near field (Prop. 4.3): u(points)[r] of configuration ci for densities rho
// [N_tot][R]; W is a work buffer of N_tot * R complex128.
// J: the per-row field factor (the Bessel diagonal J for u = L rho, or a
// formulation's w_L J - k w_M J').
void launch_nearfield(const MsdConfig* d_cfg, int ci, const MsdConfig& h_cfg, const double2* d_centre,
                      const double* d_radius, const double2* J, const double2* rho, int R, double2* W,
                      const double2* d_pts, long long P, double2* out, cudaStream_t s);

// Interior field of penetrable obstacles: u- = L- rho- at points inside the
// disks of configuration ci (0 outside), k- = km, Jm / Hm the Bessel
// diagonals at k- (the internal problem's J and H), W, V work buffers of
// N_tot * R complex128 each.
void launch_nearfield_inside(const MsdConfig* d_cfg, int ci, const MsdConfig& h_cfg, double km, const double2* d_centre,
                             const double* d_radius, const double2* Jm, const double2* Hm, const double2* rho_minus,
                             int R, double2* W, double2* V, const double2* d_pts, long long P, double2* out,
                             cudaStream_t s);

// K5': preconditioned point-source right-hand sides, sources [C][R] (x, y).
void launch_rhs_pointsource(const MsdConfig* d_cfg, int Mtot, const int* d_disk_cfg, const double2* d_centre,
                            const double* d_radius, const double2* rhs_scale, int R, const double2* d_src,
                            double2* out, cudaStream_t s);

// K5: preconditioned plane-wave right-hand sides.
void launch_rhs_planewave(const MsdConfig* d_cfg, int Mtot, const int* d_disk_cfg,
                          const double2* d_centre, const double* d_radius,
                          const double2* rhs_scale, int Nmax, int R, const double* d_betas,
                          double2* out, cudaStream_t s);

// K3: block-Toeplitz product y = x + l .* sum_q T(g^pq) (r .* x).
void launch_matvec_f64(const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, int Nmax,
                       const double2* G, const double* rf, const double2* lf, long long Ntot,
                       int R, const double2* x, double2* xs, double2* part, int nsplit,
                       double2* y, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
                       const MatvecChoice* ch = nullptr, const int* live = nullptr);
// xs_ready: xs already holds rf .* x (written by the step that made x)
void launch_matvec_f32(const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, int Nmax,
                       const float2* G, const float* rf, const float2* lf, long long Ntot,
                       int R, const float2* x, float2* xs, float2* part, int nsplit,
                       float2* y, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
                       const MatvecChoice* ch = nullptr, const int* live = nullptr, bool xs_ready = false);

// K6: far field.
// Time reversal (section 7): T = conj(F)^T F for C far-field matrices
// F [C][n][n] and the eigenvalues of every T, largest first (eig [C][n]).
// work: dort_work_bytes(C, n) bytes.  dort_set_smem_limits(n) once before
// the first launch with that n.  *err_flag (host) receives, once the stream
// reaches it, 1 if a grid-barrier wait of the tridiagonalisation expired.
size_t dort_work_bytes(int C, int n);
cudaError_t dort_set_smem_limits(int n);
cudaError_t launch_dort(int C, int n, const double2* F, double2* T, void* work, double* eig, int* err_flag,
                        cudaStream_t s);
// Eigenvectors of the K largest eigenvalues of every T after launch_dort
// (same work buffer): U [C][K][n], unit norm, largest entry real positive.
size_t dort_vec_scratch_bytes(int C, int n, int K);
cudaError_t launch_dort_vectors(int C, int n, int K, void* work, const double* eig, void* scratch, double2* U,
                                cudaStream_t s);
// Discrete Herglotz waves of K parameter vectors g [K][na] at points [P]:
// out [P][K] = (2 pi / na) sum_j g_j exp(i k x . (cos a_j, sin a_j)), a_j = 2 pi j / na.
void launch_herglotz(double k, int na, int K, const double2* g, long long P, const double2* pts, double2* out,
                     cudaStream_t s);

// J: the per-row field factor, as for launch_nearfield.
void launch_farfield(const MsdConfig* d_cfg, int C, const MsdConfig* h_cfg,
                     const double2* d_centre, const double* d_radius, const double2* J,
                     int R, int T, const double* d_thetas, const double2* rho,
                     double2* part, double2* F, cudaStream_t s);

// ---------------------------------------------------------------- K4 (GMRES) pieces
// A "system" is one (configuration, column) pair: s = cfg*R + r.

struct GmresDims {
    long long Ntot;   // rows
    int R;            // columns
    int C;            // configurations
    int S;            // systems = C*R
    int m;            // restart length
    int nchunk;       // reduction chunks
};

// out[s][i] = sum over the rows of cfg(s) of conj(u_i) w for u = V_0..V_{nv-1}
// (and w itself when self = 1); systems with skip[s] == skipval get zeros
// (skipval 1 with a skip-flag array, 0 with the active flags: inactive
// systems have zero vectors, so skipping them changes no value).
//
// With `fuse` and at most kFuseMaxSystems systems, and fuse->wn2 set (self =
// 1, ||w||^2 lands at index j + 1), the reduction also writes
// wn2[s * ostride] = ||w||^2 - sum_{i <= j} |out_i|^2, the squared norm after
// the projection, and with fuse->skip2 set the re-orthogonalisation flags of
// gm_reorth_flags; the call then returns true.  For a single group of eight
// vectors (R dividing 32 or R = 64) the reduction runs inside the projection
// kernel, else in its reduction kernel.  fuse->cnt: ncnt + 1 zeroed device
// counters, left zeroed by every launch that uses them.
constexpr int kFuseMaxSystems = 8;
struct GmDotsFuse {
    int* cnt = nullptr;
    int ncnt = 0;
    int j = 0;
    double2* wn2 = nullptr;
    const int* active = nullptr;
    int* skip2 = nullptr;
    double eta2 = 0.5;  // re-orthogonalisation threshold (msd_opts.reorth)
};
template <typename V>
bool gm_dots(const GmresDims& d, const RowChunk* chunks, const int* cfg_chunk_off, const V* Vb, long long vstride,
             int nv, int self, const V* w, const int* skip, double2* part, double2* out, int ostride,
             cudaStream_t s, int skipval = 1, const GmDotsFuse* fuse = nullptr);
// w += sign * sum_i V_i h[s][i]  (skip[s] == skipval: unchanged)
template <typename V, typename W>
void gm_update(const GmresDims& d, const RowChunk* chunks, const V* Vb, long long vstride, int nv, const double2* h,
               int hstride, const int* skip, double sign, W* w, cudaStream_t s, int skipval = 1);
// v = w * scale[s] for active systems, 0 otherwise
template <typename Vin, typename Vout>
// (rf, xs: also xs = rf .* v, the scaled input of the next FP32 product)
void gm_scale(const GmresDims& d, const RowChunk* chunks, const Vin* w, const double* scale, const int* active,
              Vout* v, cudaStream_t s, const float* rf = nullptr, float2* xs = nullptr);
// ||w'||^2 estimate (written to wn2) and the re-orthogonalisation flags
void gm_reorth_flags(const GmresDims& d, const double2* h1, int hstride, int j, double2* wn2,
                     const int* active, int* skip2, cudaStream_t s, double eta2 = 0.5);
void gm_start(const GmresDims& d, const double2* rr, int hstride, const double* tol_abs, double* beta,
              double* vscale, double2* g, int* active, int* kconv, int* any_active, cudaStream_t s);
void gm_givens(const GmresDims& d, int j, const double2* h1, const double2* h2, int hstride, const double2* wn2a,
               const double2* wn2b, const int* skip2, const double* tol_cycle, double2* H, double2* cs,
               double2* sn, double2* g, double* vscale, int* active, int* kconv, int* iters, int* any_active,
               int* nonfinite, double2* rdiag, bool fp32_maps, cudaStream_t s);
// end of a cycle: rotate the stored raw columns into R (in place), then back-substitute
void gm_lsq(const GmresDims& d, double2* H, const double2* cs, const double2* sn, const double2* rdiag,
            const double2* g, const int* kconv, double2* y, double2* work, cudaStream_t s);
void gm_residual(long long n, const double2* b, const double2* Ax, double2* r, cudaStream_t s);
void gm_zero(long long n, double2* x, cudaStream_t s);

// ---------------------------------------------------------------- K3 with other scalings, K7
void launch_product_f64(const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, int Nmax, const double2* G,
                        const double* col_r, const double2* col_c, const double* row_r, const double2* row_c,
                        int add_x, long long Ntot, int R, const double2* x, double2* xs, double2* part, int nsplit,
                        double2* y, cudaStream_t s, const MatvecChoice* ch = nullptr);
void launch_product_f32(const MsdConfig* d_cfg, const MatvecWork* d_work, int nwork, int Nmax, const float2* G,
                        const float* col_r, const float2* col_c, const float* row_r, const float2* row_c,
                        int add_x, long long Ntot, int R, const float2* x, float2* xs, float2* part, int nsplit,
                        float2* y, cudaStream_t s, const MatvecChoice* ch = nullptr);
void launch_adjoint_generators_f64(const MsdConfig* d_cfg, int C, const MsdConfig* h_cfg, const double2* G,
                                   double2* GA, cudaStream_t s);
void launch_adjoint_generators_f32(const MsdConfig* d_cfg, int C, const MsdConfig* h_cfg, const float2* G,
                                   float2* GA, cudaStream_t s);
void launch_conj_rows(long long n, const double2* a, double2* ca, float2* ca32, cudaStream_t s);
void launch_ff_table(const MsdConfig* d_cfg, int C, int nmax, int T, const double* th, double2* E, cudaStream_t s);
void launch_misfit(int C, int T, int R, const double2* F, const double2* Ft, double2* w, double* J, cudaStream_t s);
void launch_farfield_adj(const MsdConfig* d_cfg, int Mtot, const int* disk_cfg, const double2* centre,
                         const double* radius, const double2* J, int nmax, int T, int R, const double* th,
                         const double2* E, const double2* w, double2* u, cudaStream_t s);
void launch_farfield_grad(const MsdConfig* d_cfg, int Mtot, const int* disk_cfg, const double2* centre,
                          const double* radius, const double2* J, const double2* dJ, int nmax, int T, int R,
                          const double* th, const double2* E, const double2* w, const double2* rho, double* gO,
                          double* ga, double* gk, cudaStream_t s);
void launch_pair_grad(const MsdConfig* d_cfg, int C, const MsdConfig* h_cfg, const double2* centre, const double2* G,
                      int R, const double2* muh, const double2* rhoh, double* gO, double* gk, cudaStream_t s);
void launch_grad_rows(const MsdConfig* d_cfg, int Mtot, const int* disk_cfg, const double2* centre,
                      const double* radius, const int8_t* bc, const double2* J, const double2* dJ, const double2* H,
                      const double2* dH, int R, const double* betas, const double2* mu, const double2* rho,
                      const double2* sv, const double2* tv, double* gO, double* ga, double* gk, cudaStream_t s);
void launch_scale_pair_inputs(long long Ntot, int R, const double2* lf, const double* rf, const double2* mu,
                              const double2* rho, double2* muh, double2* rhoh, cudaStream_t s);
